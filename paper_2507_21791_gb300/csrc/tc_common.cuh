// Device helpers shared by the tensor-core kernels (gram_tc.cu, proj_tc.cu):
// tcgen05 descriptors and MMA issue, bounded mbarrier polling, and the exact
// splitting of an FP64 value into nine 7-bit digits relative to an exponent
// (error-free splitting in the manner of Ozaki, Ogita, Oishi and Rump,
// Numer. Algorithms 59, 2012).
#pragma once

#include "bcgs_internal.cuh"

namespace bcgs {
namespace tc {

constexpr int kDigits = 9;
constexpr long long kWaitCycles = 2000000000LL;  // about one second at GB300 clocks

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(phase));
  return ok != 0;
}

template <typename T>
__device__ __forceinline__ double ld_elem(const void* base, int64_t idx) {
  return (double)__ldg(reinterpret_cast<const T*>(base) + idx);
}

// 63-bit fixed-point magnitude of a relative to the column exponent field
// `cexp` (the biased exponent of the column's max |a|): N = |a| 2^(63 - E),
// E = cexp - 1022.  neg receives the sign bit.
__device__ __forceinline__ uint64_t fixed63(double a, int cexp, uint32_t& neg) {
  const uint64_t bits = (uint64_t)__double_as_longlong(a);
  neg = (uint32_t)(bits >> 63);
  const int e = (int)((bits >> 52) & 0x7FF);
  if (e == 0) return 0;  // zero or subnormal
  const uint64_t mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = e - cexp + 10;  // <= 10 because |a| <= max
  if (sh >= 0) return mant << (sh > 10 ? 10 : sh);
  return -sh < 64 ? (mant >> (-sh)) : 0;
}

// bf16 bit pattern of the signed integer (neg ? -d : d), 0 <= d < 128:
// (2^23 + d) - 2^23 in fp32 with the sign folded into both operands.
__device__ __forceinline__ uint32_t digit_f32(uint32_t d, uint32_t neg) {
  const float big = __int_as_float((int)(0x4B000000u | d | (neg << 31)));
  const float off = __int_as_float((int)(0xCB000000u ^ (neg << 31)));
  return __float_as_uint(big + off);
}

// Split 8 consecutive rows of one column into the 9 digit tiles: tile t gets
// the 16 bytes (8 bf16) at row `row` (the MMA M/N index), 16-byte chunk `g`,
// swizzled as SW128 expects (chunk ^ (row % 8)).
__device__ __forceinline__ void split8(const double (&v)[8], int cexp, uint8_t* tiles, int tile_bytes,
                                       int row, int g) {
  uint64_t N[8];
  uint32_t ng[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) N[e] = fixed63(v[e], cexp, ng[e]);
  const int off = row * 128 + ((g ^ (row & 7)) << 4);
#pragma unroll
  for (int t = 0; t < kDigits; ++t) {
    const int sh = 56 - 7 * t;
    uint32_t w[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const uint32_t d0 = (uint32_t)(N[2 * p] >> sh) & 0x7Fu;
      const uint32_t d1 = (uint32_t)(N[2 * p + 1] >> sh) & 0x7Fu;
      w[p] = __byte_perm(digit_f32(d0, ng[2 * p]), digit_f32(d1, ng[2 * p + 1]), 0x7632);
    }
    *reinterpret_cast<uint4*>(tiles + t * tile_bytes + off) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}


__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n");
}

// Fold nine exact level sums L_l (|L_l| <= (l+1) 64 127^2 < (l+1) 2^20) into the
// two int64 accumulators: hi += sum_{l<=4} L_l 2^(7(4-l)), lo += sum_{l>=5} L_l 2^(7(8-l)).
__device__ __forceinline__ void fold_levels(const int32_t (&L)[kDigits], long long& hi, long long& lo) {
  const int32_t c01 = (L[0] << 7) + L[1];
  const int32_t c23 = (L[2] << 7) + L[3];
  const int32_t c56 = (L[5] << 7) + L[6];
  const int32_t c78 = (L[7] << 7) + L[8];
  hi += ((long long)c01 << 21) + ((long long)c23 << 7) + (long long)L[4];
  lo += ((long long)c56 << 14) + (long long)c78;
}

// The value 2^(E_a + E_b - 70) (hi 2^28 + lo), with E = cexp - 1022.
__device__ __forceinline__ double unfold(long long hi, long long lo, int cexp_a, int cexp_b) {
  const int sc = cexp_a + cexp_b - 2044;
  return ldexp((double)hi, sc - 42) + ldexp((double)lo, sc - 70);
}

// Tensor-memory allocation of NCOLS (power of two, 32..512) columns by one warp.
template <int NCOLS>
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(dst_smem)),
               "n"(NCOLS));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
}
template <int NCOLS>
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "n"(NCOLS));
}
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
      smem_u32(mbar)));
}
__device__ __forceinline__ void mbar_init(uint64_t* mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)));
  asm volatile("fence.mbarrier_init.release.cluster;\n");
}
// Poll the barrier's phase `phase` for at most kWaitCycles; true when it completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mbar, uint32_t phase) {
  const long long t0 = clock64();
  bool ok;
  while (!(ok = mbar_try(smem_u32(mbar), phase)))
    if (clock64() - t0 > kWaitCycles) break;
  return ok;
}
__device__ __forceinline__ void fence_smem_to_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n"); }

}  // namespace tc
}  // namespace bcgs
