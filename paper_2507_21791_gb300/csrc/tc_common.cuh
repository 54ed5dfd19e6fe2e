// Device helpers shared by the tensor-core kernels (gram_tc.cu, proj_tc.cu,
// qstore.cu, gram_store.cu): tcgen05 descriptors and MMA issue, bounded mbarrier
// polling, asynchronous copies, and the exact splitting of an FP64 value into
// eight 8-bit digits relative to an exponent (error-free splitting in the manner
// of Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59, 2012).
//
// Two digit forms live here:
//   * sign-magnitude digits in bf16 (this first part): used by the kernels that
//     split their operands on the fly, gram_tc.cu and proj_tc.cu;
//   * balanced digits in f16 (the second part, "balanced digits" below): used by
//     the resident digit store of Q and the kernels that read it, qstore.cu
//     (split and projection) and gram_store.cu.
//
// Sign-magnitude digits: with E the exponent of the line's maximum (|a| < 2^E),
// a = sign N 2^(E - 63) with the integer N < 2^63 (truncated), and the digits
// are the bytes of N: N = sum_t d_t 2^(56 - 8t), t = 0..7 (d_0 < 128).  A
// signed digit is an integer of magnitude at most 255, exact in bf16.  The
// product of two digits is below 2^16; a level l = t + u of at most eight digit
// pairs summed over 32 rows stays below 8 * 32 * 255^2 < 2^24, exact in fp32.
// Keeping the pairs t + u <= 7 (36 pairs) and truncating N bound the error of
// one product term by 2^(E_a + E_b - 59.1) <= 2^-57.1 max|a| max|b|.
#pragma once

#include "bcgs_internal.cuh"

namespace bcgs {
namespace tc {

constexpr int kDigits = 8;
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

// tcgen05 shared-memory descriptor, K-major without swizzle: 8-row x 16-byte core
// matrices stored contiguously (128 B each); `lbo` = byte distance between core
// matrices adjacent along K, `sbo` = between core matrices adjacent along M/N.
__device__ __forceinline__ uint64_t desc_interleave(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// D (tensor memory, fp32) (+)= A B^T for bf16 A (M x K) and B (N x K) in shared
// memory; `accumulate` = 0 overwrites D.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// Instruction descriptor of kind::f16: fp32 D, bf16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// One bounded wait on the phase: the thread is suspended until the phase
// completes or about a microsecond has passed (suspend-time hint, in ns), so a
// waiting warp takes no issue slots from the working warps of its sub-partition.
__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(phase), "r"(1000u)
      : "memory");
  return ok != 0;
}

// Non-blocking test of the phase (for event loops that watch several barriers).
__device__ __forceinline__ bool mbar_test(uint64_t* mbar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(mbar)), "r"(phase)
      : "memory");
  return ok != 0;
}

template <typename T>
__device__ __forceinline__ double ld_elem(const void* base, int64_t idx) {
  return (double)__ldg(reinterpret_cast<const T*>(base) + idx);
}

// 63-bit fixed-point magnitude of a relative to the exponent field `cexp` (the
// biased exponent of the line's max |a|): N = |a| 2^(63 - E), E = cexp - 1022,
// truncated.  neg receives the sign bit.
__device__ __forceinline__ uint64_t fixed63(double a, int cexp, uint32_t& neg) {
  const uint64_t bits = (uint64_t)__double_as_longlong(a);
  neg = (uint32_t)(bits >> 63);
  const int e = (int)((bits >> 52) & 0x7FF);
  // N = mant 2^(e - cexp + 10): mant < 2^53, so mant 2^10 < 2^63, then shift right
  // by cexp - e >= 0 (|a| <= max).  A zero exponent field (zero, subnormal) gives 0.
  const uint64_t mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int d = cexp - e;
  return (e != 0 && d < 64) ? ((mant << 10) >> (d > 0 ? d : 0)) : 0ull;
}

// fp32 bits of the signed digit in byte `sel` of x: the byte is placed into the
// sign-carrying magic word +-2^23 (0x4B000000 / 0xCB000000) and the magic is
// removed, (+-(2^23 + d)) -/+ 2^23 = +-d exactly: one PRMT and one FADD.
__device__ __forceinline__ uint32_t digit_byte_f32(uint32_t x, uint32_t magic, float off, uint32_t sel) {
  return __float_as_uint(__uint_as_float(__byte_perm(x, magic, 0x7650u | sel)) + off);
}

// Split 8 consecutive K-elements into the 8 digit tiles, 16 bytes (8 bf16) at
// byte offset `off` of each tile.
__device__ __forceinline__ void split8_at(const double (&v)[8], int cexp, uint8_t* tiles, int tile_bytes,
                                          int off) {
  uint32_t lo[8], hi[8], mg[8];
  float ofs[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    uint32_t neg;
    const uint64_t N = fixed63(v[e], cexp, neg);
    lo[e] = (uint32_t)N;
    hi[e] = (uint32_t)(N >> 32);
    mg[e] = 0x4B000000u | (neg << 31);
    ofs[e] = __uint_as_float(0xCB000000u ^ (neg << 31));
  }
#pragma unroll
  for (int t = 0; t < kDigits; ++t) {
    const uint32_t sel = 3u - (uint32_t)(t & 3);  // digit t is byte 7 - t of N
    uint32_t w[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const uint32_t x0 = t < 4 ? hi[2 * p] : lo[2 * p];
      const uint32_t x1 = t < 4 ? hi[2 * p + 1] : lo[2 * p + 1];
      w[p] = __byte_perm(digit_byte_f32(x0, mg[2 * p], ofs[2 * p], sel),
                         digit_byte_f32(x1, mg[2 * p + 1], ofs[2 * p + 1], sel), 0x7632);
    }
    *reinterpret_cast<uint4*>(tiles + t * tile_bytes + off) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// K-major, non-swizzled digit tiles with `kc` 16-byte chunks per 8-row group:
// row `row`, chunk `g` lives at ((row / 8) kc + g) 128 + (row % 8) 16.
__device__ __forceinline__ void split8_interleave(const double (&v)[8], int cexp, uint8_t* tiles,
                                                  int tile_bytes, int row, int g, int kc) {
  split8_at(v, cexp, tiles, tile_bytes, ((row >> 3) * kc + g) * 128 + (row & 7) * 16);
}

// 4- and 8-byte asynchronous global -> shared copies; `valid` = false writes
// zeros and reads nothing.
__device__ __forceinline__ void cp_async8(void* dst_smem, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(smem_u32(dst_smem)), "l"(src),
               "r"(valid ? 8 : 0));
}
__device__ __forceinline__ void cp_async4(void* dst_smem, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_u32(dst_smem)), "l"(src),
               "r"(valid ? 4 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n");
}

// Fold the eight exact level sums L_l (|L_l| <= (l+1) 32 255^2 < 2^24) into two
// int64 accumulators: hi += sum_{l<=3} L_l 2^(8(3-l)), lo += sum_{l>=4} L_l 2^(8(7-l)).
__device__ __forceinline__ void fold_levels(const int32_t (&L)[kDigits], long long& hi, long long& lo) {
  const int32_t c01 = (L[0] << 8) + L[1];  // |L0| <= 32 255^2 < 2^21: no overflow
  const int32_t c23 = (L[2] << 8) + L[3];  // |L2| <= 3 32 255^2: 256 |L2| < 2^31
  hi += ((long long)c01 << 16) + (long long)c23;
  lo += ((long long)L[4] << 24) + ((long long)L[5] << 16) + ((long long)L[6] << 8) + (long long)L[7];
}

// The value 2^(E_a + E_b - 70) (hi 2^32 + lo), with E = cexp - 1022.
__device__ __forceinline__ double unfold(long long hi, long long lo, int cexp_a, int cexp_b) {
  const int sc = cexp_a + cexp_b - 2044;
  return ldexp((double)hi, sc - 38) + ldexp((double)lo, sc - 70);
}

// ---------------------------------------------------------------- balanced digits
// Second digit form, used by the resident digit store of Q (qstore.cu): a is
// written as the signed integer N = trunc(a 2^(62 - E)) (|N| < 2^62), and N is
// expanded in balanced base-256 digits d_t in [-128, 127]:
//     N = sum_t d_t 2^(56 - 8t),   d_t = byte_(7-t)(N + 0x8080808080808080) - 128,
// (adding 128 to every byte turns the balanced expansion into the unsigned one;
// |N| < 2^62 keeps the sum clear of the wrap-around).  |d_t| <= 128 (|d_0| <= 64),
// so a digit product is at most 2^14 and a level of at most eight pairs summed
// over 128 K-values is at most 7 2^21 < 2^24: exact in fp32 for 128 K-values
// between read-backs.  Digits are stored as f16 (integers up to 2048 are exact).
// The store keeps d_0 .. d_6 (kStoreDigits); the coefficient side of a
// projection, split in shared memory, keeps all eight.

// N + 0x8080808080808080 for a with biased exponent `e`, magnitude bits `mant`
// (implicit bit included) and sign `neg`, relative to the exponent field `cexp`
// (cexp >= e; |a| < 2^(cexp - 1022)): N = (mant 2^9) >> (cexp - e).
__device__ __forceinline__ uint64_t fixed62_offset(uint64_t mant, int e, int cexp, uint32_t neg) {
  const int d = cexp - e;
  const uint64_t mag = (e > 0 && d < 63) ? ((mant << 9) >> (d > 0 ? d : 0)) : 0ull;
  const uint64_t n = neg ? (0ull - mag) : mag;
  return n + 0x8080808080808080ull;
}
__device__ __forceinline__ uint64_t fixed62_offset(double a, int cexp) {
  const uint64_t bits = (uint64_t)__double_as_longlong(a);
  return fixed62_offset((bits & 0xFFFFFFFFFFFFFull) | (1ull << 52), (int)((bits >> 52) & 0x7FF), cexp,
                        (uint32_t)(bits >> 63));
}

// f16x2 of two offset-binary digit bytes of `w` (bytes 0 and 2 for SEL 0x4240,
// bytes 1 and 3 for SEL 0x4341): each byte b becomes the low mantissa bits of
// the f16 1024 + b, and 1152 = 1024 + 128 is taken off (exact).
template <uint32_t SEL>
__device__ __forceinline__ uint32_t f16x2_digits(uint32_t w) {
  const uint32_t h = __byte_perm(w, 0x64646464u, SEL);
  uint32_t r;
  asm("sub.rn.f16x2 %0, %1, %2;\n" : "=r"(r) : "r"(h), "r"(0x64806480u));
  return r;
}

// For two consecutive K-elements x, y with offset words (hi, lo) = (xh, xl) and
// (yh, yl): out[t] = f16x2 (digit t of x, digit t of y), t = 0..7; digit t is
// byte 3 - t of hi for t < 4 and byte 7 - t of lo otherwise.
__device__ __forceinline__ void digits_pair_f16(uint32_t xh, uint32_t xl, uint32_t yh, uint32_t yl,
                                                uint32_t (&out)[8]) {
  const uint32_t h3 = __byte_perm(xh, yh, 0x6723u);  // [x.b3, x.b2, y.b3, y.b2]
  const uint32_t h1 = __byte_perm(xh, yh, 0x4501u);  // [x.b1, x.b0, y.b1, y.b0]
  const uint32_t l3 = __byte_perm(xl, yl, 0x6723u);
  const uint32_t l1 = __byte_perm(xl, yl, 0x4501u);
  out[0] = f16x2_digits<0x4240u>(h3);
  out[1] = f16x2_digits<0x4341u>(h3);
  out[2] = f16x2_digits<0x4240u>(h1);
  out[3] = f16x2_digits<0x4341u>(h1);
  out[4] = f16x2_digits<0x4240u>(l3);
  out[5] = f16x2_digits<0x4341u>(l3);
  out[6] = f16x2_digits<0x4240u>(l1);
  out[7] = f16x2_digits<0x4341u>(l1);
}

// Instruction descriptor of kind::f16 with f16 A and B (fp32 D, both K-major).
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Bulk (non-tensor) global -> shared copy completing on an mbarrier's
// transaction count; sizes and addresses multiples of 16 bytes.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(mbar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst_smem)),
      "l"(src), "r"(bytes), "r"(smem_u32(mbar))
      : "memory");
}

// Tiled TMA load of one box of the 5-d tensor `map` at coordinates c0..c4
// (innermost first; c0 times the element size must be a multiple of 16 bytes)
// into shared memory, completing on `mbar` with the box's bytes.
__device__ __forceinline__ void tma_load_5d(void* dst_smem, const void* map, int32_t c0, int32_t c1, int32_t c2,
                                            int32_t c3, int32_t c4, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];\n" ::"r"(smem_u32(dst_smem)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(mbar))
      : "memory");
}

// tcgen05.ld without the wait (several loads in flight, then tmem_wait_ld).
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// The value of the folded levels of the balanced form, 2^(F - 1022 - 36) hi +
// 2^(F - 1022 - 68) lo, for the column exponent field F of the B operand
// (the exponents of A cancel against the scaling of B, see qstore.cu).
__device__ __forceinline__ double unfold62(long long hi, long long lo, int F) {
  return ldexp((double)hi, F - 1058) + ldexp((double)lo, F - 1090);
}

// The double nearest to (hi 2^32 + lo) 2^(F - 1090) (round to nearest, ties to
// even), built from the exact integer with integer operations and selects only
// (no FP64 pipe work, no divergent branches; GB300's FP64 rate is low).  Results
// outside the normal range take the ldexp route.
__device__ __forceinline__ double fixed_to_double(long long hi, long long lo, int F) {
  // v = H 2^32 + L with 0 <= L < 2^32, |v| < 2^95, as the 128-bit (vh, vl)
  const long long H = hi + (lo >> 32);
  const unsigned long long L = (unsigned long long)lo & 0xFFFFFFFFull;
  const unsigned long long sgn = (unsigned long long)(H >> 63);  // 0 or all ones
  unsigned long long vl = ((unsigned long long)H << 32) | L;
  unsigned long long vh = (unsigned long long)(H >> 32);
  // |v| = (v ^ sgn) + (sgn & 1)
  vl ^= sgn;
  vh ^= sgn;
  const unsigned long long vl2 = vl + (sgn & 1ull);
  vh += vl2 < vl ? 1ull : 0ull;
  vl = vl2;
  const bool hv = vh != 0ull;
  const int lzh = __clzll((long long)vh);  // 33..63 when hv
  const int lzl = __clzll((long long)vl);
  const int n = hv ? lzh : 33;
  // the 64 bits from the leading one down, and whether anything below them is set
  const unsigned long long top = hv ? ((vh << n) | (vl >> (64 - n))) : (vl << (lzl & 63));
  const unsigned long long rest = hv ? (vl << n) : 0ull;
  const int lz = hv ? lzh : 64 + lzl;
  unsigned long long mant = top >> 11;  // 53 bits
  const unsigned long long rnd = (top >> 10) & 1ull;
  const unsigned long long sticky = ((top & 0x3FFull) | rest) != 0ull ? 1ull : 0ull;
  mant += rnd & (sticky | (mant & 1ull));
  const unsigned long long carry = mant >> 53;
  mant >>= carry;
  const int be = 127 - lz + (int)carry + F - 1090 + 1023;
  const double r = __longlong_as_double((long long)((sgn << 63) | ((unsigned long long)(be & 0x7FF) << 52) |
                                                    (mant & 0xFFFFFFFFFFFFFull)));
  if (!hv && vl == 0ull) return 0.0;
  if (be <= 0 || be >= 2047) return ldexp((double)hi, F - 1058) + ldexp((double)lo, F - 1090);
  return r;
}

// Register reallocation between warpgroups (every warp of a warpgroup executes
// the same instruction): dec gives registers back to the CTA's pool, inc waits
// until the pool holds enough.  The pool is what the CTA was launched with.
template <int N>
__device__ __forceinline__ void setmaxnreg_dec() {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(N));
}
template <int N>
__device__ __forceinline__ void setmaxnreg_inc() {
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(N));
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
__device__ __forceinline__ void mbar_init_count(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(mbar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;\n");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(mbar)) : "memory");
}
// Barrier `id` (1..15) over `count` threads (a multiple of 32) of the CTA.
__device__ __forceinline__ void named_bar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(count) : "memory");
}
// Poll the barrier's phase `phase` for at most `limit` cycles; true when it completed.
__device__ __forceinline__ bool mbar_wait_limit(uint64_t* mbar, uint32_t phase, long long limit) {
  const long long t0 = clock64();
  bool ok;
  while (!(ok = mbar_try(smem_u32(mbar), phase)))
    if (clock64() - t0 > limit) break;
  return ok;
}
// ... for at most kWaitCycles (about one second).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mbar, uint32_t phase) {
  return mbar_wait_limit(mbar, phase, kWaitCycles);
}
__device__ __forceinline__ void fence_smem_to_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n"); }

}  // namespace tc
}  // namespace bcgs
