// Tensor-core Gram reduction C = A^T B with FP64-accurate products.
//
// Same result, partition and determinism as gram.cu (one synchronization point
// of the paper, Sec. 3), computed on the 5th-generation tensor cores instead of
// the GB300's narrow FP64 pipe.  The products are made exact by error-free
// splitting in the manner of Ozaki, Ogita, Oishi and Rump (Numer. Algorithms
// 59, 2012):
//
//   * every column i of A (and j of B) gets the exponent E_i with
//     max_r |a_ri| < 2^E_i (a column-max pass precedes the kernel);
//   * a_ri = sign * N * 2^(E_i - 63) with the integer N < 2^63 (truncated),
//     N = sum_t d_t 2^(56 - 7t), nine digits 0 <= d_t < 128 (t = 0..8);
//     each signed digit is an integer of at most 7 bits, exact in bf16;
//   * d^A_t (x) d^B_u for t + u <= 8 (45 digit pairs) run as bf16 tcgen05.mma
//     with fp32 accumulation in tensor memory, one accumulator per level
//     l = t + u; a level sums at most (l+1) * 64 * 127^2 < 2^24 over 64 rows,
//     so every accumulator stays an exact integer;
//   * every 64 rows the nine level accumulators are read back (tcgen05.ld),
//     combined exactly in 32-bit and added into two int64 accumulators
//     (levels 0-4 and 5-8);
//   * at the end of its chunk a CTA writes
//     2^(E_i + E_j - 70) (hi 2^28 + lo) as the FP64 chunk partial.
//
// Dropped digit pairs (t + u >= 9) and the truncation of N bound the error of a
// product term by 2^(E_i + E_j - 59.5) <= 2^-57.5 max|a_i| max|b_j|; the
// integer sums are exact, so the chunk partial carries one FP64 rounding.  The
// partials are added in chunk order by the reduction kernel of gram.cu.
// (Fixed point relative to the column maximum loses log2(max|a_i| / |a_ri|)
// bits on small entries; nine digits keep heavy-tailed columns, such as rows
// with lognormal norms, at FP64-level accuracy.)
//
// One CTA (256 threads) per (chunk, 128-column tile of A); all threads split
// a 64-row block into swizzled (SW128, K-major) bf16 tiles in shared memory,
// one thread issues the 180 MMAs of the block, all eight warps read tensor
// memory back.  Every wait on the MMA barrier is bounded; on timeout the kernel
// records BCGS_ERR_TIMEOUT and returns after freeing its tensor memory.
#include <string.h>

#include "tc_common.cuh"

namespace bcgs {
namespace {
using namespace tc;

constexpr int kThreads = 256;
constexpr int kBlockRows = 64;    // rows (K) per MMA stage: one 128-byte SW128 row of bf16
constexpr int kFlushBlocks = 1;   // 64 rows between tensor-memory read-backs
constexpr int kMTile = 128;       // A columns per CTA (MMA M)
constexpr int kATile = kMTile * 128;  // bytes of one digit tile of A (128 rows x 128 B)

struct TcCols {
  int32_t a_off[kMaxSegA + 1];
  int32_t b_off[kMaxSegB + 1];
};

template <int MAXS>
__device__ __forceinline__ int find_seg(const int32_t* off, int nseg, int col) {
  int s = 0;
#pragma unroll
  for (int k = 1; k < MAXS; ++k)
    if (k < nseg && col >= off[k]) s = k;
  return s;
}

// Column max |x| of every column of A (first na) and B (next nb), kept as the
// bit pattern of |x|: for non-negative doubles unsigned order is value order,
// and Inf (0x7FF0...) and NaN (0x7FF8... and above) compare above every
// finite value, so a non-finite column shows as exponent field 0x7FF.
template <typename T>
__global__ void colmax_kernel(GramDesc d, TcCols cm, unsigned long long* amax) {
  const int col = blockIdx.y;
  const bool is_a = col < d.na;
  const int c = is_a ? col : col - d.na;
  const int sg = is_a ? find_seg<kMaxSegA>(cm.a_off, d.nsa, c) : find_seg<kMaxSegB>(cm.b_off, d.nsb, c);
  const Seg& S = is_a ? d.a[sg] : d.b[sg];
  const int cc = c - (is_a ? cm.a_off[sg] : cm.b_off[sg]);
  const int64_t off = (int64_t)cc * S.ld;
  unsigned long long mx = 0ull;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < d.m;
       r += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long bits =
        (unsigned long long)__double_as_longlong(ld_elem<T>(S.p, off + r)) & 0x7FFFFFFFFFFFFFFFull;
    mx = bits > mx ? bits : mx;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(amax + col, mx);
}

__device__ __forceinline__ int cexp_of(unsigned long long b) { return (int)((b >> 52) & 0x7FF); }

template <typename T, int NBT>
__global__ void __launch_bounds__(kThreads, 1)
gram_tc_kernel(GramDesc d, TcCols cm, const unsigned long long* __restrict__ amax,
               double* __restrict__ partial, DevStatus* st) {
  static_assert(NBT == 16 || NBT == 32, "N tile");
  constexpr int kBTile = NBT * 128;       // bytes of one digit tile of B
  constexpr int kTmemCols = kDigits * NBT <= 256 ? (kDigits * NBT <= 128 ? 128 : 256) : 512;
  constexpr int kHalf = NBT / 2;          // output columns per thread in the read-back
  if (block_failed(st)) return;
  extern __shared__ uint8_t dyn[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base_s;
  __shared__ int s_cexp_a[kMTile];
  __shared__ int s_cexp_b[NBT];
  __shared__ int s_bad;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn) + 1023) & ~uintptr_t(1023));
  uint8_t* At = base;                         // kDigits tiles of kATile bytes
  uint8_t* Bt = base + kDigits * kATile;      // kDigits tiles of kBTile bytes

  const int chunk = blockIdx.x;
  const int col0 = blockIdx.y * kMTile;       // first A column of this tile
  const int ncol_a = min(kMTile, d.na - col0);
  const int jb0 = blockIdx.z * NBT;           // first B column of this tile
  const int nb = min(NBT, d.nb - jb0);        // B columns of this tile
  const int ldp = d.nb;                       // row length of the partial layout
  const int64_t r_begin = (int64_t)chunk * d.chunk_rows;
  const int64_t r_end = min(r_begin + d.chunk_rows, d.m);

  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int i = tid; i < kMTile; i += kThreads) {
    int e = 0;
    if (i < ncol_a) {
      const unsigned long long b = amax[col0 + i];
      e = cexp_of(b);
      if (e == 0x7FF) s_bad = 1;
    }
    s_cexp_a[i] = e;
  }
  for (int j = tid; j < NBT; j += kThreads) {
    int e = 0;
    if (j < nb) {
      const unsigned long long b = amax[d.na + jb0 + j];
      e = cexp_of(b);
      if (e == 0x7FF) s_bad = 1;
    }
    s_cexp_b[j] = e;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&tmem_base_s)),
                 "n"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = tmem_base_s;
  const bool bad = s_bad != 0;
  if (bad && tid == 0) set_failure(st, BCGS_ERR_NONFINITE, d.block);

  // read-back role: lane quadrant (warp % 4) -> A column, half (warp / 4) -> B columns
  const int my_i = 32 * (warp & 3) + lane;
  const int my_j0 = (warp >> 2) * kHalf;
  long long hi[kHalf], lo[kHalf];
#pragma unroll
  for (int j = 0; j < kHalf; ++j) hi[j] = lo[j] = 0;

  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NBT >> 3) << 17) |
                         ((uint32_t)(kMTile >> 4) << 24);
  uint32_t phase = 0;
  bool timed_out = false;
  const int nblocks = bad ? 0 : (int)((r_end - r_begin + kBlockRows - 1) / kBlockRows);

  for (int b = 0; b < nblocks; ++b) {
    const int64_t r0 = r_begin + (int64_t)b * kBlockRows;
    // ---- split A: tasks (column, 8-row group)
    for (int e = tid; e < kMTile * 8; e += kThreads) {
      const int i = e >> 3, g = e & 7;
      double v[8];
      if (i < ncol_a) {
        const int ca = col0 + i;
        const int sg = find_seg<kMaxSegA>(cm.a_off, d.nsa, ca);
        const int64_t cbase = (int64_t)(ca - cm.a_off[sg]) * d.a[sg].ld;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int64_t row = r0 + 8 * g + k;
          v[k] = row < r_end ? ld_elem<T>(d.a[sg].p, cbase + row) : 0.0;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = 0.0;
      }
      split8(v, s_cexp_a[i], At, kATile, i, g);
    }
    // ---- split B
    for (int e = tid; e < NBT * 8; e += kThreads) {
      const int j = e >> 3, g = e & 7;
      double v[8];
      if (j < nb) {
        const int sg = find_seg<kMaxSegB>(cm.b_off, d.nsb, jb0 + j);
        const int64_t cbase = (int64_t)(jb0 + j - cm.b_off[sg]) * d.b[sg].ld;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int64_t row = r0 + 8 * g + k;
          v[k] = row < r_end ? ld_elem<T>(d.b[sg].p, cbase + row) : 0.0;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = 0.0;
      }
      split8(v, s_cexp_b[j], Bt, kBTile, j, g);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    // ---- MMAs of this block (one thread)
    const bool window_start = (b % kFlushBlocks) == 0;
    if (tid == 0) {
#pragma unroll 1
      for (int t = 0; t < kDigits; ++t) {
        const uint32_t a_base = smem_u32(At + t * kATile);
#pragma unroll 1
        for (int u = 0; t + u < kDigits; ++u) {
          const uint32_t b_base = smem_u32(Bt + u * kBTile);
          const uint32_t dcol = tmem + (uint32_t)((t + u) * NBT);
#pragma unroll
          for (int kk = 0; kk < kBlockRows / 16; ++kk) {
            const uint32_t acc = (window_start && t == 0 && kk == 0) ? 0u : 1u;
            mma_bf16(dcol, desc_sw128(a_base + kk * 32), desc_sw128(b_base + kk * 32), idesc, acc);
          }
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              smem_u32(&mbar)));
    }
    bool ok = false;
    const long long t_wait = clock64();
    while (!(ok = mbar_try(smem_u32(&mbar), phase)))
      if (clock64() - t_wait > kWaitCycles) break;
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      timed_out = true;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    // ---- read back and fold the level accumulators every kFlushBlocks blocks
    if ((b % kFlushBlocks) == kFlushBlocks - 1 || b == nblocks - 1) {
      const uint32_t lane_addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)my_j0;
#pragma unroll
      for (int g8 = 0; g8 < kHalf; g8 += 8) {
        int32_t L[kDigits][8];
#pragma unroll
        for (int l = 0; l < kDigits; ++l) {
          uint32_t r[8];
          const uint32_t taddr = lane_addr + (uint32_t)(l * NBT + g8);
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                       : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                         "=r"(r[6]), "=r"(r[7])
                       : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;\n");
#pragma unroll
          for (int j = 0; j < 8; ++j) L[l][j] = __float2int_rn(__uint_as_float(r[j]));
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          // exact: |L_l| <= (l+1) 64 127^2 < (l+1) 2^20
          const int32_t c01 = (L[0][j] << 7) + L[1][j];
          const int32_t c23 = (L[2][j] << 7) + L[3][j];
          const int32_t c56 = (L[5][j] << 7) + L[6][j];
          const int32_t c78 = (L[7][j] << 7) + L[8][j];
          hi[g8 + j] += ((long long)c01 << 21) + ((long long)c23 << 7) + (long long)L[4][j];
          lo[g8 + j] += ((long long)c56 << 14) + (long long)c78;
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();  // tiles and accumulators are free for the next block
  }

  if (!bad && !timed_out) {
    if (my_i < ncol_a) {
      double* out = partial + (size_t)chunk * ((size_t)d.na * ldp) + (size_t)(col0 + my_i) * ldp + jb0;
      const int ea = s_cexp_a[my_i];
#pragma unroll
      for (int j = 0; j < kHalf; ++j) {
        const int jj = my_j0 + j;
        if (jj < nb) {
          const int sc = ea + s_cexp_b[jj] - 2044;  // E_i + E_j
          out[jj] = ldexp((double)hi[j], sc - 42) + ldexp((double)lo[j], sc - 70);
        }
      }
    }
  }
  if (timed_out && tid == 0) set_failure(st, BCGS_ERR_TIMEOUT, d.block);
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(kTmemCols));
}

__global__ void zero_u64_kernel(unsigned long long* p, int n) {
  for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < n; i += blockDim.x * gridDim.x) p[i] = 0ull;
}

template <typename T>
cudaError_t launch_t(const GramDesc& d, double* partial, double* G, int ldg, unsigned long long* amax,
                     DevStatus* st, cudaStream_t stream) {
  TcCols cm;
  cm.a_off[0] = 0;
  for (int k = 0; k < kMaxSegA; ++k) cm.a_off[k + 1] = cm.a_off[k] + (k < d.nsa ? d.a[k].ncols : 0);
  cm.b_off[0] = 0;
  for (int k = 0; k < kMaxSegB; ++k) cm.b_off[k + 1] = cm.b_off[k] + (k < d.nsb ? d.b[k].ncols : 0);
  const int ncols = d.na + d.nb;
  zero_u64_kernel<<<(ncols + 255) / 256, 256, 0, stream>>>(amax, ncols);
  {
    int gx = (int)ceil_div(d.m, 256 * 64);
    if (gx > 16) gx = 16;
    if (gx < 1) gx = 1;
    colmax_kernel<T><<<dim3(gx, ncols), 256, 0, stream>>>(d, cm, amax);
  }
  const int slot = prof_begin(stream);
  const int nbt = d.nb <= 16 ? 16 : 32;
  dim3 grid(d.nchunks, (unsigned)ceil_div(d.na, kMTile), (unsigned)ceil_div(d.nb, nbt));
#define BCGS_TC_CASE(NB)                                                                        \
  {                                                                                             \
    const size_t smem = 1024 + (size_t)kDigits * (kATile + NB * 128);                           \
    cudaError_t e = ensure_dyn_smem(gram_tc_kernel<T, NB>, smem);                               \
    if (e != cudaSuccess) return e;                                                             \
    gram_tc_kernel<T, NB><<<grid, kThreads, smem, stream>>>(d, cm, amax, partial, st);           \
  }
  if (nbt == 16) BCGS_TC_CASE(16)
  else BCGS_TC_CASE(32)
#undef BCGS_TC_CASE
  prof_end(slot, kProfGramPartial, stream, 2.0 * (double)d.m * d.na * d.nb,
           (double)d.m * (d.na + d.nb) * sizeof(T) + (double)d.nchunks * d.na * d.nb * 8.0);
  note_launch(3);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_gram_reduce(partial, d.nchunks, d.na, d.nb, G, ldg, st, stream);
}

}  // namespace

bool gram_tc_supported(const GramDesc& d) { return d.nb >= 1 && d.nb <= 64 && d.na >= 1; }

cudaError_t launch_gram_tc(const GramDesc& d, double* partial, double* G, int ldg,
                           unsigned long long* amax, DevStatus* st, cudaStream_t stream) {
  if (d.na <= 0 || d.nb <= 0) return cudaSuccess;
  const bool f32 = d.a[0].fp32 != 0;
  return f32 ? launch_t<float>(d, partial, G, ldg, amax, st, stream)
             : launch_t<double>(d, partial, G, ldg, amax, st, stream);
}

}  // namespace bcgs
