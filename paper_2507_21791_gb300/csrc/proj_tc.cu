// Tensor-core projection plus triangular-solve normalization
//     W = (V - Q C) T^{-1}
// (Alg. 1 and Alg. 2: U_{k+1} = (X_{k+1} - Q_k S) S_{k+1,k+1}^{-1} and
//  Q_{k+1} = (U_{k+1} - Q_k Y) Y_{k+1,k+1}^{-1}), same result as proj.cu up to
// rounding, with the product Q C on the tensor cores.
//
// Q C is a contraction over the c columns of Q, so the exponents of the exact
// digit splitting (tc_common.cuh) run along it: every row r of Q gets
// E_r > log2 max_k |q_rk| and every column j of C gets E_j > log2 max_k |c_kj|;
// digit pairs t + u <= 8 are multiplied on the bf16 tensor cores with exact fp32
// level sums, read back every 64 columns of Q into int64 accumulators, and the
// FP64 value 2^(E_r + E_j - 70) (hi 2^28 + lo) is formed once per output.  The
// error of one product term is at most 2^-57.5 max_k|q_rk| max_k|c_kj|.
//
// The subtraction from V and the forward substitution with T stay in FP64 on
// the row's own thread: substitution keeps the normalization backward stable
// (an explicit inverse would add a kappa(T) u residual).
//
// One CTA (256 threads) per 128-row tile: a first pass over the tile finds the
// row exponents (the tile stays in L2 for the second pass), then per 64-column
// chunk of Q all threads split the tile and the matching 64 rows of C into
// swizzled digit tiles, one thread issues the 180 MMAs, all eight warps read
// tensor memory back.
#include <string.h>

#include "tc_common.cuh"

namespace bcgs {
namespace {
using namespace tc;

constexpr int kThreads = 256;
constexpr int kRows = 128;                // rows of Q per CTA (MMA M)
constexpr int kKChunk = 64;               // columns of Q per MMA stage
constexpr int kATile = kRows * 128;       // bytes of one digit tile of the Q chunk

template <typename T>
__device__ __forceinline__ void st_elem(void* p, int64_t i, double v) {
  reinterpret_cast<T*>(p)[i] = (T)v;
}

__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}

template <typename T, int NBT>
__global__ void __launch_bounds__(kThreads, 1) proj_tc_kernel(ProjDesc d, DevStatus* st) {
  static_assert(NBT == 16 || NBT == 32, "N tile");
  constexpr int kBTile = NBT * 128;
  constexpr int kTmemCols = kDigits * NBT <= 256 ? 256 : 512;
  constexpr int kHalf = NBT / 2;
  if (block_failed(st)) return;
  extern __shared__ uint8_t dyn[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base_s;
  __shared__ int s_cexp_a[kRows];
  __shared__ int s_cexp_b[NBT];
  __shared__ unsigned long long s_rowmax[2][kRows];
  __shared__ double s_T[32 * 32];
  __shared__ int s_bad;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn) + 1023) & ~uintptr_t(1023));
  uint8_t* At = base;                                   // kDigits x kATile
  uint8_t* Bt = base + kDigits * kATile;                // kDigits x kBTile
  double* P = reinterpret_cast<double*>(Bt + kDigits * kBTile);  // kRows x NBT products

  const int s = d.s, c = d.q.ncols;
  const int64_t r0 = (int64_t)blockIdx.x * kRows;
  const int rows_here = (int)min((int64_t)kRows, d.m - r0);
  const T* Q = reinterpret_cast<const T*>(d.q.p);
  const int64_t ldq = d.q.ld;

  if (tid == 0) s_bad = 0;
  // exponents of the columns of C (over its c rows)
  for (int j = warp; j < NBT; j += kThreads / 32) {
    unsigned long long mx = 0ull;
    if (j < s)
      for (int k = lane; k < c; k += 32) {
        const unsigned long long b = abs_bits(d.C[k + (int64_t)j * d.ldc]);
        mx = b > mx ? b : mx;
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = y > mx ? y : mx;
    }
    if (lane == 0) s_cexp_b[j] = (int)((mx >> 52) & 0x7FF);
  }
  // exponents of the rows of the Q tile (two halves of the columns per row)
  {
    const int i = tid & (kRows - 1), h = tid >> 7;
    unsigned long long mx = 0ull;
    if (i < rows_here) {
      const T* qr = Q + r0 + i;
      int k = h;
      for (; k + 14 < c; k += 16) {  // eight independent loads in flight
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = (double)__ldg(qr + (int64_t)(k + 2 * u) * ldq);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const unsigned long long b = abs_bits(v[u]);
          mx = b > mx ? b : mx;
        }
      }
      for (; k < c; k += 2) {
        const unsigned long long b = abs_bits((double)__ldg(qr + (int64_t)k * ldq));
        mx = b > mx ? b : mx;
      }
    }
    s_rowmax[h][i] = mx;
  }
  for (int e = tid; e < s * s; e += kThreads) {
    const int i = e % s, j = e / s;
    s_T[i * 32 + j] = d.T ? d.T[i + (int64_t)j * d.ldt] : (i == j ? 1.0 : 0.0);
  }
  if (warp == 0) tmem_alloc<kTmemCols>(&tmem_base_s);
  if (tid == 0) mbar_init(&mbar);
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  for (int i = tid; i < kRows; i += kThreads) {
    const unsigned long long mx = s_rowmax[0][i] > s_rowmax[1][i] ? s_rowmax[0][i] : s_rowmax[1][i];
    const int e = (int)((mx >> 52) & 0x7FF);
    s_cexp_a[i] = e;
    if (e == 0x7FF) s_bad = 1;
  }
  for (int j = tid; j < s; j += kThreads)
    if (s_cexp_b[j] == 0x7FF) s_bad = 1;
  __syncthreads();
  const uint32_t tmem = tmem_base_s;
  const bool bad = s_bad != 0;
  if (bad && tid == 0) set_failure(st, BCGS_ERR_NONFINITE, 0);

  const int my_i = 32 * (warp & 3) + lane;
  const int my_j0 = (warp >> 2) * kHalf;
  long long hi[kHalf], lo[kHalf];
#pragma unroll
  for (int j = 0; j < kHalf; ++j) hi[j] = lo[j] = 0;

  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NBT >> 3) << 17) |
                         ((uint32_t)(kRows >> 4) << 24);
  uint32_t phase = 0;
  bool timed_out = false;
  const int nchunks = bad ? 0 : (c + kKChunk - 1) / kKChunk;

  for (int kc = 0; kc < nchunks; ++kc) {
    const int k0 = kc * kKChunk;
    // split the Q chunk: task (row i, 8-column group g); consecutive threads take
    // consecutive rows, so every column load is coalesced across the warp
    for (int e = tid; e < kRows * 8; e += kThreads) {
      const int i = e & (kRows - 1), g = e >> 7;
      double v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int col = k0 + 8 * g + k;
        v[k] = (i < rows_here && col < c) ? (double)__ldg(Q + r0 + i + (int64_t)col * ldq) : 0.0;
      }
      split8(v, s_cexp_a[i], At, kATile, i, g);
    }
    // split the matching rows of C: task (column j, 8-row group g)
    for (int e = tid; e < NBT * 8; e += kThreads) {
      const int j = e >> 3, g = e & 7;
      double v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int row = k0 + 8 * g + k;
        v[k] = (j < s && row < c) ? d.C[row + (int64_t)j * d.ldc] : 0.0;
      }
      split8(v, s_cexp_b[j], Bt, kBTile, j, g);
    }
    fence_smem_to_async();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (tid == 0) {
#pragma unroll 1
      for (int t = 0; t < kDigits; ++t) {
        const uint32_t a_base = smem_u32(At + t * kATile);
#pragma unroll 1
        for (int u = 0; t + u < kDigits; ++u) {
          const uint32_t b_base = smem_u32(Bt + u * kBTile);
          const uint32_t dcol = tmem + (uint32_t)((t + u) * NBT);
#pragma unroll
          for (int kk = 0; kk < kKChunk / 16; ++kk)
            mma_bf16(dcol, desc_sw128(a_base + kk * 32), desc_sw128(b_base + kk * 32), idesc,
                     (t == 0 && kk == 0) ? 0u : 1u);
        }
      }
      mma_commit(&mbar);
    }
    const bool ok = mbar_wait_bounded(&mbar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      timed_out = true;
      break;
    }
    tc_after_sync();
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)my_j0;
#pragma unroll
    for (int g8 = 0; g8 < kHalf; g8 += 8) {
      int32_t L[8][kDigits];
#pragma unroll
      for (int l = 0; l < kDigits; ++l) {
        uint32_t r[8];
        tmem_ld8(lane_addr + (uint32_t)(l * NBT + g8), r);
#pragma unroll
        for (int j = 0; j < 8; ++j) L[j][l] = __float2int_rn(__uint_as_float(r[j]));
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) fold_levels(L[j], hi[g8 + j], lo[g8 + j]);
    }
    tc_before_sync();
    __syncthreads();
  }

  // products to shared memory, then the FP64 epilogue per row
  if (!bad && !timed_out) {
#pragma unroll
    for (int j = 0; j < kHalf; ++j) {
      const int jj = my_j0 + j;
      P[my_i * NBT + jj] = (jj < s) ? unfold(hi[j], lo[j], s_cexp_a[my_i], s_cexp_b[jj]) : 0.0;
    }
  }
  __syncthreads();
  if (!bad && !timed_out && tid < kRows && tid < rows_here) {
    const int64_t r = r0 + tid;
    double w[NBT];
#pragma unroll
    for (int j = 0; j < NBT; ++j)
      if (j < s) w[j] = (double)__ldg(reinterpret_cast<const T*>(d.v.p) + r + (int64_t)j * d.v.ld) -
                        (c > 0 ? P[tid * NBT + j] : 0.0);
    if (d.T != nullptr) {
#pragma unroll
      for (int j = 0; j < NBT; ++j) {
        if (j < s) {
          double x = w[j];
#pragma unroll
          for (int l = 0; l < NBT; ++l)
            if (l < j) x = fma(-w[l], s_T[l * 32 + j], x);
          w[j] = x / s_T[j * 32 + j];
        }
      }
    }
#pragma unroll
    for (int j = 0; j < NBT; ++j)
      if (j < s) st_elem<T>(d.w, r + (int64_t)j * d.ldw, w[j]);
  }
  if (timed_out && tid == 0) set_failure(st, BCGS_ERR_TIMEOUT, 0);
  tc_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc<kTmemCols>(tmem);
}

template <typename T>
cudaError_t launch_t(const ProjDesc& d, DevStatus* st, cudaStream_t stream) {
  const unsigned grid = (unsigned)ceil_div(d.m, kRows);
  if (grid == 0) return cudaSuccess;
  const int slot = prof_begin(stream);
#define BCGS_PTC_CASE(NB)                                                                          \
  {                                                                                                \
    const size_t smem = 1024 + (size_t)kDigits * (kATile + NB * 128) + (size_t)kRows * NB * 8;     \
    cudaError_t e = ensure_dyn_smem(proj_tc_kernel<T, NB>, smem);                                  \
    if (e != cudaSuccess) return e;                                                                \
    proj_tc_kernel<T, NB><<<grid, kThreads, smem, stream>>>(d, st);                                \
  }
  if (d.s <= 16) BCGS_PTC_CASE(16)
  else BCGS_PTC_CASE(32)
#undef BCGS_PTC_CASE
  prof_end(slot, kProfProject, stream, 2.0 * (double)d.m * d.q.ncols * d.s + (double)d.m * d.s * d.s,
           (double)d.m * (d.q.ncols + 2.0 * d.s) * sizeof(T));
  note_launch(1);
  return cudaGetLastError();
}

}  // namespace

bool project_tc_supported(const ProjDesc& d) { return d.s >= 1 && d.s <= 32 && d.q.ncols >= 1; }

cudaError_t launch_project_tc(const ProjDesc& d, DevStatus* st, cudaStream_t stream) {
  return d.w_fp32 ? launch_t<float>(d, st, stream) : launch_t<double>(d, st, stream);
}

}  // namespace bcgs
