// Tensor-core projection plus triangular-solve normalization
//     W = (V - Q C) T^{-1}
// (Alg. 1 and Alg. 2: U_{k+1} = (X_{k+1} - Q_k S) S_{k+1,k+1}^{-1} and
//  Q_{k+1} = (U_{k+1} - Q_k Y) Y_{k+1,k+1}^{-1}), same result as proj.cu up to
// rounding, with the product Q C on the tensor cores.
//
// Q C is a contraction over the c columns of Q, so the exponents of the exact
// digit splitting (tc_common.cuh) run along it: every row r of Q gets
// E_r > log2 max_k |q_rk| and every column j of C gets E_j > log2 max_k |c_kj|;
// digit pairs t + u <= 7 are multiplied on the bf16 tensor cores with exact fp32
// level sums, read back every 32 columns of Q into int64 accumulators, and the
// FP64 value 2^(E_r + E_j - 70) (hi 2^32 + lo) is formed once per output.  The
// error of one product term is at most 2^-57.1 max_k|q_rk| max_k|c_kj|.
//
// The subtraction from V and the forward substitution with T stay in FP64 on
// the row's own thread: substitution keeps the normalization backward stable
// (an explicit inverse would add a kappa(T) u residual); the division by
// t_jj is a multiplication by its reciprocal, formed once per CTA.
//
// One CTA (256 threads) per 128-row tile: a first pass over the tile finds the
// row exponents (the tile stays in L2 for the second pass); then, pipelined over
// 32-column chunks of Q, cp.async stages chunk k+2, all threads split chunk k+1
// (and the matching 32 rows of C) into K-major bf16 digit tiles while the tensor
// cores run the MMAs of chunk k, and all eight warps read its level sums
// back.
#include <string.h>

#include "tc_common.cuh"

namespace bcgs {
namespace {
using namespace tc;

constexpr int kThreads = 256;
constexpr int kRows = 128;                // rows of Q per CTA (MMA M)
constexpr int kKChunk = 32;               // columns of Q per MMA stage
constexpr int kChunks = kKChunk / 8;      // 16-byte chunks of K per operand row in a digit tile
constexpr int kATile = kRows * kKChunk * 2;  // bytes of one digit tile of the Q chunk

template <typename T>
__device__ __forceinline__ void st_elem(void* p, int64_t i, double v) {
  reinterpret_cast<T*>(p)[i] = (T)v;
}

__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}

// Buffers of digit tiles: one for s <= 16 (two CTAs per SM overlap each other's
// phases), two for s <= 32 (one CTA per SM pipelines its own chunks).
template <int NBT>
struct ProjCfg {
  static constexpr int kBuf = NBT <= 16 ? 1 : 2;
  static constexpr int kCtasPerSm = NBT <= 16 ? 2 : 1;
};

template <typename T, int NBT>
__global__ void __launch_bounds__(kThreads, ProjCfg<NBT>::kCtasPerSm) proj_tc_kernel(ProjDesc d, DevStatus* st) {
  static_assert(NBT == 16 || NBT == 32, "N tile");
  constexpr int kBuf = ProjCfg<NBT>::kBuf;
  constexpr int kBTile = NBT * kKChunk * 2;            // bytes of one digit tile of C
  constexpr int kStage = kDigits * (kATile + kBTile);
  constexpr int kTmemCols = kDigits * NBT <= 128 ? 128 : (kDigits * NBT <= 256 ? 256 : 512);
  constexpr int kGroups = kThreads / 128;    // column groups (warp / 4)
  constexpr int kHalf = NBT / kGroups;       // output columns per thread in the read-back
  if (block_failed(st)) return;
  extern __shared__ uint8_t dyn[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base_s;
  __shared__ int s_cexp_a[kRows];
  __shared__ int s_cexp_b[NBT];
  __shared__ unsigned long long s_rowmax[kThreads / kRows][kRows];
  __shared__ double s_inv[32];
  __shared__ double s_T[NBT * NBT];
  __shared__ int s_bad;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t* digits = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn) + 1023) & ~uintptr_t(1023));
  T* staging = reinterpret_cast<T*>(digits + kBuf * kStage);       // kKChunk columns x kRows rows
  double* P = reinterpret_cast<double*>(digits + kBuf * kStage);   // reuses staging: kRows x NBT

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
        const unsigned long long bb = abs_bits(d.C[k + (int64_t)j * d.ldc]);
        mx = bb > mx ? bb : mx;
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = y > mx ? y : mx;
    }
    if (lane == 0) s_cexp_b[j] = (int)((mx >> 52) & 0x7FF);
  }
  // exponents of the rows of the Q tile: kept by the writers of Q, or found by
  // a pass over the tile (which then stays in L2 for the chunks)
  constexpr int kParts = kThreads / kRows;  // threads per row
  if (d.q_rowmax != nullptr) {
    for (int i = tid; i < kRows; i += kThreads) s_rowmax[0][i] = i < rows_here ? d.q_rowmax[r0 + i] : 0ull;
    for (int h = 1; h < kParts; ++h)
      for (int i = tid; i < kRows; i += kThreads) s_rowmax[h][i] = 0ull;
  } else {
    const int i = tid & (kRows - 1), h = tid / kRows;
    unsigned long long mx = 0ull;
    if (i < rows_here) {
      const T* qr = Q + r0 + i;
      int k = h;
      for (; k + 7 * kParts < c; k += 8 * kParts) {  // eight independent loads in flight
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = (double)__ldg(qr + (int64_t)(k + kParts * u) * ldq);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const unsigned long long bb = abs_bits(v[u]);
          mx = bb > mx ? bb : mx;
        }
      }
      for (; k < c; k += kParts) {
        const unsigned long long bb = abs_bits((double)__ldg(qr + (int64_t)k * ldq));
        mx = bb > mx ? bb : mx;
      }
    }
    s_rowmax[h][i] = mx;
  }
  for (int e = tid; e < s * s; e += kThreads) {
    const int i = e % s, j = e / s;
    s_T[i * NBT + j] = d.T ? d.T[i + (int64_t)j * d.ldt] : (i == j ? 1.0 : 0.0);
  }
  if (warp == 0) tmem_alloc<kTmemCols>(&tmem_base_s);
  if (tid == 0) mbar_init(&mbar);
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  for (int i = tid; i < kRows; i += kThreads) {
    unsigned long long mx = 0ull;
#pragma unroll
    for (int h = 0; h < kThreads / kRows; ++h) mx = s_rowmax[h][i] > mx ? s_rowmax[h][i] : mx;
    const int e = (int)((mx >> 52) & 0x7FF);
    s_cexp_a[i] = e;
    if (e == 0x7FF) s_bad = 1;
  }
  for (int j = tid; j < s; j += kThreads) {
    if (s_cexp_b[j] == 0x7FF) s_bad = 1;
    s_inv[j] = 1.0 / s_T[j * NBT + j];  // one division per diagonal entry per CTA
  }
  __syncthreads();
  const uint32_t tmem = tmem_base_s;
  const bool bad = s_bad != 0;
  if (bad && tid == 0) set_failure(st, BCGS_ERR_NONFINITE, 0);

  // Q chunk -> staging (column-major; consecutive threads copy consecutive rows)
  auto stage_copy = [&](int k0) {
    for (int e = tid; e < kKChunk * kRows; e += kThreads) {
      const int col = e / kRows, i = e - col * kRows;
      const bool valid = i < rows_here && k0 + col < c;
      const T* src = valid ? Q + r0 + i + (int64_t)(k0 + col) * ldq : Q;
      if constexpr (sizeof(T) == 8) cp_async8(staging + col * kRows + i, src, valid);
      else cp_async4(staging + col * kRows + i, src, valid);
    }
    cp_async_commit();
  };
  // staging + C rows -> digit tiles of buffer `buf`
  auto split_chunk = [&](int buf, int k0) {
    uint8_t* dA = digits + buf * kStage;
    uint8_t* dB = dA + kDigits * kATile;
    for (int e = tid; e < kRows * kChunks; e += kThreads) {
      const int i = e & (kRows - 1), g = e >> 7;   // consecutive threads: consecutive rows
      double v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = (double)staging[(8 * g + k) * kRows + i];
      split8_interleave(v, s_cexp_a[i], dA, kATile, i, g, kChunks);
    }
    for (int e = tid; e < NBT * kChunks; e += kThreads) {
      const int j = e % NBT, g = e / NBT;
      double v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int row = k0 + 8 * g + k;
        v[k] = (j < s && row < c) ? d.C[row + (int64_t)j * d.ldc] : 0.0;
      }
      split8_interleave(v, s_cexp_b[j], dB, kBTile, j, g, kChunks);
    }
  };
  // One MMA per (digit t of A, 16-row K step): the B digit tiles are contiguous,
  // so [B_0 ... B_{8-t}] is a single K-major operand of (9-t) NBT rows whose
  // product with A_t lands, tile u, in the accumulator of level t + u (tensor
  // memory columns (t + u) NBT); pieces of at most 256 columns.
  auto issue_mma = [&](int buf) {
    const uint32_t a0 = smem_u32(digits + buf * kStage);
    const uint32_t b0 = a0 + kDigits * kATile;
    constexpr int kMaxLev = 256 / NBT;
#pragma unroll 1
    for (int t = 0; t < kDigits; ++t) {
      const int nlev = kDigits - t;
#pragma unroll 1
      for (int l0 = 0; l0 < nlev; l0 += kMaxLev) {
        const int nl = nlev - l0 < kMaxLev ? nlev - l0 : kMaxLev;
        const uint32_t id = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((nl * NBT) >> 3) << 17) |
                            ((uint32_t)(kRows >> 4) << 24);
        const uint32_t dcol = tmem + (uint32_t)((t + l0) * NBT);
#pragma unroll
        for (int kk = 0; kk < kKChunk / 16; ++kk)
          mma_bf16(dcol, desc_interleave(a0 + t * kATile + kk * 256, 128, kChunks * 128),
                   desc_interleave(b0 + l0 * kBTile + kk * 256, 128, kChunks * 128), id,
                   (t == 0 && kk == 0) ? 0u : 1u);
      }
    }
    mma_commit(&mbar);
  };

  const int my_i = 32 * (warp & 3) + lane;
  const int my_j0 = (warp >> 2) * kHalf;
  const bool reader = (warp >> 2) < kGroups;
  long long hi[kHalf], lo[kHalf];
#pragma unroll
  for (int j = 0; j < kHalf; ++j) hi[j] = lo[j] = 0;

  uint32_t phase = 0;
  bool timed_out = false;
  const int nchunks = bad ? 0 : (c + kKChunk - 1) / kKChunk;
  auto read_back = [&]() {
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
  };
  if constexpr (kBuf == 2) {
    // chunk k's MMAs run while chunk k+1 is split; chunk k+2 is being staged
    if (nchunks > 0) {
      stage_copy(0);
      cp_async_wait_all();
      __syncthreads();
      split_chunk(0, 0);
      __syncthreads();
      if (nchunks > 1) stage_copy(kKChunk);
      fence_smem_to_async();
      tc_before_sync();
      __syncthreads();
      tc_after_sync();
      if (tid == 0) issue_mma(0);
    }
    for (int kc = 0; kc < nchunks; ++kc) {
      const bool more = kc + 1 < nchunks;
      if (more) {
        cp_async_wait_all();
        __syncthreads();
        split_chunk((kc + 1) & 1, (kc + 1) * kKChunk);
        __syncthreads();
        if (kc + 2 < nchunks) stage_copy((kc + 2) * kKChunk);
      }
      const bool ok = mbar_wait_bounded(&mbar, phase);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        timed_out = true;
        break;
      }
      tc_after_sync();
      read_back();
      fence_smem_to_async();
      tc_before_sync();
      __syncthreads();
      tc_after_sync();
      if (more && tid == 0) issue_mma((kc + 1) & 1);
    }
  } else {
    // one buffer: chunk k+1 is staged while chunk k is split, multiplied and
    // read back; the other CTA on the SM fills the gaps
    if (nchunks > 0) stage_copy(0);
    for (int kc = 0; kc < nchunks; ++kc) {
      cp_async_wait_all();
      __syncthreads();
      split_chunk(0, kc * kKChunk);
      __syncthreads();
      if (kc + 1 < nchunks) stage_copy((kc + 1) * kKChunk);
      fence_smem_to_async();
      tc_before_sync();
      __syncthreads();
      tc_after_sync();
      if (tid == 0) issue_mma(0);
      const bool ok = mbar_wait_bounded(&mbar, phase);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        timed_out = true;
        break;
      }
      tc_after_sync();
      read_back();
      tc_before_sync();
      __syncthreads();
    }
  }
  cp_async_wait_all();
  __syncthreads();  // staging is free: reuse it for the products

  if (!bad && !timed_out && reader) {
#pragma unroll
    for (int j = 0; j < kHalf; ++j) {
      const int jj = my_j0 + j;
      P[my_i * NBT + jj] = (jj < s) ? unfold(hi[j], lo[j], s_cexp_a[my_i], s_cexp_b[jj]) : 0.0;
    }
  }
  __syncthreads();
  if (!bad && !timed_out && tid < kRows) {  // warps 0..3, one row per thread
    const bool live = tid < rows_here;
    const int64_t r = r0 + tid;
    double w[NBT];
#pragma unroll
    for (int j = 0; j < NBT; ++j) w[j] = 0.0;
    if (live) {
#pragma unroll
      for (int j = 0; j < NBT; ++j)
        if (j < s) w[j] = (double)__ldg(reinterpret_cast<const T*>(d.v.p) + r + (int64_t)j * d.v.ld) -
                          P[tid * NBT + j];
      if (d.T != nullptr) {
#pragma unroll
        for (int j = 0; j < NBT; ++j) {
          if (j < s) {
            double x = w[j];
#pragma unroll
            for (int l = 0; l < NBT; ++l)
              if (l < j) x = fma(-w[l], s_T[l * NBT + j], x);
            w[j] = x * s_inv[j];
          }
        }
      }
#pragma unroll
      for (int j = 0; j < NBT; ++j)
        if (j < s) st_elem<T>(d.w, r + (int64_t)j * d.ldw, w[j]);
      if (d.wmax.row != nullptr) {
        unsigned long long mx = 0ull;
#pragma unroll
        for (int j = 0; j < NBT; ++j)
          if (j < s) mx = umax64(mx, abs_bits64((double)(T)w[j]));
        d.wmax.row[r] = umax64(d.wmax.row[r], mx);
      }
    }
    if (d.wmax.col != nullptr) {
#pragma unroll
      for (int j = 0; j < NBT; ++j)
        if (j < s) warp_max_to(live ? abs_bits64((double)(T)w[j]) : 0ull, d.wmax.col + j);
    }
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
    const size_t smem = 1024 + (size_t)ProjCfg<NB>::kBuf * kDigits * (kATile + NB * kKChunk * 2) + \
                        (size_t)kKChunk * kRows * 8;                                               \
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
