// Resident digit store of Q and the projection that reads it.
//
// Every projection of the block step multiplies the whole basis Q_{1:c} by a
// small coefficient matrix (Alg. 1 and Alg. 2: U = (X - Q S) S_kk^{-1},
// Q_k = (U - Q Y) Y_kk^{-1}).  Q only grows, so its exact digit form
// (tc_common.cuh, balanced 8-bit digits) is made once per block column, when the
// block is written, and kept in HBM beside Q: each later projection bulk-copies
// the digit tiles into shared memory and runs the tensor cores on them, with no
// per-element work on Q.
//
// Exponents are per 128-row block b and column k (E_bk > log2 max_{i in b}
// |q_ik|).  In  sum_k q_ik B_kj  the factor 2^E_bk moves onto row k of B, so
// B'_kj = B_kj 2^E_bk is split against one exponent per column j,
// F_j > log2 max_k |B'_kj|, and the products of all k add up in one exact
// fixed-point sum: q_ik B_kj = N_ik M_kj 2^(F_j - 124).  The store keeps seven of
// the eight digits of N_ik (off by at most 129 units of 2^(E_bk - 62)); with the
// truncation of B' and the dropped levels the error of one product term is below
// 2^-53.9 max_k |B_kj| max_{i in b} |q_ik|.
//
// Paired form (BCGSI+P-1S / -2S): the step's two projections share one pass
// over [Q_{1:k-1} U_k] with B = [[Y, Z - Y M]; [0, M]], M = Y_kk^{-1} W (tail.cu):
//     Q_k     = (U_k - [Q U_k] B[:, 0:s]) Y_kk^{-1}
//     U_{k+1} = (X_{k+1} - [Q U_k] B[:, s:2s]) S_{k+1,k+1}^{-1}   (1S; 2S: no solve)
// which is Q_{1:k} S_{1:k,k+1} = Q_{1:k-1} Z + Q_k W regrouped (eq. (1)).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include <climits>
#include <mutex>

#include "tc_common.cuh"

namespace bcgs {

size_t qstore_bytes(int64_t m, int32_t n_max) {
  const int64_t nblk = ceil_div(m, kStoreRows);
  const int64_t ngroups = ceil_div(n_max, kStoreCols);
  const size_t dig = (size_t)nblk * ngroups * kStoreTileBytes;
  const size_t exps = (size_t)nblk * ngroups * kStoreCols * sizeof(int32_t);
  return dig + (exps + 255) / 256 * 256;
}

QStore qstore_at(void* base, int64_t m, int32_t n_max) {
  QStore q;
  q.nblk = ceil_div(m, kStoreRows);
  q.ngroups = (int32_t)ceil_div(n_max, kStoreCols);
  q.ld_exp = q.ngroups * kStoreCols;
  q.dig = reinterpret_cast<uint8_t*>(base);
  q.exps = reinterpret_cast<int32_t*>(q.dig + (size_t)q.nblk * q.ngroups * kStoreTileBytes);
  return q;
}

namespace {
using namespace tc;

constexpr int kQsplitMaxCols = 72;  // s <= 64 plus up to 7 columns of the group before k0

__device__ __forceinline__ int exp_field(double v) {
  return (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7FF);
}

// One CTA per 128-row block, one thread per row.  T is the storage type of src
// and Q (float values convert to double exactly).
template <typename T>
__global__ void __launch_bounds__(kStoreRows) qsplit_kernel(QStore qs, const T* src, int64_t lds, const T* Q,
                                                            int64_t ldq, int64_t m, int32_t k0, int32_t s,
                                                            DevStatus* st, int32_t block) {
  if (block_failed(st)) return;
  __shared__ int s_wmax[kStoreRows / 32][kQsplitMaxCols];
  __shared__ int s_e[kQsplitMaxCols];
  const int i = threadIdx.x, warp = i >> 5, lane = i & 31;
  const int64_t b = blockIdx.x, r = b * kStoreRows + i;
  const bool live = r < m;
  const int klo = k0 & ~7, kend = k0 + s;
  const int kwr = (kend + 15) & ~15;
  // column k of the store: src column k - k0, or (k < k0) column k of Q
  auto at = [&](int k) -> double {
    return k >= k0 ? (double)src[r + (int64_t)(k - k0) * lds] : (double)Q[r + (int64_t)k * ldq];
  };
  for (int k = klo; k < kend; ++k) {
    const int e = live ? exp_field(at(k)) : 0;
    const int mx = __reduce_max_sync(0xffffffffu, e);
    if (lane == 0) s_wmax[warp][k - klo] = mx;
  }
  __syncthreads();
  for (int k = klo + i; k < kend; k += kStoreRows) {
    int e = 0;
#pragma unroll
    for (int w = 0; w < kStoreRows / 32; ++w) e = max(e, s_wmax[w][k - klo]);
    s_e[k - klo] = e;
    qs.exps[b * qs.ld_exp + k] = e;
    if (e == 0x7FF) set_failure(st, BCGS_ERR_NONFINITE, block);
  }
  __syncthreads();
  for (int g8 = klo; g8 < kwr; g8 += 8) {
    uint64_t N[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int k = g8 + u;
      const double v = (live && k < kend) ? at(k) : 0.0;
      N[u] = fixed62_offset(v, k < kend ? s_e[k - klo] : 0);
    }
    uint32_t w[4][8];
#pragma unroll
    for (int p = 0; p < 4; ++p)
      digits_pair_f16((uint32_t)(N[2 * p] >> 32), (uint32_t)N[2 * p], (uint32_t)(N[2 * p + 1] >> 32),
                      (uint32_t)N[2 * p + 1], w[p]);
    const int G = g8 / kStoreCols, g = (g8 % kStoreCols) / 8;
    uint8_t* dst = qs.dig + ((size_t)(b * qs.ngroups + G) * kStoreDigits) * (kStoreRows * kStoreCols * 2) +
                   (size_t)(g * 16 + (i >> 3)) * 128 + (i & 7) * 16;
#pragma unroll
    for (int t = 0; t < kStoreDigits; ++t)
      *reinterpret_cast<uint4*>(dst + (size_t)t * (kStoreRows * kStoreCols * 2)) =
          make_uint4(w[0][t], w[1][t], w[2][t], w[3][t]);
  }
}

// The common case of the split: k0 a multiple of 8 and at most NC <= 16 columns
// (s <= 16): each thread holds its row's values in registers, so all loads are
// in flight at once and Q is read once.
template <int NC, typename T>
__global__ void __launch_bounds__(kStoreRows) qsplit_reg_kernel(QStore qs, const T* src, int64_t lds, int64_t m,
                                                                int32_t k0, int32_t s, DevStatus* st,
                                                                int32_t block) {
  if (block_failed(st)) return;
  __shared__ int s_wmax[kStoreRows / 32][NC];
  const int i = threadIdx.x, warp = i >> 5, lane = i & 31;
  const int64_t b = blockIdx.x, r = b * kStoreRows + i;
  const bool live = r < m;
  double v[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) v[k] = (live && k < s) ? (double)src[r + (int64_t)k * lds] : 0.0;
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    const int mx = __reduce_max_sync(0xffffffffu, exp_field(v[k]));
    if (lane == 0) s_wmax[warp][k] = mx;
  }
  __syncthreads();
  int ce[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    int e = 0;
#pragma unroll
    for (int w = 0; w < kStoreRows / 32; ++w) e = max(e, s_wmax[w][k]);
    ce[k] = k < s ? e : 0;
  }
  if (i < s) {
    int e = 0;
#pragma unroll
    for (int w = 0; w < kStoreRows / 32; ++w) e = max(e, s_wmax[w][i]);
    qs.exps[b * qs.ld_exp + k0 + i] = e;
    if (e == 0x7FF) set_failure(st, BCGS_ERR_NONFINITE, block);
  }
  // columns [k0, k0 + s) and zeros up to the end of the 16-column chunk
  const int kwr = (((k0 + s) + 15) & ~15) - k0;
#pragma unroll
  for (int g8 = 0; g8 < NC + 16; g8 += 8) {
    if (g8 < kwr) {
      uint64_t N[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) N[u] = (g8 + u < NC) ? fixed62_offset(v[g8 + u], ce[g8 + u]) : fixed62_offset(0.0, 0);
      uint32_t w[4][8];
#pragma unroll
      for (int p = 0; p < 4; ++p)
        digits_pair_f16((uint32_t)(N[2 * p] >> 32), (uint32_t)N[2 * p], (uint32_t)(N[2 * p + 1] >> 32),
                        (uint32_t)N[2 * p + 1], w[p]);
      const int col = k0 + g8;
      const int G = col / kStoreCols, g = (col % kStoreCols) / 8;
      uint8_t* dst = qs.dig + ((size_t)(b * qs.ngroups + G) * kStoreDigits) * (kStoreRows * kStoreCols * 2) +
                     (size_t)(g * 16 + (i >> 3)) * 128 + (i & 7) * 16;
#pragma unroll
      for (int t = 0; t < kStoreDigits; ++t)
        *reinterpret_cast<uint4*>(dst + (size_t)t * (kStoreRows * kStoreCols * 2)) =
            make_uint4(w[0][t], w[1][t], w[2][t], w[3][t]);
    }
  }
}

// ---------------------------------------------------------------- projection
// Persistent, one CTA per SM, warp-specialized:
//   warp 0       bulk copies of the A digit chunks and the MMAs (one thread);
//   warps 1..3   per row block: its exponents, the column exponents F_j of B',
//                and the B' digits of every chunk;
//   warps 4..11  read-back of the accumulators and the FP64 epilogue;
//   warps 12..15 (paired form only) the epilogue of the second output: V minus
//                the products, the triangular solve and the stores, so that the
//                FP64 solve of block b runs while warps 4..11 read back block b+1.
// Chunks, B' splits, read-backs and epilogues of consecutive row blocks overlap
// through mbarriers; two accumulator sets in tensor memory alternate per group
// of 128 K-values.
constexpr int kRows = 128;                       // rows per block (MMA M)
constexpr int kK = 16;                           // K-values per chunk (one MMA K step)
constexpr int kStages = 3;                       // chunks in flight
constexpr int kATileT = kRows * kK * 2;          // one digit of one chunk: 4 KB
constexpr int kAStage = kStoreDigits * kATileT;  // 28 KB: the store's digits of one chunk
constexpr int kGroupChunks = 8;                  // 128 K-values between read-backs
constexpr int kMaxK = 2048;                      // store columns of one projection at most
constexpr size_t kDigTile = (size_t)kStoreRows * kStoreCols * 2;  // one digit of a store tile
constexpr int kCtl = 0;                          // warp roles
constexpr int kSplit0 = 1, kSplitWarps = 3;
constexpr int kRead0 = 4, kReadWarps = 8;
constexpr int kEpi0 = 12, kEpiWarps = 4;         // paired form only
// s_exp (the K block exponents of a row block), rounded to 16 bytes
__host__ __device__ constexpr size_t exp_bytes(int K) { return ((size_t)(K + 16) * 4 + 15) / 16 * 16; }

// Threads and the register split per warpgroup (setmaxnreg; warpgroup 0 =
// control + splitters, 1 and 2 = read-back, 3 = epilogue of the paired form).
// The shares, times 128 threads each, add up to at most the launch's registers
// (threads x kLaunchRegs); launch_sp checks that against the compiled kernel.
template <int NOUT>
struct Roles {
  static constexpr int kThreads = 32 * (NOUT == 2 ? kEpi0 + kEpiWarps : kRead0 + kReadWarps);
  static constexpr int kLaunchRegs = NOUT == 2 ? 128 : 168;  // 65536 / threads, a multiple of 8
  static constexpr int kRegsLow = NOUT == 2 ? 96 : 104;       // control + splitters
  static constexpr int kRegsHigh = NOUT == 2 ? 168 : 192;     // read-back
  static constexpr int kRegsEpi = 80;                         // epilogue warps (paired form)
  static constexpr int kSplitTotal = 128 * (kRegsLow + 2 * kRegsHigh + (NOUT == 2 ? kRegsEpi : 0));
  static_assert(kSplitTotal <= kThreads * kLaunchRegs, "register split above the launch's registers");
};

// Output o occupies tile columns [o SMAX, o SMAX + s) (B column o s + jj); with
// two outputs each read-back thread holds one output of its row: the first
// output's epilogue runs from its registers, the second output's products go
// through W (128 rows x SMAX doubles, column-major) to the epilogue warps; the
// single form stages products in P.  B itself is staged in shared memory when it
// fits (kSmemLimit).
template <int NBT, int NOUT>
struct SPCfg {
  static constexpr int kBTileT = NBT * kK * 2;   // one digit of one B chunk
  static constexpr int kBStage = kDigits * kBTileT;
  static constexpr int kBRing = 4;               // B chunks in the ring (>= kStages)
  static constexpr int kAcc = kDigits * NBT;     // TMEM columns of one accumulator set
  static constexpr int kTmem = 2 * kAcc;
  static constexpr int kSmax = NBT / NOUT;       // columns per output
  static constexpr size_t kPBytes = (size_t)kRows * (NOUT == 1 ? NBT : kSmax) * 8;  // P, or W (paired)
  // everything but s_exp (exp_bytes(K)) and the staged B
  static constexpr size_t kFixed = 1024 + (size_t)kStages * kAStage + (size_t)kBRing * kBStage + kPBytes +
                                   32 * 32 * 8;
};
constexpr size_t kSmemLimit = 232448 - 4096;     // dynamic shared memory we ask for at most

// Column exponents of B' = diag(2^E_b) B for every row block b:
//     F_bj = max_k (e(B_k,bcol(j)) + E_bk) - 1022   (exponent fields; 0 for none)
// one warp per block, the exponent fields of B staged once per CTA.  A
// non-finite entry of B or of the block exponents raises BCGS_ERR_NONFINITE.
template <int NBT, int NOUT>
__global__ void __launch_bounds__(256) proj_fexp_kernel(StoreProjDesc d, DevStatus* st) {
  constexpr int SMAX = NBT / NOUT;
  if (block_failed(st)) return;
  extern __shared__ int16_t eB[];  // K x NBT, tile columns
  const int K = d.c, s = d.s;
  for (int e = threadIdx.x; e < K * NBT; e += blockDim.x) {
    const int j = e / K, k = e - j * K;  // consecutive threads: consecutive rows of one column
    const int o = j / SMAX, jj = j - o * SMAX;
    eB[k * NBT + j] = (int16_t)((o < NOUT && jj < s) ? exp_field(d.B[k + (int64_t)(o * s + jj) * d.ldb]) : 0);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  bool nf = false;
  for (int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; b < d.qs.nblk; b += nw) {
    const int32_t* ex = d.qs.exps + b * d.qs.ld_exp;
    int F = INT_MIN;
    for (int k0 = 0; k0 < K; k0 += 32) {
      const int E = k0 + lane < K ? ex[k0 + lane] : 0;
      nf |= E == 0x7FF;
      const int kn = K - k0 < 32 ? K - k0 : 32;
      for (int u = 0; u < kn; ++u) {
        const int Eu = __shfl_sync(0xffffffffu, E, u);
        const int eb = lane < NBT ? eB[(k0 + u) * NBT + lane] : 0;
        nf |= eb == 0x7FF;
        if (eb != 0 && Eu != 0 && Eu != 0x7FF && eb != 0x7FF) F = max(F, eb + Eu - 1022);
      }
    }
    if (lane < NBT) d.fexp[b * NBT + lane] = F == INT_MIN ? 0 : F;
  }
  if (__any_sync(0xffffffffu, nf) && lane == 0) set_failure(st, BCGS_ERR_NONFINITE, d.block);
}

// Poll `mbar` for phase `parity` until it completes, *abort is raised, or the
// bound runs out (then *abort is raised): true when the phase completed.
__device__ __forceinline__ bool wait_or_abort(uint64_t* mbar, uint32_t parity, volatile int* abort) {
  const long long t0 = clock64();
  while (!mbar_try(smem_u32(mbar), parity)) {
    if (*abort) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort = 1;
      return false;
    }
  }
  return true;
}

template <int NBT, int NOUT, bool F32>
__global__ void __launch_bounds__(Roles<NOUT>::kThreads, 1) proj_store_kernel(StoreProjDesc d, int32_t b_staged,
                                                                               const __grid_constant__ CUtensorMap amap,
                                                                               int32_t use_amap, DevStatus* st) {
  using C = SPCfg<NBT, NOUT>;
  using Rl = Roles<NOUT>;
  constexpr int kThreads = Rl::kThreads;
  static_assert(NBT == 16 || NBT == 32, "N tile");
  constexpr int kHalf = NBT / 2;                 // read-back columns per thread
  constexpr int SMAX = C::kSmax;
  if (block_failed(st)) return;
  extern __shared__ uint8_t dyn[];
  __shared__ __align__(8) uint64_t fullA[kStages];    // A chunk landed (copy)
  __shared__ __align__(8) uint64_t done[kStages];     // MMAs of the chunk in the slot done
  __shared__ __align__(8) uint64_t bready[C::kBRing]; // B' digits of the chunk written (splitter warps)
  __shared__ __align__(8) uint64_t bdone[C::kBRing];  // MMAs that read the B slot done
  __shared__ __align__(8) uint64_t accdone[2];        // accumulator set complete
  __shared__ __align__(8) uint64_t accfree[2];        // accumulator set read (8 warps)
  __shared__ __align__(8) uint64_t fready[2];         // F_j of a block written
  __shared__ __align__(8) uint64_t ffree[2];          // F_j of a block used
  __shared__ __align__(8) uint64_t wfull;             // paired: W holds the block's second-output products
  __shared__ __align__(8) uint64_t wempty;            // paired: W read by the epilogue warps
  __shared__ uint32_t tmem_base_s;
  __shared__ int s_F[2][NBT];
  __shared__ double s_inv[32];
  __shared__ volatile int s_abort;
  __shared__ int s_bad;

  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn) + 1023) & ~uintptr_t(1023));
  const int K = d.c, s = d.s;
  uint8_t* Aring = base;
  uint8_t* Bring = Aring + kStages * kAStage;
  double* P = reinterpret_cast<double*>(Bring + C::kBRing * C::kBStage);  // W in the paired form
  double* s_T = reinterpret_cast<double*>(reinterpret_cast<uint8_t*>(P) + C::kPBytes);
  int* s_exp = reinterpret_cast<int*>(s_T + 32 * 32);
  // staged B (b_staged != 0), row-major by tile column: B'_(k, j) at Bsm[k * kLdj + j]; a pitch
  // of NBT + 4 doubles keeps the column-per-lane and pair-per-lane reads at two wavefronts
  constexpr int kLdj = NBT + 4;
  double* Bsm = reinterpret_cast<double*>(reinterpret_cast<uint8_t*>(s_exp) + exp_bytes(K));

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nch = (K + kK - 1) / kK;
  const int ngrp = (nch + kGroupChunks - 1) / kGroupChunks;
  const int64_t nblk = d.qs.nblk;
  const int nbl = blockIdx.x < nblk ? (int)((nblk - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  const int total = nbl * nch;
  const ProjOut& tri = d.out[NOUT - 1];  // only the last output may have a solve
  const bool has_t = tri.T != nullptr;
  auto blk_of = [&](int bi) { return (int64_t)blockIdx.x + (int64_t)bi * gridDim.x; };

  if (tid == 0) {
    s_abort = 0;
    s_bad = 0;
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&fullA[i]);
      mbar_init(&done[i]);
    }
    for (int i = 0; i < C::kBRing; ++i) {
      mbar_init_count(&bready[i], kSplitWarps);
      mbar_init(&bdone[i]);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accdone[i]);
      mbar_init_count(&accfree[i], kReadWarps);
      mbar_init(&fready[i]);
      mbar_init(&ffree[i]);
    }
    mbar_init_count(&wfull, 32 * kReadWarps / 2);  // the second output's 128 read-back threads
    mbar_init_count(&wempty, 32 * kEpiWarps);      // the 128 epilogue threads
  }
  if (has_t) {
    for (int e = tid; e < s * s; e += kThreads) {
      const int i = e % s, j = e / s;
      s_T[i * 32 + j] = tri.T[i + (int64_t)j * tri.ldt];
    }
  }
  // B column of tile column j, -1 for a padding column
  auto bcol = [&](int j) { const int o = j / SMAX, jj = j - o * SMAX; return (o < NOUT && jj < s) ? o * s + jj : -1; };
  // B: staged once per CTA (it is the same for every row block) when it fits
  if (b_staged)
    for (int e = tid; e < NBT * K; e += kThreads) {
      const int j = e / K, k = e - j * K;
      const int bc = bcol(j);
      Bsm[k * kLdj + j] = bc >= 0 ? d.B[k + (int64_t)bc * d.ldb] : 0.0;
    }
  // element (k, tile column j) of B
  auto bval = [&](int k, int j) -> double {
    if (b_staged) return Bsm[k * kLdj + j];
    const int bc = bcol(j);
    return bc >= 0 ? d.B[k + (int64_t)bc * d.ldb] : 0.0;
  };
  // X and the outputs in the storage type (float when F32; the products and the
  // epilogue stay FP64); the maxima are those of the stored values
  auto vload = [&](const ProjOut& o, int64_t idx) -> double {
    if constexpr (F32)
      return (double)reinterpret_cast<const float*>(o.v)[idx];
    else
      return o.v[idx];
  };
  auto wstore = [&](const ProjOut& o, int64_t idx, double x) {
    if constexpr (F32)
      reinterpret_cast<float*>(o.w)[idx] = (float)x;
    else
      o.w[idx] = x;
  };
  auto stored = [&](double x) -> double {
    if constexpr (F32)
      return (double)(float)x;
    else
      return x;
  };
  if (warp == kCtl) tmem_alloc<C::kTmem>(&tmem_base_s);
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  if (has_t)
    for (int j = tid; j < s; j += kThreads) s_inv[j] = 1.0 / s_T[j * 32 + j];
  __syncthreads();
  const uint32_t tmem = tmem_base_s;

  // Warpgroup 0 (control + splitters), and the epilogue warpgroup of the paired
  // form, hand registers to the two read-back warpgroups (Roles: the shares add
  // up to at most the launch's registers).
  if (warp < kRead0) setmaxnreg_dec<Rl::kRegsLow>();
  else if (warp < kRead0 + kReadWarps) setmaxnreg_inc<Rl::kRegsHigh>();
  else setmaxnreg_dec<Rl::kRegsEpi>();

  if (warp == kCtl) {
    // ------------------------------------------------ copies and MMAs
    if (lane == 0) {
      // one chunk = the 4 KB piece kc & 7 of the 7 digit tiles of store tile (b, kc >> 3):
      // one tensor copy through amap (box {256, 2, 1, 7, 1} of u64 at x = 0), else 7 bulk copies
      // The loop keeps every index as a counter (chunk, slot, phase, block) that
      // steps by one: no division by the run-time chunk count on this thread,
      // whose per-chunk instructions set the pace of the MMAs.
      // copy side: chunk `issued` = piece ikc of block ibi, into slot islot (phase iph)
      int issued = 0, islot = 0, iph = 0, ikc = 0, ibi = 0, got = 0;
      auto issue_copy = [&]() {
        const int64_t b = blk_of(ibi);
        mbar_arrive_expect_tx(&fullA[islot], kAStage);
        if (use_amap) {
          tma_load_5d(Aring + islot * kAStage, &amap, 0, 0, ikc & 7, 0,
                      (int32_t)(b * d.qs.ngroups + (ikc >> 3)), &fullA[islot]);
        } else {
          const uint8_t* src = d.qs.dig + (size_t)b * d.qs.ngroups * kStoreTileBytes +
                               (size_t)(ikc >> 3) * kStoreTileBytes + (size_t)(ikc & 7) * kATileT;
#pragma unroll
          for (int t = 0; t < kStoreDigits; ++t)
            bulk_g2s(Aring + islot * kAStage + t * kATileT, src + (size_t)t * kDigTile, kATileT, &fullA[islot]);
        }
        ++issued;
        if (++islot == kStages) islot = 0, iph ^= 1;
        if (++ikc == nch) ikc = 0, ++ibi;
      };
      while (issued < kStages && issued < total) issue_copy();
      // Event loop: a slot is refilled as soon as the MMAs of its last chunk are
      // done, and a chunk's MMAs go out as soon as its operands are ready, so all
      // kStages copies stay in flight while the tensor core waits for data.  No
      // progress for kWaitCycles (or an abort elsewhere) ends the loop.
      // MMA side: chunk g = piece kc of block bi, A slot `slot` (phase aph), B slot
      // `bslot` (phase bph), accumulator group gg (first chunk of its group: kq == 0)
      int g = 0, slot = 0, aph = 0, bslot = 0, bph = 0, kc = 0, kq = 0, gg = 0;
      int need = 0;  // 0 = A of chunk g, 1 = its B' digits, 2 = a free accumulator set
      long long idle0 = clock64();
      while (g < total) {
        bool progress = false;
        // the slot of chunk `issued` last held chunk issued - kStages (< g: its MMAs went out)
        if (issued < total && issued - kStages < g && mbar_test(&done[islot], iph ^ 1)) {
          issue_copy();
          progress = true;
        }
        if (need == 0 && mbar_test(&fullA[slot], aph)) {
          need = 1;
          got = g + 1;
        }
        if (need == 1 && mbar_test(&bready[bslot], bph)) need = 2;
        if (need == 2 && (kq != 0 || gg < 2 || mbar_test(&accfree[gg & 1], ((gg >> 1) - 1) & 1))) {
          tc_after_sync();
          const uint32_t a0 = smem_u32(Aring + slot * kAStage);
          const uint32_t b0 = smem_u32(Bring + bslot * C::kBStage);
          const uint32_t acc = tmem + (uint32_t)((gg & 1) * C::kAcc);
          // digit t of A (t < 7: the store keeps seven) times digit tiles
          // [B_0 .. B_{7-t}] of B' (eight): tile u lands in level t + u
#pragma unroll
          for (int t = 0; t < kStoreDigits; ++t)
            mma_bf16(acc + (uint32_t)(t * NBT), desc_interleave(a0 + t * kATileT, 2048, 128),
                     desc_interleave(b0, 128, 256), idesc_f16(kRows, (kDigits - t) * NBT),
                     (kq == 0 && t == 0) ? 0u : 1u);
          mma_commit(&done[slot]);
          mma_commit(&bdone[bslot]);
          const bool blk_end = kc == nch - 1;
          if (kq == kGroupChunks - 1 || blk_end) mma_commit(&accdone[gg & 1]);
          ++g;
          if (++slot == kStages) slot = 0, aph ^= 1;
          if (++bslot == C::kBRing) bslot = 0, bph ^= 1;
          if (blk_end) {
            kc = 0, kq = 0, ++gg;
          } else {
            ++kc;
            if (++kq == kGroupChunks) kq = 0, ++gg;
          }
          need = 0;
          progress = true;
        }
        if (progress) {
          idle0 = clock64();
        } else if (s_abort) {
          break;
        } else if (clock64() - idle0 > kWaitCycles) {
          s_abort = 1;
          break;
        }
      }
      // copies still in flight land before the CTA's shared memory goes away
      for (int g = got; g < issued; ++g) mbar_wait_bounded(&fullA[g % kStages], (g / kStages) & 1);
    }
  } else if (warp < kRead0) {
    // ------------------------------------------------ per-block exponents and B' digits
    // (after an abort every wait returns at once and the work is skipped, but the
    // named barriers are still passed by all splitter threads)
    constexpr int kSp = 32 * kSplitWarps;
    const int sp = tid - 32 * kSplit0;          // 0..kSp-1
    // The block's exponents and F come from global memory; for K <= kPre * kSp
    // those of block bi + 1 are loaded into registers while block bi is split,
    // so a block's start does not wait for them (small K: a block's splits are
    // shorter than that latency).
    constexpr int kPre = 3;
    const bool pre = K <= kPre * kSp;
    int pe[kPre], pf = 0;
    auto fetch = [&](int64_t b) {
#pragma unroll
      for (int u = 0; u < kPre; ++u) {
        const int k = sp + u * kSp;
        pe[u] = k < K ? d.qs.exps[b * d.qs.ld_exp + k] : 0;
      }
      pf = sp < NBT ? d.fexp[b * NBT + sp] : 0;
    };
    if (pre && nbl > 0) fetch(blk_of(0));
    for (int bi = 0; bi < nbl; ++bi) {
      const int64_t b = blk_of(bi);
      // this block's exponents (the previous block's splits are all done: same warps)
      named_bar_sync(1, kSp);
      if (!s_abort) {
        if (pre) {
#pragma unroll
          for (int u = 0; u < kPre; ++u)
            if (sp + u * kSp < K) s_exp[sp + u * kSp] = pe[u];
        } else {
          for (int k = sp; k < K; k += kSp) s_exp[k] = d.qs.exps[b * d.qs.ld_exp + k];
        }
      }
      named_bar_sync(1, kSp);
      // F of block bi (proj_fexp_kernel) goes to buffer bi & 1, free once block bi - 2 is unfolded
      if (bi >= 2) wait_or_abort(&ffree[bi & 1], ((bi >> 1) - 1) & 1, &s_abort);
      named_bar_sync(1, kSp);
      if (sp < NBT && !s_abort) s_F[bi & 1][sp] = pre ? pf : d.fexp[b * NBT + sp];
      named_bar_sync(1, kSp);
      if (sp == 0) mbar_arrive(&fready[bi & 1]);
      if (pre && bi + 1 < nbl && !s_abort) fetch(blk_of(bi + 1));
      const int* sF = s_F[bi & 1];
      for (int kc = 0; kc < nch; ++kc) {
        const int g = bi * nch + kc, slot = g % C::kBRing;
        bool ok = true;
        if (g >= C::kBRing)
          ok = __all_sync(0xffffffffu, wait_or_abort(&bdone[slot], ((g / C::kBRing) - 1) & 1, &s_abort));
        if (ok && !s_abort) {
          uint8_t* dst = Bring + slot * C::kBStage;
          // K-pairs e = sp, sp + kSp, ... -> column j, K-values kk, kk + 1
#pragma unroll
          for (int h = 0; h < (NBT * 8 + kSp - 1) / kSp; ++h) {
            const int e = sp + kSp * h;
            if (e < NBT * 8) {
              const int el = e & 31, ew = e >> 5;
              const int jl = el >> 2, pp = el & 3, jr = ew % (NBT / 8), gq = ew / (NBT / 8);
              const int j = jr * 8 + jl, kk = gq * 8 + 2 * pp;
              const int k = kc * kK + kk;
              const bool jv = bcol(j) >= 0;
              const bool v0 = jv && k < K, v1 = jv && k + 1 < K;
              const double xy[2] = {v0 ? bval(k, j) : 0.0, v1 ? bval(k + 1, j) : 0.0};
              const int exk[2] = {v0 ? s_exp[k] : 0, v1 ? s_exp[k + 1] : 0};
              const int Fj = sF[j];
              uint64_t nxy[2];
#pragma unroll
              for (int u = 0; u < 2; ++u) {
                const uint64_t bits = (uint64_t)__double_as_longlong(xy[u]);
                const int e2 = (int)((bits >> 52) & 0x7FF);
                const bool nz = e2 != 0 && exk[u] != 0;
                const int dd = Fj - (e2 + exk[u] - 1022);
                const uint64_t mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
                const uint64_t mag = (nz && dd < 63) ? ((mant << 9) >> (dd > 0 ? dd : 0)) : 0ull;
                nxy[u] = ((bits >> 63) ? (0ull - mag) : mag) + 0x8080808080808080ull;
              }
              uint32_t out[8];
              digits_pair_f16((uint32_t)(nxy[0] >> 32), (uint32_t)nxy[0], (uint32_t)(nxy[1] >> 32),
                              (uint32_t)nxy[1], out);
              uint8_t* pp8 = dst + jr * 256 + gq * 128 + jl * 16 + pp * 4;
#pragma unroll
              for (int t = 0; t < kDigits; ++t) *reinterpret_cast<uint32_t*>(pp8 + t * C::kBTileT) = out[t];
            }
          }
          fence_smem_to_async();
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&bready[slot]);
      }
    }
  } else if (warp < kRead0 + kReadWarps) {
    // ------------------------------------------------ read-back and epilogue
    // (same rule: after an abort the work is skipped, the named barriers are not)
    const int rt = tid - 32 * kRead0;           // 0..255; TMEM quadrant warp % 4
    const int half = (warp - kRead0) / 4;       // column half of the read-back
    const int qrow = 32 * (warp & 3) + lane;    // TMEM lane = row of the block
    const int my_j0 = half * kHalf;
    for (int bi = 0; bi < nbl; ++bi) {
      const int64_t b = blk_of(bi), r0 = b * kRows;
      long long hi[kHalf], lo[kHalf];
#pragma unroll
      for (int j = 0; j < kHalf; ++j) hi[j] = lo[j] = 0;
      for (int grp = 0; grp < ngrp; ++grp) {
        const int gg = bi * ngrp + grp;
        const bool ok = __all_sync(0xffffffffu, wait_or_abort(&accdone[gg & 1], (gg >> 1) & 1, &s_abort));
        const bool go = __all_sync(0xffffffffu, ok && !s_abort);
        if (go) {
          tc_after_sync();
          const uint32_t addr =
              tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((gg & 1) * C::kAcc + my_j0);
          // Levels 4..7 of every column octet stay raw in registers; levels 0..3 are
          // folded into hi octet by octet.  Once every load has landed the accumulator
          // set goes back to the MMAs, and levels 4..7 are folded into lo after that.
          constexpr int kOct = kHalf / 8;
          uint32_t rk[kOct][4][8], ra[4][8];
#pragma unroll
          for (int oc = 0; oc < kOct; ++oc)
#pragma unroll
            for (int l = 0; l < 4; ++l) tmem_ld8_nowait(addr + (uint32_t)((4 + l) * NBT + 8 * oc), rk[oc][l]);
#pragma unroll
          for (int oc = 0; oc < kOct; ++oc) {
#pragma unroll
            for (int l = 0; l < 4; ++l) tmem_ld8_nowait(addr + (uint32_t)(l * NBT + 8 * oc), ra[l]);
            tmem_wait_ld();
            // levels 0..3 into hi (weights 2^24, 2^16, 2^8, 1 above 2^32):
            // |L0 2^8 + L1| < 2^30 and |L2 2^8 + L3| < 2^31 fit int32
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int32_t L0 = __float2int_rn(__uint_as_float(ra[0][j]));
              const int32_t L1 = __float2int_rn(__uint_as_float(ra[1][j]));
              const int32_t L2 = __float2int_rn(__uint_as_float(ra[2][j]));
              const int32_t L3 = __float2int_rn(__uint_as_float(ra[3][j]));
              hi[8 * oc + j] += ((long long)((L0 << 8) + L1) << 16) + (long long)((L2 << 8) + L3);
            }
          }
          tc_before_sync();
          __syncwarp();
          if (lane == 0) mbar_arrive(&accfree[gg & 1]);
#pragma unroll
          for (int oc = 0; oc < kOct; ++oc)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int32_t L4 = __float2int_rn(__uint_as_float(rk[oc][0][j]));
              const int32_t L5 = __float2int_rn(__uint_as_float(rk[oc][1][j]));
              const int32_t L6 = __float2int_rn(__uint_as_float(rk[oc][2][j]));
              const int32_t L7 = __float2int_rn(__uint_as_float(rk[oc][3][j]));
              lo[8 * oc + j] +=
                  ((long long)L4 << 24) + ((long long)L5 << 16) + ((long long)L6 << 8) + (long long)L7;
            }
        } else {
          __syncwarp();
          if (lane == 0) mbar_arrive(&accfree[gg & 1]);
        }
      }
      const bool fok = __all_sync(0xffffffffu, wait_or_abort(&fready[bi & 1], (bi >> 1) & 1, &s_abort));
      const int* sF = s_F[bi & 1];
      if constexpr (NOUT == 2) {
        // this warp's output (half) of row qrow, straight from the accumulators
        const int64_t r = r0 + qrow;
        const bool live = fok && !s_abort && r < d.m;
        double w[kHalf];
#pragma unroll
        for (int j = 0; j < kHalf; ++j)
          w[j] = (live && j < s) ? fixed_to_double(hi[j], lo[j], sF[my_j0 + j]) : 0.0;
        named_bar_sync(2, 32 * kReadWarps);
        if (rt == 0) mbar_arrive(&ffree[bi & 1]);
        if (half == 1) {
          // the second output's epilogue runs on the epilogue warps: hand them
          // the products once they have taken the previous block's
          if (bi >= 1) wait_or_abort(&wempty, (bi - 1) & 1, &s_abort);
          if (!s_abort) {
#pragma unroll
            for (int j = 0; j < kHalf; ++j) P[j * kRows + qrow] = w[j];
          }
          mbar_arrive(&wfull);
        } else {
          // the first output has no triangular solve (launch_project_store checks)
          const ProjOut& out = d.out[0];
          if (live) {
            if (out.v != nullptr) {
#pragma unroll
              for (int j = 0; j < kHalf; ++j)
                if (j < s) w[j] = vload(out, r + (int64_t)j * out.ldv) - w[j];
            }
#pragma unroll
            for (int j = 0; j < kHalf; ++j)
              if (j < s) wstore(out, r + (int64_t)j * out.ldw, w[j]);
            if (out.wmax.row != nullptr) {
              unsigned long long mx = 0ull;
#pragma unroll
              for (int j = 0; j < kHalf; ++j)
                if (j < s) mx = umax64(mx, abs_bits64(stored(w[j])));
              out.wmax.row[r] = umax64(out.wmax.row[r], mx);
            }
          }
          if (out.wmax.col != nullptr) {  // warp-uniform
#pragma unroll
            for (int j = 0; j < kHalf; ++j)
              if (j < s) warp_max_to(live ? abs_bits64(stored(w[j])) : 0ull, out.wmax.col + j);
          }
        }
      } else {
        // one output: the two halves of a row meet in P, one thread per row
        if (fok && !s_abort) {
#pragma unroll
          for (int j = 0; j < kHalf; ++j)
            P[qrow * NBT + my_j0 + j] = fixed_to_double(hi[j], lo[j], sF[my_j0 + j]);
        }
        named_bar_sync(2, 32 * kReadWarps);
        if (rt == 0) mbar_arrive(&ffree[bi & 1]);
        const int i = rt & (kRows - 1);
        const int64_t r = r0 + i;
        const bool mine = rt < kRows;
        const bool live = mine && r < d.m && fok && !s_abort;
        const ProjOut& out = d.out[0];
        double w[SMAX];
#pragma unroll
        for (int j = 0; j < SMAX; ++j) w[j] = 0.0;
        if (live) {
#pragma unroll
          for (int j = 0; j < SMAX; ++j)
            if (j < s)
              w[j] = out.v != nullptr ? vload(out, r + (int64_t)j * out.ldv) - P[i * NBT + j] : P[i * NBT + j];
        }
        named_bar_sync(2, 32 * kReadWarps);  // P read before the next block writes it
        if (live) {
          if (has_t) {
#pragma unroll
            for (int j = 0; j < SMAX; ++j) {
              if (j < s) {
                double x = w[j];
#pragma unroll
                for (int l = 0; l < SMAX; ++l)
                  if (l < j) x = fma(-w[l], s_T[l * 32 + j], x);
                w[j] = x * s_inv[j];
              }
            }
          }
#pragma unroll
          for (int j = 0; j < SMAX; ++j)
            if (j < s) wstore(out, r + (int64_t)j * out.ldw, w[j]);
          if (out.wmax.row != nullptr) {
            unsigned long long mx = 0ull;
#pragma unroll
            for (int j = 0; j < SMAX; ++j)
              if (j < s) mx = umax64(mx, abs_bits64(stored(w[j])));
            out.wmax.row[r] = umax64(out.wmax.row[r], mx);
          }
        }
        if (mine && out.wmax.col != nullptr) {  // warp-uniform: rt < 128 is
#pragma unroll
          for (int j = 0; j < SMAX; ++j)
            if (j < s) warp_max_to(live ? abs_bits64(stored(w[j])) : 0ull, out.wmax.col + j);
        }
      }
    }
  } else if constexpr (NOUT == 2) {
    // ------------------------------------------------ epilogue of the second output (paired form)
    // One thread per row of the block: V minus the products (from W), the
    // triangular solve, the stores and the maxima.  Only bounded mbarrier waits;
    // after an abort the work is skipped.
    constexpr int kSm = C::kSmax;
    const int i = tid - 32 * kEpi0;
    const ProjOut& out = d.out[1];
    for (int bi = 0; bi < nbl; ++bi) {
      const int64_t r = blk_of(bi) * kRows + i;
      const bool inrow = r < d.m;
      // V of this row is loaded while the read-back finishes the block, and the
      // next block's rows of V are sent toward L2 (when these warps set the pace
      // the wait below is short and the load latency would show)
      double v[kSm];
#pragma unroll
      for (int j = 0; j < kSm; ++j) v[j] = (out.v != nullptr && inrow && j < s) ? vload(out, r + (int64_t)j * out.ldv) : 0.0;
      if (out.v != nullptr && bi + 1 < nbl) {
        const int64_t rn = blk_of(bi + 1) * kRows + i;
        if (rn < d.m)
          for (int j = 0; j < s; ++j)
            asm volatile("prefetch.global.L2 [%0];\n" ::"l"(reinterpret_cast<const char*>(out.v) +
                                                            (rn + (int64_t)j * out.ldv) * (F32 ? 4 : 8)));
      }
      const bool ok = wait_or_abort(&wfull, bi & 1, &s_abort);
      double w[kSm];
#pragma unroll
      for (int j = 0; j < kSm; ++j) w[j] = P[j * kRows + i];
      mbar_arrive(&wempty);
      const bool live = ok && !s_abort && inrow;
      if (live) {
        if (out.v != nullptr) {
#pragma unroll
          for (int j = 0; j < kSm; ++j) w[j] = v[j] - w[j];
        }
        if (has_t) {
#pragma unroll
          for (int j = 0; j < kSm; ++j) {
            if (j < s) {
              double x = w[j];
#pragma unroll
              for (int l = 0; l < kSm; ++l)
                if (l < j) x = fma(-w[l], s_T[l * 32 + j], x);
              w[j] = x * s_inv[j];
            }
          }
        }
#pragma unroll
        for (int j = 0; j < kSm; ++j)
          if (j < s) wstore(out, r + (int64_t)j * out.ldw, w[j]);
        if (out.wmax.row != nullptr) {
          unsigned long long mx = 0ull;
#pragma unroll
          for (int j = 0; j < kSm; ++j)
            if (j < s) mx = umax64(mx, abs_bits64(stored(w[j])));
          out.wmax.row[r] = umax64(out.wmax.row[r], mx);
        }
      }
      if (out.wmax.col != nullptr) {  // warp-uniform
#pragma unroll
        for (int j = 0; j < kSm; ++j)
          if (j < s) warp_max_to(live ? abs_bits64(stored(w[j])) : 0ull, out.wmax.col + j);
      }
    }
  }
  tc_before_sync();
  __syncthreads();
  if (tid == 0) {
    if (s_bad) set_failure(st, BCGS_ERR_NONFINITE, d.block);
    else if (s_abort) set_failure(st, BCGS_ERR_TIMEOUT, d.block);
  }
  if (warp == kCtl) tmem_dealloc<C::kTmem>(tmem);
}

int g_sm_count = 0;

// cuTensorMapEncodeTiled from the CUDA driver, looked up once through the runtime
// (no link against libcuda); null when the driver does not provide it.
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// The digit store as a 5-d tensor of u64 (innermost first): 256 x 2 (one 4 KB
// piece = 16 columns of one digit of a tile), 8 pieces, 7 digits, nblk * ngroups
// tiles; strides 2 KB, 4 KB, 32 KB, 224 KB.  False when it cannot be encoded.
bool store_tensor_map(const QStore& qs, CUtensorMap* map) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
  if (fn == nullptr) return false;
  const cuuint64_t dims[5] = {256, 2, 8, (cuuint64_t)kStoreDigits, (cuuint64_t)qs.nblk * (cuuint64_t)qs.ngroups};
  const cuuint64_t strides[4] = {2048, (cuuint64_t)kATileT, (cuuint64_t)kDigTile, (cuuint64_t)kStoreTileBytes};
  const cuuint32_t box[5] = {256, 2, 1, (cuuint32_t)kStoreDigits, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  if (dims[4] == 0 || dims[4] > (1ull << 32)) return false;
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, qs.dig, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The kernel was compiled with at least the registers its split hands out.
template <int NBT, int NOUT, bool F32>
bool split_regs_ok() {
  cudaFuncAttributes fa;
  return cudaFuncGetAttributes(&fa, proj_store_kernel<NBT, NOUT, F32>) == cudaSuccess &&
         (int64_t)fa.numRegs * Roles<NOUT>::kThreads >= Roles<NOUT>::kSplitTotal;
}

template <int NBT, int NOUT, bool F32>
cudaError_t launch_sp(const StoreProjDesc& d, DevStatus* st, cudaStream_t stream) {
  using C = SPCfg<NBT, NOUT>;
  using Rl = Roles<NOUT>;
  const size_t bbytes = (size_t)(NBT + 4) * (size_t)d.c * sizeof(double);
  const size_t fixed = C::kFixed + exp_bytes(d.c);
  const int32_t staged = fixed + bbytes <= kSmemLimit ? 1 : 0;
  const size_t smem = fixed + (staged ? bbytes : 0);
  // the register split draws on the registers the CTA is launched with: refuse a
  // build whose kernel was compiled with fewer than the split adds up to
  static const bool regs_ok = split_regs_ok<NBT, NOUT, F32>();
  if (!regs_ok) return cudaErrorInvalidConfiguration;
  cudaError_t e = ensure_dyn_smem(proj_store_kernel<NBT, NOUT, F32>, smem);
  if (e != cudaSuccess) return e;
  int sms = g_sm_count;
  if (sms <= 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 152;
    g_sm_count = sms;
  }
  const size_t fsmem = (size_t)d.c * NBT * sizeof(int16_t);
  e = ensure_dyn_smem(proj_fexp_kernel<NBT, NOUT>, fsmem);
  if (e != cudaSuccess) return e;
  const int64_t fgrid = ceil_div(d.qs.nblk, 8);
  proj_fexp_kernel<NBT, NOUT><<<(unsigned)(fgrid < 4 * sms ? fgrid : 4 * sms), 256, fsmem, stream>>>(d, st);
  const unsigned grid = (unsigned)(d.qs.nblk < sms ? d.qs.nblk : (int64_t)sms);
  CUtensorMap amap;
  memset(&amap, 0, sizeof(amap));
  const int32_t use_amap = store_tensor_map(d.qs, &amap) ? 1 : 0;
  proj_store_kernel<NBT, NOUT, F32><<<grid, Rl::kThreads, smem, stream>>>(d, staged, amap, use_amap, st);
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_qsplit(const QStore& qs, const void* src, int64_t lds, const void* Q, int64_t ldq, int64_t m,
                          int32_t k0, int32_t s, int32_t fp32, DevStatus* st, int32_t block, cudaStream_t stream) {
  if (s < 1 || s > 64 || qs.nblk <= 0 || k0 < 0 || k0 + s > qs.ld_exp) return cudaErrorInvalidValue;
  const int slot = prof_begin(stream);
  const unsigned grid = (unsigned)qs.nblk;
  auto run = [&](auto tag) {
    using T = decltype(tag);
    const T* sp = reinterpret_cast<const T*>(src);
    const T* qp = reinterpret_cast<const T*>(Q);
    if (k0 % 8 == 0 && s <= 8)
      qsplit_reg_kernel<8, T><<<grid, kStoreRows, 0, stream>>>(qs, sp, lds, m, k0, s, st, block);
    else if (k0 % 8 == 0 && s <= 16)
      qsplit_reg_kernel<16, T><<<grid, kStoreRows, 0, stream>>>(qs, sp, lds, m, k0, s, st, block);
    else
      qsplit_kernel<T><<<grid, kStoreRows, 0, stream>>>(qs, sp, lds, qp, ldq, m, k0, s, st, block);
  };
  if (fp32)
    run(0.0f);
  else
    run(0.0);
  // reads the s new columns, writes 2 kStoreDigits bytes of digits per element
  prof_end(slot, kProfStoreSplit, stream, 0.0, (double)m * s * ((fp32 ? 4.0 : 8.0) + 2.0 * kStoreDigits));
  note_launch(1);
  return cudaGetLastError();
}

bool project_store_supported(int32_t s, int32_t nouts) {
  if (s < 1) return false;
  return nouts == 2 ? s <= 16 : (nouts == 1 && s <= 32);
}

cudaError_t launch_project_store(const StoreProjDesc& d, DevStatus* st, cudaStream_t stream) {
  if (!project_store_supported(d.s, d.nouts) || d.c < 0 || d.c > kMaxK || d.c > d.qs.ld_exp ||
      d.qs.nblk < ceil_div(d.m, kRows) || d.fexp == nullptr)
    return cudaErrorInvalidValue;
  for (int o = 0; o + 1 < d.nouts; ++o)
    if (d.out[o].T != nullptr) return cudaErrorInvalidValue;  // only the last output has a solve
  if (d.m == 0) return cudaSuccess;
  const int slot = prof_begin(stream);
  cudaError_t e;
  if (d.fp32) {
    if (d.nouts == 2) e = launch_sp<32, 2, true>(d, st, stream);
    else if (d.s <= 16) e = launch_sp<16, 1, true>(d, st, stream);
    else e = launch_sp<32, 1, true>(d, st, stream);
  } else {
    if (d.nouts == 2) e = launch_sp<32, 2, false>(d, st, stream);
    else if (d.s <= 16) e = launch_sp<16, 1, false>(d, st, stream);
    else e = launch_sp<32, 1, false>(d, st, stream);
  }
  if (e != cudaSuccess) return e;
  note_launch(1);  // the exponent kernel
  const double K = (double)d.c, nw = (double)d.nouts * d.s;
  double nv = 0;
  for (int o = 0; o < d.nouts; ++o) nv += d.out[o].v != nullptr ? d.s : 0;
  prof_end(slot, kProfProject, stream, 2.0 * (double)d.m * K * nw + (double)d.m * d.s * d.s,
           8.0 * (double)d.m * (K + nv + nw));
  note_launch(1);
  return cudaGetLastError();
}

}  // namespace bcgs
