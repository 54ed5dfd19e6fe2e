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
// fixed-point sum: q_ik B_kj = N_ik M_kj 2^(F_j - 124).  The error of one product
// term is below 9 2^(F_j - 62) <= 2^-56.8 max_k |B_kj| max_{i in b} |q_ik|.
//
// Paired form (BCGSI+P-1S / -2S): the step's two projections share one pass
// over [Q_{1:k-1} U_k] with B = [[Y, Z - Y M]; [0, M]], M = Y_kk^{-1} W (tail.cu):
//     Q_k     = (U_k - [Q U_k] B[:, 0:s]) Y_kk^{-1}
//     U_{k+1} = (X_{k+1} - [Q U_k] B[:, s:2s]) S_{k+1,k+1}^{-1}   (1S; 2S: no solve)
// which is Q_{1:k} S_{1:k,k+1} = Q_{1:k-1} Z + Q_k W regrouped (eq. (1)).
#include <string.h>

#include <climits>

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

// One CTA per 128-row block, one thread per row.
__global__ void __launch_bounds__(kStoreRows) qsplit_kernel(QStore qs, const double* src, int64_t lds,
                                                            const double* Q, int64_t ldq, int64_t m,
                                                            int32_t k0, int32_t s, DevStatus* st,
                                                            int32_t block) {
  if (block_failed(st)) return;
  __shared__ int s_wmax[kStoreRows / 32][kQsplitMaxCols];
  __shared__ int s_e[kQsplitMaxCols];
  const int i = threadIdx.x, warp = i >> 5, lane = i & 31;
  const int64_t b = blockIdx.x, r = b * kStoreRows + i;
  const bool live = r < m;
  const int klo = k0 & ~7, kend = k0 + s;
  const int kwr = (kend + 15) & ~15;
  // column k of the store: src column k - k0, or (k < k0) column k of Q
  auto at = [&](int k) { return k >= k0 ? src[r + (int64_t)(k - k0) * lds] : Q[r + (int64_t)k * ldq]; };
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
    uint8_t* dst = qs.dig + ((size_t)(b * qs.ngroups + G) * 8) * (kStoreRows * kStoreCols * 2) +
                   (size_t)(g * 16 + (i >> 3)) * 128 + (i & 7) * 16;
#pragma unroll
    for (int t = 0; t < 8; ++t)
      *reinterpret_cast<uint4*>(dst + (size_t)t * (kStoreRows * kStoreCols * 2)) =
          make_uint4(w[0][t], w[1][t], w[2][t], w[3][t]);
  }
}

// ---------------------------------------------------------------- projection
// Two CTAs per SM (one accumulator set of tensor memory and half the shared
// memory each): the prologue, the read-backs and the FP64 epilogue of one CTA
// overlap the digit stream of the other.
constexpr int kThreads = 256;
constexpr int kRows = 128;                       // rows per CTA (MMA M) = one store block
constexpr int kK = 16;                           // K-values per chunk (one MMA K step)
constexpr int kStages = 2;                       // chunks in flight per CTA
constexpr int kATileT = kRows * kK * 2;          // one digit of one chunk: 4 KB
constexpr int kAStage = kDigits * kATileT;       // 32 KB
constexpr int kGroupChunks = 8;                  // 128 K-values between read-backs
constexpr int kExpInts = 2048 + 64;              // s_exp: c + next <= 2048 + 16
constexpr int kTBytes = 32 * 32 * 8;             // one s x s triangle (s <= 32)
constexpr size_t kDigTile = (size_t)kStoreRows * kStoreCols * 2;  // one digit of a store tile

// NBT: columns of B (all outputs); NOUT: outputs; EXT: an extra A segment of at
// most 16 columns split on the fly, taken as chunk 0 of the contraction.
template <int NBT, int NOUT, bool EXT>
struct SPCfg {
  static constexpr int kBTileT = NBT * kK * 2;   // one digit of one B chunk
  static constexpr int kBStage = kDigits * kBTileT;
  static constexpr int kTmem = kDigits * NBT;    // TMEM columns: the eight levels
  static constexpr int kSmax = NBT / NOUT;       // columns per output
  static constexpr size_t kSmem =
      1024 + (size_t)kStages * kAStage + (size_t)kStages * kBStage + kExpInts * 4 + kTBytes;
};

// Raw B' operands of one thread for one chunk (loaded a chunk ahead).
struct BPair {
  double x, y;
  int kx, ky;  // rows of B (and of s_exp), -1 for none
};

template <int NBT, int NOUT, bool EXT>
__global__ void __launch_bounds__(kThreads, 2) proj_store_kernel(StoreProjDesc d, DevStatus* st) {
  using C = SPCfg<NBT, NOUT, EXT>;
  static_assert(NBT == 16 || NBT == 32, "N tile");
  constexpr int kHalf = NBT / 2;                 // read-back columns per thread
  constexpr int SMAX = C::kSmax;
  constexpr int X0 = EXT ? 1 : 0;                // chunk index of the first Q chunk
  if (block_failed(st)) return;
  extern __shared__ uint8_t dyn[];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ __align__(8) uint64_t done[kStages];
  __shared__ uint32_t tmem_base_s;
  __shared__ int s_F[NBT];
  __shared__ int s_wmax[8][8];
  __shared__ double s_inv[32];
  __shared__ int s_bad;

  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn) + 1023) & ~uintptr_t(1023));
  uint8_t* Aring = base;
  uint8_t* Bring = Aring + kStages * kAStage;
  int* s_exp = reinterpret_cast<int*>(Bring + kStages * C::kBStage);
  double* s_T = reinterpret_cast<double*>(reinterpret_cast<uint8_t*>(s_exp) + kExpInts * 4);
  double* P = reinterpret_cast<double*>(Aring);  // after the last MMA: kRows x NBT products

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c = d.c, s = d.s;
  const int next = EXT ? d.next : 0;
  const int ncolsB = NOUT * s;
  const int64_t b = blockIdx.x, r0 = b * kRows;
  const int nq = (c + kK - 1) / kK;
  const int nch = nq + X0;
  const uint8_t* qblk = d.qs.dig + (size_t)b * d.qs.ngroups * kStoreTileBytes;
  const ProjOut& tri = d.out[NOUT - 1];  // only the last output may have a solve
  const bool has_t = tri.T != nullptr;

  // chunk kc >= X0 holds columns [16 q, 16 q + 16) of Q, q = kc - X0: digit bytes
  // (q % 8) * 4 KB of column group q / 8, for each digit t
  auto issue_copy = [&](int kc) {
    const int slot = kc % kStages, q = kc - X0;
    mbar_arrive_expect_tx(&full[slot], kAStage);
    const uint8_t* src = qblk + (size_t)(q >> 3) * kStoreTileBytes + (size_t)(q & 7) * kATileT;
#pragma unroll
    for (int t = 0; t < kDigits; ++t)
      bulk_g2s(Aring + slot * kAStage + t * kATileT, src + (size_t)t * kDigTile, kATileT, &full[slot]);
  };

  // phase of full[slot] for the copy of chunk kc: the copies into its slot before
  // it (chunk 0 of an extra segment is split in place, not copied)
  auto full_parity = [&](int kc) -> uint32_t {
    return (uint32_t)((kc / kStages) - ((X0 > 0 && kc % kStages == 0) ? 1 : 0)) & 1u;
  };
  int issued = X0;  // chunks whose A operand is on its way (thread 0)
  if (tid == 0) {
    s_bad = 0;
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&full[i]);
      mbar_init(&done[i]);
    }
  }
  for (int k = tid; k < c; k += kThreads) s_exp[k] = d.qs.exps[b * d.qs.ld_exp + k];
  if (has_t)
    for (int e = tid; e < s * s; e += kThreads) {
      const int i = e % s, j = e / s;
      s_T[i * 32 + j] = tri.T[i + (int64_t)j * tri.ldt];
    }
  // extra segment: this thread's row, 8 columns
  double ev[8];
  if constexpr (EXT) {
    const int i = tid & (kRows - 1), h = tid >> 7;
    const int64_t r = r0 + i;
    const bool live = r < d.m;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int col = 8 * h + u;
      ev[u] = (live && col < next) ? d.ext[r + (int64_t)col * d.ld_ext] : 0.0;
      const int mx = __reduce_max_sync(0xffffffffu, exp_field(ev[u]));
      if (lane == 0) s_wmax[warp][u] = mx;
    }
  }
  if (warp == 0) tmem_alloc<C::kTmem>(&tmem_base_s);
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = tmem_base_s;
  if (tid == 0)  // the first Q chunks stream in while the coefficients are prepared
    for (; issued < kStages && issued < nch; ++issued) issue_copy(issued);
  if constexpr (EXT) {
    if (tid < 16) {
      const int h = tid >> 3;
      int e = 0;
#pragma unroll
      for (int w = 0; w < 4; ++w) e = max(e, s_wmax[4 * h + w][tid & 7]);
      s_exp[c + tid] = e;
      if (e == 0x7FF) s_bad = 1;
    }
  }
  if (has_t)
    for (int j = tid; j < s; j += kThreads) s_inv[j] = 1.0 / s_T[j * 32 + j];
  __syncthreads();
  // column exponents of B' = diag(2^E_k) B over k < c + next (eight independent
  // loads in flight per thread)
  {
    const int j = tid >> 3, p = tid & 7;
    int F = INT_MIN;
    bool nf = false;
    if (j < ncolsB) {
      const int K = c + next;
      const double* bj = d.B + (int64_t)j * d.ldb;
      for (int k0 = p; k0 < K; k0 += 64) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = k0 + 8 * u < K ? bj[k0 + 8 * u] : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int k = k0 + 8 * u;
          const int ex = k < K ? s_exp[k] : 0;
          const int e = exp_field(v[u]);
          if (e == 0x7FF || ex == 0x7FF) nf = true;
          else if (e != 0 && ex != 0) F = max(F, e + ex - 1022);
        }
      }
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) F = max(F, __shfl_xor_sync(0xffffffffu, F, o));
    if (__any_sync(0xffffffffu, nf) && lane == 0) s_bad = 1;
    if (p == 0 && j < NBT) s_F[j] = F == INT_MIN ? 0 : F;
  }
  if constexpr (EXT) {
    // digits of the extra segment: chunk 0, ring slot 0 (no copy goes there first)
    const int i = tid & (kRows - 1), h = tid >> 7;
    uint64_t N[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) N[u] = fixed62_offset(ev[u], s_exp[c + 8 * h + u]);
    uint32_t w[4][8];
#pragma unroll
    for (int p = 0; p < 4; ++p)
      digits_pair_f16((uint32_t)(N[2 * p] >> 32), (uint32_t)N[2 * p], (uint32_t)(N[2 * p + 1] >> 32),
                      (uint32_t)N[2 * p + 1], w[p]);
    uint8_t* dst = Aring + h * 2048 + (i >> 3) * 128 + (i & 7) * 16;
#pragma unroll
    for (int t = 0; t < kDigits; ++t)
      *reinterpret_cast<uint4*>(dst + t * kATileT) = make_uint4(w[0][t], w[1][t], w[2][t], w[3][t]);
  }
  __syncthreads();
  const bool bad = s_bad != 0;

  // B' rows of chunk kc -> digit tiles [t][j / 8][g][8 rows x 16 B] (wide-N contiguous).
  // This thread's pair: column j, K-values kk, kk + 1 of the chunk.
  const bool bworker = tid < NBT * 8;
  const int b_jl = lane >> 2, b_pp = lane & 3;
  const int b_jr = warp % (NBT / 8), b_g = warp / (NBT / 8);
  const int b_j = b_jr * 8 + b_jl, b_kk = b_g * 8 + 2 * b_pp;
  const bool b_jv = bworker && b_j < ncolsB;
  const double* b_col = d.B + (int64_t)(b_jv ? b_j : 0) * d.ldb;
  auto load_B = [&](int kc) {
    BPair q;
    int k;
    bool v0, v1;
    if (kc >= X0) {
      k = (kc - X0) * kK + b_kk;
      v0 = k < c;
      v1 = k + 1 < c;
    } else {
      k = c + b_kk;
      v0 = b_kk < next;
      v1 = b_kk + 1 < next;
    }
    v0 = v0 && b_jv;
    v1 = v1 && b_jv;
    q.x = v0 ? b_col[k] : 0.0;
    q.y = v1 ? b_col[k + 1] : 0.0;
    q.kx = v0 ? k : -1;
    q.ky = v1 ? k + 1 : -1;
    return q;
  };
  auto split_B = [&](const BPair& q, uint8_t* dst) {
    if (!bworker) return;
    const int F = s_F[b_j];
    const double xy[2] = {q.x, q.y};
    const int kx[2] = {q.kx, q.ky};
    uint64_t nxy[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const uint64_t bits = (uint64_t)__double_as_longlong(xy[u]);
      const int e = (int)((bits >> 52) & 0x7FF);
      const int ex = kx[u] >= 0 ? s_exp[kx[u]] : 0;
      const bool nz = e != 0 && ex != 0;
      const int dd = F - (e + ex - 1022);
      const uint64_t mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
      const uint64_t mag = (nz && dd < 63) ? ((mant << 9) >> (dd > 0 ? dd : 0)) : 0ull;
      nxy[u] = ((bits >> 63) ? (0ull - mag) : mag) + 0x8080808080808080ull;
    }
    uint32_t out[8];
    digits_pair_f16((uint32_t)(nxy[0] >> 32), (uint32_t)nxy[0], (uint32_t)(nxy[1] >> 32), (uint32_t)nxy[1],
                    out);
    uint8_t* pp = dst + b_jr * 256 + b_g * 128 + b_jl * 16 + b_pp * 4;
#pragma unroll
    for (int t = 0; t < kDigits; ++t) *reinterpret_cast<uint32_t*>(pp + t * C::kBTileT) = out[t];
  };
  // digit t of A times digit tiles [B_0 .. B_{7-t}] (one operand of (8 - t) NBT
  // rows) lands tile u in level t + u: TMEM columns (t + u) NBT.
  auto issue_mma = [&](int kc) {
    const int slot = kc % kStages;
    const uint32_t a0 = smem_u32(Aring + slot * kAStage);
    const uint32_t b0 = smem_u32(Bring + slot * C::kBStage);
    const bool first = (kc % kGroupChunks) == 0;
#pragma unroll 1
    for (int t = 0; t < kDigits; ++t)
      mma_bf16(tmem + (uint32_t)(t * NBT), desc_interleave(a0 + t * kATileT, 2048, 128),
               desc_interleave(b0, 128, 256), idesc_f16(kRows, (kDigits - t) * NBT),
               (first && t == 0) ? 0u : 1u);
    mma_commit(&done[slot]);
  };

  const int my_j0 = (warp >> 2) * kHalf;
  long long hi[kHalf], lo[kHalf];
#pragma unroll
  for (int j = 0; j < kHalf; ++j) hi[j] = lo[j] = 0;
  // levels 0..3 fold into hi, 4..7 into lo (the fold of fold_levels in two halves)
  auto read_back = [&]() {
    const uint32_t addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)my_j0;
#pragma unroll
    for (int g8 = 0; g8 < kHalf; g8 += 8) {
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        uint32_t r[4][8];
#pragma unroll
        for (int l = 0; l < 4; ++l) tmem_ld8_nowait(addr + (uint32_t)((4 * half + l) * NBT + g8), r[l]);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int32_t L0 = __float2int_rn(__uint_as_float(r[0][j]));
          const int32_t L1 = __float2int_rn(__uint_as_float(r[1][j]));
          const int32_t L2 = __float2int_rn(__uint_as_float(r[2][j]));
          const int32_t L3 = __float2int_rn(__uint_as_float(r[3][j]));
          if (half == 0)
            hi[g8 + j] += ((long long)((L0 << 8) + L1) << 16) + (long long)((L2 << 8) + L3);
          else
            lo[g8 + j] += ((long long)L0 << 24) + ((long long)L1 << 16) + ((long long)L2 << 8) + (long long)L3;
        }
      }
    }
  };

  bool timed_out = false;
  int waited = X0;    // chunks whose copies thread 0 saw land
  bool t0_fail = false;
  const int nrun = bad ? 0 : nch;
  BPair cur = load_B(0);
  for (int kc = 0; kc < nrun; ++kc) {
    const int slot = kc % kStages;
    bool ok = true;
    if (kc >= kStages) ok = mbar_wait_bounded(&done[slot], ((kc / kStages) - 1) & 1);  // B slot free
    if (ok) split_B(cur, Bring + slot * C::kBStage);
    if (kc + 1 < nrun) cur = load_B(kc + 1);  // in flight during the barrier and the MMAs
    fence_smem_to_async();
    tc_before_sync();
    if (__syncthreads_or(!ok || t0_fail)) {
      timed_out = true;
      break;
    }
    tc_after_sync();
    if (tid == 0) {
      bool okc = true;
      if (kc >= X0) {
        okc = mbar_wait_bounded(&full[slot], full_parity(kc));
        if (okc) waited = kc + 1;
      }
      if (okc) {
        issue_mma(kc);
        // refill the slot of chunk kc - 1 (free once its MMAs are done) with chunk kc + 1
        const int nk = kc + kStages - 1;
        if (kc >= 1 && nk < nch && nk >= issued) {
          if (mbar_wait_bounded(&done[(kc - 1) % kStages], ((kc - 1) / kStages) & 1)) {
            issue_copy(nk);
            issued = nk + 1;
          } else {
            okc = false;
          }
        }
      }
      t0_fail = !okc;
    }
    if ((kc + 1) % kGroupChunks == 0 && kc + 1 < nrun) {
      // the group ends with chunk kc: read it back before the next group overwrites it
      const bool okr = mbar_wait_bounded(&done[slot], (kc / kStages) & 1);
      if (__syncthreads_or(!okr || t0_fail)) {
        timed_out = true;
        break;
      }
      tc_after_sync();
      read_back();
      tc_before_sync();
    }
  }
  if (!timed_out && nrun > 0) {
    const bool okr = mbar_wait_bounded(&done[(nrun - 1) % kStages], ((nrun - 1) / kStages) & 1);
    if (__syncthreads_or(!okr || t0_fail)) {
      timed_out = true;
    } else {
      tc_after_sync();
      read_back();
    }
  }
  if (timed_out && tid == 0) {
    // let the copies still in flight land before the CTA's shared memory goes away
    for (int kc = waited; kc < issued; ++kc) mbar_wait_bounded(&full[kc % kStages], full_parity(kc));
  }
  __syncthreads();
  const bool run = !bad && !timed_out;
  if (run) {
    const int i = 32 * (warp & 3) + lane;
#pragma unroll
    for (int j = 0; j < kHalf; ++j) P[i * NBT + my_j0 + j] = fixed_to_double(hi[j], lo[j], s_F[my_j0 + j]);
  }
  __syncthreads();
  // epilogue: one thread per (output, row)
  const int o = tid >> 7, i = tid & (kRows - 1);
  const int64_t r = r0 + i;
  const bool mine = run && o < NOUT;
  const bool live = mine && r < d.m;
  const ProjOut& out = d.out[o < NOUT ? o : 0];
  double w[SMAX];
#pragma unroll
  for (int j = 0; j < SMAX; ++j) w[j] = 0.0;
  if (live) {
#pragma unroll
    for (int j = 0; j < SMAX; ++j)
      if (j < s) w[j] = out.v != nullptr ? out.v[r + (int64_t)j * out.ldv] - P[i * NBT + o * s + j]
                                         : P[i * NBT + o * s + j];
  }
  __syncthreads();  // every V (and E) read before any W, which may overwrite them, is written
  if (live) {
    if (o == NOUT - 1 && has_t) {
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
      if (j < s) out.w[r + (int64_t)j * out.ldw] = w[j];
    if (out.wmax.row != nullptr) {
      unsigned long long mx = 0ull;
#pragma unroll
      for (int j = 0; j < SMAX; ++j)
        if (j < s) mx = umax64(mx, abs_bits64(w[j]));
      out.wmax.row[r] = umax64(out.wmax.row[r], mx);
    }
  }
  if (mine && out.wmax.col != nullptr) {  // warp-uniform: o and run are
#pragma unroll
    for (int j = 0; j < SMAX; ++j)
      if (j < s) warp_max_to(live ? abs_bits64(w[j]) : 0ull, out.wmax.col + j);
  }
  if (bad && tid == 0) set_failure(st, BCGS_ERR_NONFINITE, d.block);
  if (timed_out && tid == 0) set_failure(st, BCGS_ERR_TIMEOUT, d.block);
  tc_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc<C::kTmem>(tmem);
}

template <int NBT, int NOUT, bool EXT>
cudaError_t launch_sp(const StoreProjDesc& d, DevStatus* st, cudaStream_t stream) {
  const size_t smem = SPCfg<NBT, NOUT, EXT>::kSmem;
  cudaError_t e = ensure_dyn_smem(proj_store_kernel<NBT, NOUT, EXT>, smem);
  if (e != cudaSuccess) return e;
  proj_store_kernel<NBT, NOUT, EXT><<<(unsigned)d.qs.nblk, kThreads, smem, stream>>>(d, st);
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_qsplit(const QStore& qs, const double* src, int64_t lds, const double* Q, int64_t ldq,
                          int64_t m, int32_t k0, int32_t s, DevStatus* st, int32_t block,
                          cudaStream_t stream) {
  if (s < 1 || s > 64 || qs.nblk <= 0 || k0 < 0 || k0 + s > qs.ld_exp) return cudaErrorInvalidValue;
  const int slot = prof_begin(stream);
  qsplit_kernel<<<(unsigned)qs.nblk, kStoreRows, 0, stream>>>(qs, src, lds, Q, ldq, m, k0, s, st, block);
  // reads the s new columns, writes 16 bytes of digits per element
  prof_end(slot, kProfStoreSplit, stream, 0.0, (double)m * s * (8.0 + 16.0));
  note_launch(1);
  return cudaGetLastError();
}

bool project_store_supported(int32_t s, int32_t nouts, int32_t next) {
  if (s < 1 || next < 0 || next > 16) return false;
  if (nouts == 2) return s <= 16;
  return nouts == 1 && (next > 0 ? s <= 16 : s <= 32);
}

cudaError_t launch_project_store(const StoreProjDesc& d, DevStatus* st, cudaStream_t stream) {
  if (!project_store_supported(d.s, d.nouts, d.next) || d.c < 0 || d.c + d.next > kExpInts - 64 ||
      d.qs.nblk < ceil_div(d.m, kRows))
    return cudaErrorInvalidValue;
  for (int o = 0; o + 1 < d.nouts; ++o)
    if (d.out[o].T != nullptr) return cudaErrorInvalidValue;  // only the last output has a solve
  if (d.m == 0) return cudaSuccess;
  const int slot = prof_begin(stream);
  cudaError_t e;
  if (d.nouts == 2) e = launch_sp<32, 2, true>(d, st, stream);
  else if (d.next > 0) e = launch_sp<16, 1, true>(d, st, stream);
  else if (d.s <= 16) e = launch_sp<16, 1, false>(d, st, stream);
  else e = launch_sp<32, 1, false>(d, st, stream);
  if (e != cudaSuccess) return e;
  const double K = (double)d.c + d.next, nw = (double)d.nouts * d.s;
  double nv = 0;
  for (int o = 0; o < d.nouts; ++o) nv += d.out[o].v != nullptr ? d.s : 0;
  prof_end(slot, kProfProject, stream, 2.0 * (double)d.m * K * nw + (double)d.m * d.s * d.s,
           8.0 * (double)d.m * (K + nv + nw));
  note_launch(1);
  return cudaGetLastError();
}

}  // namespace bcgs
