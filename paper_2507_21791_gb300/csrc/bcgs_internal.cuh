// Internal declarations shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/bcgs_qr.h"

namespace bcgs {

// ---------------------------------------------------------------- status word
// Lives at the start of every workspace.  code != 0 makes every later kernel of
// the same factorization return immediately.
struct DevStatus {
  int32_t code;
  int32_t block;   // 1-based block column where the failure happened
  int32_t pad[62]; // keeps the following buffers 256-byte aligned
};
static_assert(sizeof(DevStatus) == 256, "status block is 256 bytes");

__device__ __forceinline__ bool failed(const DevStatus* st) {
  return st != nullptr && *((volatile const int32_t*)&st->code) != 0;
}
__device__ __forceinline__ void set_failure(DevStatus* st, int code, int block) {
  if (st != nullptr && atomicCAS(&st->code, 0, code) == 0) st->block = block;
}
// The same answer for every thread of the CTA (thread 0 reads, then a barrier).
// Needed in kernels whose own CTAs may set a failure while others start: a
// per-thread read could then send part of a CTA home before a barrier.
__device__ __forceinline__ bool block_failed(const DevStatus* st) {
  __shared__ int s_failed;
  if (threadIdx.x == 0) s_failed = failed(st) ? 1 : 0;
  __syncthreads();
  const bool f = s_failed != 0;
  __syncthreads();
  return f;
}

// ---------------------------------------------------------------- operands
// A column segment of a tall matrix: ncols columns of m rows, leading dim ld.
// `fp32` selects the storage type (float when nonzero, double otherwise).
struct Seg {
  const void* p;
  int64_t ld;
  int32_t ncols;
  int32_t fp32;
  // Optional per-column max |x| of this segment (bit patterns of non-negative
  // doubles, unsigned order = value order), kept by the kernel that wrote it;
  // null means the tensor-core Gram computes it.
  const unsigned long long* amax;
};

// Running maxima of |x| over what a kernel writes, as above.  `col` gets one
// atomicMax per written column (may be null); `row[r]` is raised to the max of
// the written row r by the thread that owns the row (may be null).
struct MaxOut {
  unsigned long long* col;
  unsigned long long* row;
};

__device__ __forceinline__ unsigned long long abs_bits64(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}
// Warp-wide max of v; lane 0 adds it to *dst.
__device__ __forceinline__ void warp_max_to(unsigned long long v, unsigned long long* dst) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = umax64(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0 && v != 0ull) atomicMax(dst, v);
}

constexpr int kMaxSegA = 4;
constexpr int kMaxSegB = 3;

struct GramDesc {
  Seg a[kMaxSegA];
  Seg b[kMaxSegB];
  int32_t nsa, nsb;
  int32_t na, nb;     // total columns of A and B
  int64_t m;
  int64_t chunk_rows; // rows per partial-sum chunk (fixed by m)
  int32_t nchunks;
  int32_t block;      // 1-based block column reported with a failure (0 = none)
};

inline int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) only when `bytes` exceeds what
// was already set for this kernel (keyed by its address) on the current device.
cudaError_t ensure_dyn_smem_ptr(const void* kernel, size_t bytes);
template <typename Kernel>
inline cudaError_t ensure_dyn_smem(Kernel kern, size_t bytes) {
  return ensure_dyn_smem_ptr(reinterpret_cast<const void*>(kern), bytes);
}

// Deterministic row partition of the Gram reduction: depends on m only.
void gram_partition(int64_t m, int64_t* chunk_rows, int32_t* nchunks);
size_t gram_partial_doubles(int64_t m, int32_t na, int32_t nb);

// Launchers (return cudaError_t of the launch).
cudaError_t launch_gram(const GramDesc& d, double* partial, double* G, int ldg,
                        DevStatus* st, cudaStream_t stream);
// Chunk partials -> G, added in a fixed order that depends on the chunk count only.
cudaError_t launch_gram_reduce(const double* partial, int32_t nchunks, int32_t na, int32_t nb,
                               double* G, int32_t ldg, const DevStatus* st, cudaStream_t stream);
// Tensor-core Gram (gram_tc.cu): same partition and partial layout; needs
// na + nb unsigned 64-bit words of scratch for the column maxima; nb <= 64.
bool gram_tc_supported(const GramDesc& d);
cudaError_t launch_gram_tc(const GramDesc& d, double* partial, double* G, int ldg,
                           unsigned long long* amax, DevStatus* st, cudaStream_t stream);
// Library-wide choice of the Gram engine (bcgs_set_option).
int gram_engine();       // 0 FP64 pipe only, 1 tensor cores for large shapes (default), 2 always
int64_t gram_tc_min_rows();
bool use_tensor_gram(const GramDesc& d);

// W = (V - Qseg C) T^{-1}; C (c x s, ldc) and T (s x s, ldt) on device; T may be null.
struct ProjDesc {
  Seg v;            // m x s input
  Seg q;            // m x c basis (q.ncols = c; may be 0)
  const double* C; int32_t ldc;
  const double* T; int32_t ldt;
  void* w; int64_t ldw; int32_t w_fp32;
  int64_t m; int32_t s;
  // Optional max |q_rk| over k < c per row r of Q (bit patterns); null makes
  // the tensor-core kernel find the row maxima itself.
  const unsigned long long* q_rowmax;
  MaxOut wmax;      // maxima of the written W
};
cudaError_t launch_project(const ProjDesc& d, DevStatus* st, cudaStream_t stream);
// Tensor-core form (proj_tc.cu): s <= 32 and c >= 1.
bool project_tc_supported(const ProjDesc& d);
cudaError_t launch_project_tc(const ProjDesc& d, DevStatus* st, cudaStream_t stream);
bool use_tensor_project(const ProjDesc& d);

// ---------------------------------------------------------------- resident digit store of Q
// Q is kept a second time as digit tiles ready for the tensor cores
// (qstore.cu).  Per 128-row block b and column k: the exponent field exps[b][k]
// of max_{i in b} |q_ik|, and the seven leading balanced 8-bit digits
// (tc_common.cuh) of every q_ik relative to it, as f16: the 62-bit fixed-point
// value without its last digit, which is off by at most 2^-55 of the block's
// column maximum.  Tiles of 128 rows x 128 columns per (b, column group G),
// 224 KB each:
//   [t: digit 0..6][g: 8-column group 0..15][r: 8-row group 0..15][8 rows x 16 B]
// so a 16-column chunk of one digit is 4 KB of contiguous bytes.
constexpr int kStoreRows = 128;
constexpr int kStoreCols = 128;
constexpr int kStoreDigits = 7;
constexpr size_t kStoreTileBytes = (size_t)kStoreDigits * kStoreRows * kStoreCols * 2;
struct QStore {
  uint8_t* dig;
  int32_t* exps;
  int64_t nblk;      // row blocks
  int32_t ngroups;   // column groups
  int32_t ld_exp;    // ngroups * 128
};
size_t qstore_bytes(int64_t m, int32_t n_max);
QStore qstore_at(void* base, int64_t m, int32_t n_max);
// Digits and exponents of store columns [k0, k0 + s) from the s columns of src
// (FP64, ld lds).  The rest of the 16-column chunk holding column k0 + s - 1 is
// written as zeros, and columns of the 8-column group before k0 are rewritten
// from Q (ld ldq) with their unchanged exponents.
// src and Q are float when fp32 (the storage type), else double.
cudaError_t launch_qsplit(const QStore& qs, const void* src, int64_t lds, const void* Q, int64_t ldq, int64_t m,
                          int32_t k0, int32_t s, int32_t fp32, DevStatus* st, int32_t block, cudaStream_t stream);

// Gram from the store (gram_store.cu): G = A^T B with A = store columns [0, na)
// and B = store columns [b0, b0 + nb), b0 a multiple of 8, nb <= 32.  Chunks of
// whole 128-row blocks (gram_store_partition); partials in the layout of
// launch_gram_reduce, which it calls.
struct GramStoreDesc {
  QStore qs;
  int32_t na, b0, nb;
  int32_t nchunks, bpc;   // chunks of bpc blocks
  int64_t m;
  int32_t block;
};
void gram_store_partition(int64_t m, int32_t* nchunks, int32_t* bpc);
bool gram_store_supported(int32_t na, int32_t b0, int32_t nb);
cudaError_t launch_gram_store(const GramStoreDesc& d, double* partial, double* G, int32_t ldg, DevStatus* st,
                              cudaStream_t stream);

// One output of the store projection: W = (V - P_o) T^{-1}; V null means W = P_o T^{-1},
// T null means no solve.
// v and w point to the storage type of the factorization (double, or float
// under StoreProjDesc::fp32); T is always FP64.
struct ProjOut {
  const double* v; int64_t ldv;
  const double* T; int32_t ldt;
  double* w; int64_t ldw;
  MaxOut wmax;
};
// P = Q_{1:c} B with the first c store columns (Q, and the current U block when
// the Grams use the store) and B (c x nouts s, column-major, ldb); output o takes
// columns [o s, o s + s) of P; only the last output may have a triangle T.  A V
// is read before the W of the same row is written, so W may overwrite V.
struct StoreProjDesc {
  QStore qs; int32_t c;
  const double* B; int32_t ldb;
  int32_t s, nouts;
  ProjOut out[2];
  int64_t m;
  int32_t block;
  int32_t* fexp;  // scratch: 32 ints per row block (column exponents of B')
  int32_t fp32;   // X (v) and the outputs (w) are float
};
bool project_store_supported(int32_t s, int32_t nouts);
cudaError_t launch_project_store(const StoreProjDesc& d, DevStatus* st, cudaStream_t stream);

// TSQR of an m x s block.
struct TsqrPlan {
  int64_t m; int32_t s;
  int32_t mt;            // leaf tile rows
  int32_t fan;           // children per tree node
  int32_t nlevels;       // leaf level + node levels (root has 1 node)
  int32_t nodes[32];     // nodes per level (level 0 = leaf tiles)
  size_t off_h;          // leaf reflectors: nodes[0] * mt * s doubles
  size_t off_t0;         // leaf WY triangles T (H_0 ... H_{s-1} = I - V T V^T): nodes[0] * s * s
  size_t off_tau[32];    // taus per level: nodes * s
  size_t off_lvl[32];    // node-level stacked matrices (level >= 1): nodes * (fan*s) * s
  size_t off_b[32];      // apply-phase coefficient blocks per level: nodes * s * s
  size_t doubles;        // total
};
void tsqr_plan(int64_t m, int32_t s, TsqrPlan* plan);
cudaError_t launch_tsqr(const TsqrPlan& plan, Seg a, void* q, int64_t ldq, int32_t q_fp32,
                        double* R, int32_t ldr, double* work, DevStatus* st, int32_t block,
                        cudaStream_t stream, MaxOut qmax = MaxOut{nullptr, nullptr});

// Row-partitioned form (Sec. 3): the rank-ordered sum of the gathered local
// Grams, NaN into a buffer of a failed factorization, the stacked R factors of
// the cross-rank TSQR level and W = A B for the local rows.
cudaError_t launch_rank_sum(const double* recv, int32_t nranks, int32_t na, int32_t nb, int32_t ld, double* G,
                            const DevStatus* st, cudaStream_t stream);
cudaError_t launch_poison_if_failed(double* p, int64_t n, const DevStatus* st, cudaStream_t stream);
cudaError_t launch_stack_r(const double* recv, int32_t nranks, int32_t s, double* out, const DevStatus* st,
                           cudaStream_t stream);
cudaError_t launch_rows_times_small(int64_t m, int32_t s, const void* A, int64_t lda, const double* B, int32_t ldb,
                                    void* W, int64_t ldw, int32_t fp32, MaxOut wmax, const DevStatus* st,
                                    cudaStream_t stream);

// Small FP64 tails (one CTA each); see tail.cu for the exact formulas.
struct TailDesc {
  int32_t s, c;         // block size; rows of the Y / Z blocks (columns of the previous basis)
  const double* G; int32_t ldg;  // reduced Gram output
  int32_t gy, gz, gom, gp, gt;   // row/col offsets, see tail.cu
  const double* S_prev;  // c x s first-pass coefficients S_{1:k-1,k}  (ld = n_max)
  const double* Sd_prev; // s x s S_kk
  double* S_next;        // (c+s) x s S_{1:k,k+1} (ld = n_max)
  double* Sd_next;       // s x s
  double* Y; double* Yd; // c x s (ld n_max) copy of Y_{1:k-1,k}; s x s Y_kk
  double* R; int32_t ldr; int32_t r_row0, r_col0; // R block column destination
  int32_t has_next, chol_next, block;
  int32_t ldsm;          // leading dim of S/Y buffers (n_max)
  // Optional: coefficients of the projections from the digit store, (c+s) rows,
  // leading dimension ldb.  Columns [0, s): [-Y Y_kk^{-1}; Y_kk^{-1}], so that
  // Q_k = [Q_{1:k-1} U_k] B[:, 0:s].  With has_next also columns [s, 2s):
  // [Z - Y M; M] with M = Y_kk^{-1} W (W the bottom s rows of S_{1:k,k+1}).
  double* Bpair; int32_t ldb;
};
cudaError_t launch_tail_1s2s(const TailDesc& d, DevStatus* st, cudaStream_t stream);
// R_kk = chol(T - S^T S) from G = [S; T] = [Q_{1:k} V]^T V, S the top c rows
// (Alg. 1's two normalizations; c = s is the BCGSI+P-1S startup).  S is copied
// to S_out (ld ldsm) unless S_out is null.
cudaError_t launch_tail_pchol(int32_t c, int32_t s, const double* G, int32_t ldg, double* S_out,
                              int32_t ldsm, double* Rkk, int32_t block, DevStatus* st, cudaStream_t stream);
// Copy S12 = G[0:s,0:s] (2S startup), and BCGSI+ R assembly.
cudaError_t launch_copy_small(int32_t rows, int32_t cols, const double* A, int32_t lda,
                              double* B, int32_t ldb, DevStatus* st, cudaStream_t stream);
cudaError_t launch_r_assemble(int32_t c, int32_t s, const double* S, int32_t lds,
                              const double* Y, int32_t ldy, const double* Sd, const double* Yd,
                              double* R, int32_t ldr, int32_t col0, DevStatus* st,
                              cudaStream_t stream);
cudaError_t launch_chol(int32_t s, const double* A, int32_t lda, double* R, int32_t ldr,
                        int32_t block, DevStatus* st, cudaStream_t stream);
cudaError_t launch_zero_lower(int32_t n, double* R, int32_t ldr, cudaStream_t stream);
cudaError_t launch_zero_u64(unsigned long long* p, int64_t n, cudaStream_t stream);
cudaError_t launch_reset_status(DevStatus* st, cudaStream_t stream, DevStatus* st2 = nullptr);
cudaError_t launch_merge_status(DevStatus* st, DevStatus* side, cudaStream_t stream);
// A = I (s x s, leading dimension s).
cudaError_t launch_set_identity(int32_t s, double* A, cudaStream_t stream);
// One bounded wait that runs out after `cycles`: records BCGS_ERR_TIMEOUT.
cudaError_t launch_wait_selftest(DevStatus* st, long long cycles, cudaStream_t stream);

// ---------------------------------------------------------------- instrumentation
// Kernel classes timed by the optional profiler (bcgs_profile_read).
enum ProfClass { kProfGramPartial = 0, kProfGramReduce = 1, kProfProject = 2, kProfTsqr = 3,
                 kProfTail = 4, kProfStoreSplit = 5, kProfClasses = 6 };
void note_launch(int n);
int prof_begin(cudaStream_t stream);  // -1 when profiling is off
void prof_end(int slot, int cls, cudaStream_t stream, double flops, double bytes);

}  // namespace bcgs
