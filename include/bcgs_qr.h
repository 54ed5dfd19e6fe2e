/*
 * bcgs_qr.h -- C ABI of the GB300 (sm_103a) reorthogonalized block classical
 * Gram-Schmidt QR library.
 *
 * Operation (Sec. 1): the economic QR X = Q R of a tall-skinny m x n matrix X,
 * Q^T Q = I, R upper triangular with positive diagonal, computed block column
 * by block column, X = [X_1 ... X_q], q = ceil(n / s) blocks of s columns (the
 * last one ragged, n mod s columns, when s does not divide n), by one of
 *   BCGS_BCGSI_PLUS       BCGSI+ (Sec. 1, Table 1: 4 synchronizations per block)
 *   BCGS_BCGSI_PLUS_P_1S  BCGSI+P-1S (Alg. 2: 1 synchronization per block)
 *   BCGS_BCGSI_PLUS_P_2S  BCGSI+P-2S (Sec. 2: Alg. 2 with TSQR as the first
 *                         intraorthogonalization, 2 synchronizations per block)
 *   BCGS_BCGS_PIPI_PLUS   BCGS-PIPI+ (Alg. 1: both passes normalized by the
 *                         Pythagorean Cholesky, 2 synchronizations per block;
 *                         O(u) loss of orthogonality only while O(u) kappa^2 <= 1)
 *   BCGS_BCGSI_PLUS_1S    BCGSI+1s, also called BCGSI+LS (Sec. 2, one-sync
 *                         subsection; Table 1): Alg. 2 without its first
 *                         Cholesky line, so the first pass is not normalized
 *                         (S_{k+1,k+1} = I, no T); 1 synchronization per block,
 *                         O(u) kappa^2 loss of orthogonality while
 *                         O(u) kappa^3 <= 1
 * A synchronization point of the paper (one MPI_Allreduce, Sec. 3) is here one
 * streaming pass over HBM that ends in a deterministic grid-wide reduction.
 *
 * Conventions for every entry point:
 *   - Matrices are column-major (MATLAB indexing, Sec. 1) with a leading
 *     dimension >= their row count.  X, Q, U and all workspace are DEVICE
 *     pointers; R is a device FP64 n x n array whose strictly lower triangle
 *     the library sets to zero.
 *   - Under BCGS_FP64, X and Q are double*.  Under BCGS_FP32_STORAGE, X and Q are
 *     float* (stored and streamed in FP32) while every inner product is
 *     accumulated, and every small factor (Cholesky, triangular solves, R) is
 *     computed, in FP64.  R is always double*.
 *   - The caller owns every buffer.  The library never allocates device memory
 *     and never frees caller memory; X is read-only and must not alias Q:
 *     bcgs_qr_factor, bcgs_qr_factor_host (Xd, Qd) and bcgs_qr_factor_batched
 *     return BCGS_ERR_INVALID_ARG, before enqueueing anything, when the memory
 *     of X and Q overlaps (in-place factorization is not supported).
 *   - Calls are asynchronous and ordered on the given CUDA stream (a
 *     cudaStream_t passed as void*; NULL = the legacy default stream).
 *     Invalid arguments are reported synchronously by the return value and
 *     nothing is enqueued.  Numerical breakdown, non-finite data and device
 *     timeouts are recorded in a status word inside the workspace; once it is
 *     set, the remaining kernels of that factorization do nothing, and the
 *     status is returned by bcgs_qr_sync / bcgs_qr_factor_status.
 *   - Results are deterministic: the reduction order depends only on the
 *     problem shape, never on scheduling.
 */
#ifndef BCGS_QR_H
#define BCGS_QR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define BCGS_API __attribute__((visibility("default")))
#else
#define BCGS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BCGS_OK = 0,
  BCGS_ERR_INVALID_ARG = 1,    /* bad size, leading dimension, pointer or enum  */
  BCGS_ERR_NOT_SPD = 2,        /* a Pythagorean Cholesky (Alg. 1, Alg. 2) met a pivot <= 0 */
  BCGS_ERR_RANK_DEFICIENT = 3, /* an intraorthogonalization (TSQR) gave a zero R diagonal */
  BCGS_ERR_NONFINITE = 4,      /* NaN or Inf reached a factor                    */
  BCGS_ERR_WORKSPACE = 5,      /* workspace too small or misaligned              */
  BCGS_ERR_TIMEOUT = 6,        /* a bounded device wait gave up                  */
  BCGS_ERR_STATE = 7,          /* call out of order (step after finish, ...)    */
  BCGS_ERR_CUDA = 8,           /* a CUDA runtime call failed                     */
  BCGS_ERR_COMM = 9            /* the all-gather callback of the row-partitioned form failed */
} bcgs_status;

typedef enum {
  BCGS_BCGSI_PLUS = 0,
  BCGS_BCGSI_PLUS_P_1S = 1,
  BCGS_BCGSI_PLUS_P_2S = 2,
  BCGS_BCGS_PIPI_PLUS = 3,
  BCGS_BCGSI_PLUS_1S = 4
} bcgs_variant;

typedef enum { BCGS_FP64 = 0, BCGS_FP32_STORAGE = 1 } bcgs_precision;

typedef struct bcgs_qr_s* bcgs_qr_t;

/* Human-readable name of a status code (static string, never NULL). */
BCGS_API const char* bcgs_status_string(int status);

/* Library version as major*10000 + minor*100 + patch. */
BCGS_API int bcgs_version(void);

/* ---------------------------------------------------------------------------
 * Whole factorization.
 * ------------------------------------------------------------------------- */

/* Bytes of device workspace needed by a factorization (or a handle) of an
 * m x n_max matrix with block size s.  Requirements: 1 <= s <= 64,
 * 1 <= n_max <= m, n_max <= 2048.  The paper takes n = q s; when s does not
 * divide n the last block is ragged (r = n mod s columns): the full blocks are
 * factored by the variant (BCGSI+P-1S / -2S finalize their delayed block first),
 * then the ragged block takes one step of the variant of the same stability
 * range that finalizes a block at once: a BCGS-PIPI+ step (Alg. 1) under
 * BCGSI+P-1S and BCGS-PIPI+, a BCGSI+ step under BCGSI+ and BCGSI+P-2S
 * (n < s: TSQR alone).  Writes *bytes; returns BCGS_OK or
 * BCGS_ERR_INVALID_ARG.  With s <= 32 and the tensor engine selected for m
 * rows (BCGS_OPT_GRAM_ENGINE below), under either storage type, the size
 * includes the digit store of Q: 14 bytes per element of the m x n_max basis
 * (rounded up to 128
 * columns), one 32-bit exponent per 128 rows and column, and 32 more per 128
 * rows.  A factorization given a workspace sized without the store (for example
 * under the FP64 engine) runs without it. */
BCGS_API int bcgs_qr_workspace_size(int64_t m, int32_t n_max, int32_t s, int variant,
                           int precision, size_t* bytes);

/* Factor X (m x n, leading dimension ldx) into Q (m x n, ldq) and R (n x n,
 * ldr): the whole of Alg. 2 (or the chosen variant) enqueued on `stream`.
 * `workspace` is a device buffer of at least bcgs_qr_workspace_size bytes,
 * 256-byte aligned, not shared with any other call in flight.  Returns after
 * enqueueing; read the outcome with bcgs_qr_factor_status.  From 2^17 rows,
 * with the digit store and s a multiple of 16, the digit split of each next
 * block of X runs ahead on a side stream of the calling thread while the
 * current step's small FP64 tail runs: it is forked from `stream` by an event
 * after the step's Gram and joined back before the step's projection, so all
 * work stays ordered on `stream` (also inside a graph capture of `stream`; the
 * side stream is created on a first call outside capture, and a first call
 * under capture runs without it).  The results are the same bits either way. */
BCGS_API int bcgs_qr_factor(int64_t m, int32_t n, int32_t s, int variant, int precision,
                   const void* X, int64_t ldx, void* Q, int64_t ldq, double* R,
                   int32_t ldr, void* workspace, size_t ws_bytes, void* stream);

/* The same factorization end to end from host memory.  X_host (m x n,
 * leading dimension ldxh) is copied to the device buffer Xd (ldx) one block
 * column at a time on a copy stream, so that block j + 1 travels while block
 * j is factored on `stream`; every block column of Q is copied from Qd (ldq)
 * to Q_host (ldqh) on a second copy stream as soon as it is final (delayed
 * normalization, Sec. 2: block j - 1 after step j under BCGSI+P-1S and -2S,
 * block j under BCGSI+ and BCGS-PIPI+), and R (n x n) goes from Rd (ldr) to
 * R_host (ldrh) at the end.  Xd, Qd, Rd and the workspace (as for
 * bcgs_qr_factor) are caller-owned device memory; X_host, Q_host and R_host
 * are host memory, page-locked for the copies to overlap (pageable memory
 * works, without overlap).  Everything is ordered on `stream`: the results
 * are on the host once `stream` has completed, and the status is read with
 * bcgs_qr_factor_status.  Safe to call from several host threads (the copy
 * streams are shared per device; calls enqueue one after the other).  Returns BCGS_ERR_INVALID_ARG for a null pointer or
 * a leading dimension below m (n for R). */
BCGS_API int bcgs_qr_factor_host(int64_t m, int32_t n, int32_t s, int variant, int precision,
                   const void* X_host, int64_t ldxh, void* Q_host, int64_t ldqh, double* R_host,
                   int32_t ldrh, void* Xd, int64_t ldx, void* Qd, int64_t ldq, double* Rd,
                   int32_t ldr, void* workspace, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Row-partitioned form (Sec. 3: each of P processes holds a block of rows of
 * X, Q and U and a replicated copy of every small matrix; the only global
 * operations are the sums of the tall-skinny products, one MPI_Allreduce per
 * synchronization on the paper's cluster, and the R-factor reduction of TSQR).
 *
 * Here each rank runs the same block steps on its own rows.  At every
 * synchronization the library calls `allgather` once: every rank contributes
 * `bytes` from the device buffer `send` and must receive all ranks'
 * contributions, rank after rank, in the device buffer `recv` (P * bytes);
 * both buffers lie inside the rank's workspace.  The library then adds the P
 * copies in rank order with its own kernel, so the sum, and the replicated
 * small tail after it, has the same bits on every rank and on every run.  TSQR
 * (the first block, and every block of BCGSI+ and BCGSI+P-2S) factors the
 * local rows, gathers the P local R factors the same way, factors their stack
 * (the same bits on every rank) and forms this rank's rows of Q from its
 * block of the stacked factor's Q.
 *
 * The callback runs on the calling host thread, between launches on `stream`:
 * it must order the exchange on `stream` (after the work enqueued before the
 * call, before the work enqueued after it) and return 0, or nonzero to stop the
 * factorization with BCGS_ERR_COMM (the other ranks then wait in their own
 * callbacks: a collective with a timeout, such as a process group's, ends them).
 * With NCCL it is one all-gather on `stream`.  No device code waits on another
 * rank: every exchange happens through the callback.
 *
 * A rank whose factorization has failed (a non-finite local value, ...) sends
 * NaN, so every rank reports a failure, at a block index within one of the
 * failing rank's (the block whose small factors the NaN reaches first).
 * ------------------------------------------------------------------------- */
typedef int (*bcgs_allgather_fn)(void* ctx, const void* send, void* recv, size_t bytes, void* stream);

/* The rows [*row0, *row0 + *rows) of an m-row matrix that rank `rank` of
 * `nranks` owns: whole 128-row blocks, as even as possible (the first
 * ceil(m / 128) mod nranks ranks get one block more; the last block may be
 * ragged; a rank may get none when m is small).  Host only. */
BCGS_API int bcgs_row_partition(int64_t m, int32_t nranks, int32_t rank, int64_t* row0, int64_t* rows);

/* Workspace of bcgs_qr_factor_rows for a rank with m_local rows.  With
 * nranks = 1 the same as bcgs_qr_workspace_size; with nranks > 1 the slab
 * needs m_local >= s rows (not n), and the workspace adds the gathered copies
 * (nranks * n * 2s doubles), the stacked R factors and a local TSQR block. */
BCGS_API int bcgs_qr_workspace_size_rows(int64_t m_local, int32_t n, int32_t s, int variant, int precision,
                                         int32_t nranks, size_t* bytes);

/* This rank's part of the factorization of the m x n matrix whose rows
 * [row0, row0 + m_local) are X (m_local x n, ldx): Q gets the same rows of the
 * global Q (m_local x n, ldq) and R (n x n, ldr) the whole R, the same bits on
 * every rank.  All ranks call it with the same n, s, variant and precision.
 * The arguments are as for bcgs_qr_factor, plus rank, nranks (1..4096) and the
 * callback (may be NULL only for nranks = 1, which is bcgs_qr_factor).  Returns
 * after the whole factorization is enqueued; read the outcome with
 * bcgs_qr_factor_status; BCGS_ERR_COMM when a callback returned nonzero. */
BCGS_API int bcgs_qr_factor_rows(int64_t m_local, int32_t n, int32_t s, int variant, int precision,
                                 const void* X, int64_t ldx, void* Q, int64_t ldq, double* R, int32_t ldr,
                                 void* workspace, size_t ws_bytes, void* stream, int32_t rank, int32_t nranks,
                                 bcgs_allgather_fn allgather, void* ctx);

/* Self-test of the timeout path, with no fault involved: one bounded device
 * wait on a barrier that nothing completes gives up after `cycles` SM clock
 * cycles (1 .. 2e9, about one second at most) and records BCGS_ERR_TIMEOUT in
 * the status word at the start of `workspace` (device memory, at least 256
 * bytes, 256-byte aligned), as the library's kernels do when one of their
 * bounded waits runs out.  The status is reset first; read it with
 * bcgs_qr_factor_status.  The context stays usable.
 * Returns BCGS_ERR_INVALID_ARG for a null or short workspace or cycles out of
 * range, BCGS_ERR_WORKSPACE for a misaligned one. */
BCGS_API int bcgs_wait_selftest(void* workspace, size_t ws_bytes, int64_t cycles, void* stream);

/* Synchronize `stream`, then return the device status word of the last
 * factorization that used `workspace`; *fail_block (may be NULL) gets the
 * 1-based block column at which it failed, 0 on success. */
BCGS_API int bcgs_qr_factor_status(const void* workspace, void* stream, int32_t* fail_block);

/* ---------------------------------------------------------------------------
 * Block-by-block interface (s-step Krylov use, serving).
 *
 * bcgs_qr_init binds a handle to caller-owned Q, R and workspace; each
 * bcgs_qr_step ingests the next m x s block X_j; bcgs_qr_finish runs the last
 * block's branch of Alg. 2.  Delayed normalization (Sec. 2, eq. (1)) means that
 * under BCGSI+P-1S and -2S, after step j (j >= 2) the columns of Q and R of
 * blocks 1..j-1 are final and block j is still provisional; under BCGSI+ and
 * BCGS-PIPI+ block j is final after step j (bcgs_qr_finish enqueues nothing).
 * bcgs_qr_sync reports how many columns are final.
 * The handle is a small host object (the only host allocation of the library).
 * ------------------------------------------------------------------------- */
BCGS_API int bcgs_qr_init(bcgs_qr_t* handle, int64_t m, int32_t n_max, int32_t s,
                 int variant, int precision, void* Q, int64_t ldq, double* R,
                 int32_t ldr, void* workspace, size_t ws_bytes, void* stream);

/* Ingest the next block X_j (m x s, leading dimension ldx; the last block is
 * m x (n_max mod s) when s does not divide n_max, and after it every column is
 * final).  Returns BCGS_ERR_STATE after bcgs_qr_finish or once n_max columns
 * were ingested. */
BCGS_API int bcgs_qr_step(bcgs_qr_t handle, const void* X_block, int64_t ldx);

/* Finalize the last block (the else-branch of Alg. 2).  Idempotent. */
BCGS_API int bcgs_qr_finish(bcgs_qr_t handle);

/* Synchronize the handle's stream and return its device status; *n_final gets
 * the number of final columns of Q and R, *fail_block the failing block (0 if
 * none).  Either pointer may be NULL. */
BCGS_API int bcgs_qr_sync(bcgs_qr_t handle, int32_t* n_final, int32_t* fail_block);

/* Rebind the handle to another stream (ordering is the caller's business). */
BCGS_API int bcgs_qr_set_stream(bcgs_qr_t handle, void* stream);

/* Release the host handle (device buffers stay the caller's). */
BCGS_API int bcgs_qr_destroy(bcgs_qr_t handle);

/* ---------------------------------------------------------------------------
 * Batched interface: many independent factorizations, one launch per phase.
 * ------------------------------------------------------------------------- */
typedef struct {
  int64_t m;         /* rows                                 */
  int32_t n, s;      /* columns and block size (ragged last block when s does not divide n) */
  int32_t variant;   /* bcgs_variant                         */
  int32_t precision; /* bcgs_precision                        */
  const void* X; int64_t ldx;
  void* Q; int64_t ldq;
  double* R; int32_t ldr;
  int32_t engine;    /* product engine of this problem: 0 = the BCGS_OPT_GRAM_ENGINE option;
                        otherwise 1 + an option value (1 FP64 pipe, 2 tensor cores from
                        BCGS_OPT_TC_MIN_ROWS rows, 3 tensor cores always); other values
                        are INVALID_ARG.  It decides the workspace (the digit store) too. */
} bcgs_problem;

/* Workspace for a batch (host array `probs` of `count` problems). */
BCGS_API int bcgs_qr_batched_workspace_size(int32_t count, const bcgs_problem* probs, size_t* bytes);

/* Enqueue all `count` factorizations, ordered after the work already on
 * `stream` and before anything enqueued on it later; statuses go to the
 * workspace, read them with bcgs_qr_batched_status.  Problems run concurrently
 * on 16 internal streams (created on the first call on a device and kept until
 * exit) that fork from and join back into `stream`, so capturing `stream` into
 * a CUDA graph captures the whole batch as one graph.  Each problem's result is
 * the same as bcgs_qr_factor's for it alone (fixed reduction order).  Safe to
 * call from several host threads (the internal streams are shared per device;
 * calls enqueue one after the other). */
BCGS_API int bcgs_qr_factor_batched(int32_t count, const bcgs_problem* probs, void* workspace,
                           size_t ws_bytes, void* stream);

/* Synchronize and copy the `count` status codes and failing blocks to host
 * arrays (either may be NULL); returns the first nonzero status or BCGS_OK. */
BCGS_API int bcgs_qr_batched_status(int32_t count, const void* workspace, void* stream,
                           int32_t* codes, int32_t* fail_blocks);

/* ---------------------------------------------------------------------------
 * Building blocks, exposed for reuse and testing (FP64 only).
 * ------------------------------------------------------------------------- */

/* C (ka x kb, ldc, device FP64) = A^T B for A (m x ka, lda) and B (m x kb,
 * ldb): one synchronization point (Sec. 3).  ka*kb <= 65536. */
BCGS_API int bcgs_gram_workspace_size(int64_t m, int32_t ka, int32_t kb, size_t* bytes);
BCGS_API int bcgs_gram(int64_t m, int32_t ka, int32_t kb, const double* A, int64_t lda,
              const double* B, int64_t ldb, double* C, int32_t ldc,
              void* workspace, size_t ws_bytes, void* stream);

/* Allocation-free C = A^T B.  The paper has no counterpart: this entry point
 * exists for callers that can neither call cudaMalloc nor lend the library a
 * workspace, such as a host framework that owns all device memory through its
 * own pool (allocating behind its back fragments the pool, and cudaMalloc /
 * cudaFree may synchronize the device) or a latency-bound loop that must never
 * reach the allocator.  It computes the same result as bcgs_gram, with the
 * same deterministic reduction order, but keeps the chunk partial sums in a
 * fixed array compiled into the library: BCGS_GRAM_NOALLOC_MAX_PARTIALS doubles
 * (8 MiB) of partials plus 65536 words of column maxima for the tensor-core
 * engine (BCGS_OPT_GRAM_ENGINE picks the engine as for bcgs_gram); every GPU
 * that loads the library holds that array until the process exits.  The
 * caller still passes A, B and C.
 *   Limit: the number of row chunks of m times ka * kb must not exceed
 *   BCGS_GRAM_NOALLOC_MAX_PARTIALS.  The row chunk count is at most
 *   min(304, ceil(m / 64)), so ka * kb <= 3449 always fits; larger requests
 *   return BCGS_ERR_WORKSPACE and enqueue nothing.  ka * kb <= 65536 and the
 *   argument rules of bcgs_gram apply (BCGS_ERR_INVALID_ARG otherwise).
 *   Set-up: the first call on each device looks up the device address of the
 *   array (once per device, with that device current), so make the first call
 *   on a device before any stream capture begins.
 *   Sharing: all calls use the same array.  Calls whose kernels may overlap on
 *   the GPU (different streams, or host threads without ordering) race on it
 *   and give wrong results; order them on one stream.
 *   Errors: there is no status word.  A non-finite entry of A or B (and a
 *   device wait of the tensor engine that runs out) shows as NaN entries of C;
 *   every partial slot is rewritten by each call, so C never holds what an
 *   earlier call left in the array.  The device address is looked up once per
 *   device and kept: do not use the entry point across a cudaDeviceReset.
 *   No cudaMalloc, cudaFree or allocating library routine is called. */
#define BCGS_GRAM_NOALLOC_MAX_PARTIALS 1048576
BCGS_API int bcgs_gram_noalloc(int64_t m, int32_t ka, int32_t kb, const double* A, int64_t lda,
                               const double* B, int64_t ldb, double* C, int32_t ldc, void* stream);

/* W = (V - Q C) T^{-1}: projection plus triangular-solve normalization (Alg. 1
 * and Alg. 2, the U and Q updates).  V, W: m x s; Q: m x c; C: c x s (device);
 * T: s x s upper triangular (device) or NULL for no normalization.  c may be 0
 * (Q and C ignored).  W may alias V.  1 <= s <= 64. */
BCGS_API int bcgs_project(int64_t m, int32_t c, int32_t s, const double* V, int64_t ldv,
                 const double* Q, int64_t ldq, const double* C, int32_t ldc,
                 const double* T, int32_t ldt, double* W, int64_t ldw, void* stream);

/* TSQR (Sec. 1, Alg. 1, Alg. 2): economic QR of an m x s block A (lda) into
 * Q (ldq) and R (s x s, ldr, device), diag(R) >= 0; Householder QR of row
 * tiles, a fixed reduction tree of the stacked R factors, and an explicit-Q
 * pass.  Q may alias A.  A zero diagonal of R sets BCGS_ERR_RANK_DEFICIENT
 * in the workspace status word (read it with bcgs_qr_factor_status). */
BCGS_API int bcgs_tsqr_workspace_size(int64_t m, int32_t s, size_t* bytes);
BCGS_API int bcgs_tsqr(int64_t m, int32_t s, const double* A, int64_t lda, double* Q,
              int64_t ldq, double* R, int32_t ldr, void* workspace, size_t ws_bytes,
              void* stream);

/* Upper Cholesky factor R (s x s) of a symmetric positive definite A (s x s)
 * on the device (chol of Alg. 1 and Alg. 2).  A non-positive pivot sets
 * BCGS_ERR_NOT_SPD in the workspace status word.  workspace >= 256 bytes. */
BCGS_API int bcgs_chol(int32_t s, const double* A, int32_t lda, double* R, int32_t ldr,
              void* workspace, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Options (process-wide, host side).
 *
 * BCGS_OPT_GRAM_ENGINE selects how the inner products of the synchronization
 * (the Gram reduction) and of the projection (Q C in (V - Q C) T^{-1}) are
 * computed:
 *   0  the FP64 pipe (DFMA, chunked fixed-order sums);
 *   1  (default) tensor cores when the call has at least BCGS_OPT_TC_MIN_ROWS
 *      rows (and, for the Gram, at most 64 columns on the right; for the
 *      projection s <= 32): each FP64 (or FP32) operand
 *      is split exactly into eight 8-bit integer digits relative to the
 *      maximum along its contraction line (a column of a Gram operand, a row
 *      of Q), digit pairs are multiplied on the tensor cores
 *      with exact integer sums, and one FP64 rounding per row chunk remains
 *      (error per product term <= 2^-57.1 max|a_i| max|b_j|).  A factorization
 *      with s <= 32 (either storage type) keeps Q as such digits (the seven
 *      leading balanced digits in [-128, 127], one exponent per 128 rows and
 *      column, error per term about 2^-53.9 max|a| max|b| over the 128-row
 *      block, below the FP64 unit roundoff) and computes its Grams (s a
 *      multiple of 8) and projections from them;
 *   2  tensor cores whenever the shape allows it.
 * A factorization reads the engine when it is initialized (bcgs_qr_init,
 * bcgs_qr_factor): that fixes whether it keeps the digit store.
 * BCGS_OPT_TC_MIN_ROWS is the row threshold of engine 1 (default 16384).
 * Both engines use the same row partition, so each is deterministic; they
 * differ by rounding.
 * BCGS_OPT_DEBUG_SYNC (diagnostics, default 0): 1 makes the factorization
 * calls synchronize their stream after every launch and name a failing launch
 * on stderr.
 * Returns BCGS_ERR_INVALID_ARG for an unknown option or value.
 * ------------------------------------------------------------------------- */
#define BCGS_OPT_GRAM_ENGINE 1
#define BCGS_OPT_TC_MIN_ROWS 2
#define BCGS_OPT_DEBUG_SYNC 3
BCGS_API int bcgs_set_option(int option, int64_t value);
BCGS_API int64_t bcgs_get_option(int option);

/* ---------------------------------------------------------------------------
 * Instrumentation (host side; no device memory).
 * ------------------------------------------------------------------------- */

/* Number of CUDA kernels this library has launched since it was loaded. */
BCGS_API int64_t bcgs_launch_count(void);

/* enable != 0: bracket every Gram-partial, Gram-reduce, projection, TSQR,
 * tail and digit-store split launch with CUDA events recorded on its stream
 * (cudaEventCreate is the only resource used).  Adds a few microseconds per
 * launch. */
BCGS_API int bcgs_profile_enable(int enable);

/* Drop recorded events and totals. */
BCGS_API int bcgs_profile_reset(void);

/* Totals for a kernel class (0 Gram partial, 1 Gram reduce, 2 projection,
 * 3 TSQR, 4 tail, 5 digit-store split of Q) over the recorded launches: count,
 * summed event time in ms, algorithmic flops and bytes.  Waits for the recorded
 * events. */
BCGS_API int bcgs_profile_read(int kernel_class, int64_t* launches, double* total_ms,
                               double* flops, double* bytes);

#ifdef __cplusplus
}
#endif
#endif /* BCGS_QR_H */
