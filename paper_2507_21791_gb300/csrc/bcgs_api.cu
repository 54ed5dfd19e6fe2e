// Host driver and C ABI: the four variants as block-step state machines over
// the kernels of gram.cu, proj.cu, tsqr.cu and tail.cu.
//
// Every step is a fixed sequence of stream-ordered launches; nothing here
// synchronizes except bcgs_qr_sync / *_status.  All device memory is the
// caller's: the workspace is carved into the buffers below.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>

#include <nvtx3/nvToolsExt.h>  // header-only; a no-op unless a profiler is attached

#include "bcgs_internal.cuh"

using namespace bcgs;

namespace {

constexpr int kMaxS = 64;
constexpr int kMaxN = 2048;

struct Layout {
  size_t status, status_side, S[2], Sd[2], Yd, Rt1, Rt2, G, G2, Bp, partial, amax, amaxQ, amaxU, rowmaxQ, U, V, tsqr,
      qstore, fexp, total;
  // row-partitioned form (nranks > 1): gathered copies, the stacked R factors,
  // the stacked factor's Q, the local TSQR factor and R, and the stacked TSQR's work
  size_t comm_recv, stack, stackq, Tq, Rloc, tsqr_stack;
  int nranks;
  TsqrPlan tp_stack, tp_stack_last;
  int store;    // the digit store of Q is part of the workspace
  int ldg;      // leading dimension of G, G2 (= n_max)
  int64_t ldu;  // leading dimension of U, V
  TsqrPlan tp;
  TsqrPlan tp_last;  // TSQR of the ragged last block (n_max mod s columns), if any
};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

bool valid_shape(int64_t m, int32_t n, int32_t s) {
  return s >= 1 && s <= kMaxS && n >= 1 && m >= n && n <= kMaxN;
}

// The digit store of Q pays for itself where the projections run on the tensor
// cores: s <= 32 and the row count the engine option selects (FP32 storage
// converts to FP64 exactly, so both storage types share it).
bool want_store(int64_t m, int32_t s, int precision) {
  const int e = gram_engine();
  (void)precision;
  return s <= 32 && e != 0 && (e == 2 || m >= gram_tc_min_rows());
}

void make_layout(int64_t m, int32_t n_max, int32_t s, int variant, int precision, int store,
                 Layout* L, int nranks = 1) {
  const size_t esz = precision == BCGS_FP32_STORAGE ? 4 : 8;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  L->status = take(sizeof(DevStatus));
  // failures of work run ahead on the side stream, merged in stream order
  L->status_side = take(sizeof(DevStatus));
  const size_t ss = (size_t)s * s * sizeof(double);
  for (int i = 0; i < 2; ++i) L->S[i] = take((size_t)n_max * s * sizeof(double));
  for (int i = 0; i < 2; ++i) L->Sd[i] = take(ss);
  L->Yd = take(ss);
  L->Rt1 = take(ss);
  L->Rt2 = take(ss);
  L->ldg = n_max;
  L->G = take((size_t)n_max * 2 * s * sizeof(double));
  L->G2 = take((size_t)n_max * 2 * s * sizeof(double));
  // (c + s) x 2s coefficients of the paired projection (BCGSI+P-1S / -2S, BCGSI+1s)
  const bool paired = variant == BCGS_BCGSI_PLUS_P_1S || variant == BCGS_BCGSI_PLUS_P_2S ||
                      variant == BCGS_BCGSI_PLUS_1S;
  L->Bp = paired ? take((size_t)n_max * 2 * s * sizeof(double)) : off;
  L->partial = take(gram_partial_doubles(m, n_max, 2 * s) * sizeof(double));
  L->amax = take(((size_t)n_max + 4 * (size_t)s) * sizeof(unsigned long long));
  // maxima kept by the writers: per column of Q, per column of U, per row of Q
  L->amaxQ = take((size_t)n_max * sizeof(unsigned long long));
  L->amaxU = take((size_t)s * sizeof(unsigned long long));
  L->rowmaxQ = take((size_t)m * sizeof(unsigned long long));
  L->ldu = round_up(m, 64);
  L->U = take((size_t)L->ldu * s * esz);
  // the projected block TSQR reads (no TSQR after block 1 under 1S, PIPI+ and 1s)
  const bool tsqr_in = variant == BCGS_BCGSI_PLUS || variant == BCGS_BCGSI_PLUS_P_2S;
  L->V = tsqr_in ? take((size_t)L->ldu * s * esz) : off;
  tsqr_plan(m, s, &L->tp);
  const int32_t s_last = n_max % s;
  tsqr_plan(m, s_last > 0 ? s_last : s, &L->tp_last);
  L->tsqr = take((L->tp.doubles > L->tp_last.doubles ? L->tp.doubles : L->tp_last.doubles) * sizeof(double));
  L->store = store;
  L->qstore = store ? take(qstore_bytes(m, n_max)) : off;
  L->fexp = store ? take((size_t)ceil_div(m, kStoreRows) * 32 * sizeof(int32_t)) : off;
  L->nranks = nranks;
  if (nranks > 1) {
    const size_t per = (size_t)n_max * 2 * s > (size_t)s * s ? (size_t)n_max * 2 * s : (size_t)s * s;
    L->comm_recv = take((size_t)nranks * per * sizeof(double));
    L->stack = take((size_t)nranks * s * s * sizeof(double));
    L->stackq = take((size_t)nranks * s * s * sizeof(double));
    L->Tq = take((size_t)L->ldu * s * esz);
    L->Rloc = take(ss);
    tsqr_plan((int64_t)nranks * s, s, &L->tp_stack);
    tsqr_plan((int64_t)nranks * (s_last > 0 ? s_last : s), s_last > 0 ? s_last : s, &L->tp_stack_last);
    const size_t d1 = L->tp_stack.doubles, d2 = L->tp_stack_last.doubles;
    L->tsqr_stack = take((d1 > d2 ? d1 : d2) * sizeof(double));
  } else {
    L->comm_recv = L->stack = L->stackq = L->Tq = L->Rloc = L->tsqr_stack = off;
  }
  L->total = off;
}

// True when the byte ranges of two column-major m x n arrays (leading
// dimensions lda, ldb; element size esz) overlap.  Host-only pointer
// arithmetic: nothing is read.
bool overlaps(const void* a, int64_t lda, const void* b, int64_t ldb, int64_t m, int32_t n, size_t esz) {
  if (a == nullptr || b == nullptr || m < 1 || n < 1) return false;
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(a), b0 = reinterpret_cast<uintptr_t>(b);
  const uintptr_t a1 = a0 + ((uintptr_t)(n - 1) * (uintptr_t)lda + (uintptr_t)m) * esz;
  const uintptr_t b1 = b0 + ((uintptr_t)(n - 1) * (uintptr_t)ldb + (uintptr_t)m) * esz;
  return a0 < b1 && b0 < a1;
}

Seg seg(const void* p, int64_t ld, int ncols, int fp32, const unsigned long long* amax = nullptr) {
  Seg g;
  g.p = p;
  g.ld = ld;
  g.ncols = ncols;
  g.fp32 = fp32;
  g.amax = amax;
  return g;
}

}  // namespace

namespace bcgs {
namespace {
std::atomic<int> g_engine{1};
std::atomic<long long> g_tc_min_rows{16384};
// Engine of the factorization being enqueued on this thread when a batched
// problem names its own (-1: the BCGS_OPT_GRAM_ENGINE option).
thread_local int t_engine = -1;
}  // namespace
int gram_engine() {
  const int t = t_engine;
  return t >= 0 ? t : g_engine.load();
}
// Sets the engine of this thread's enqueues for a scope (bcgs_problem::engine:
// 0 = the option, 1 + the option's value otherwise).
struct EngineScope {
  int prev;
  explicit EngineScope(int problem_engine) : prev(t_engine) { t_engine = problem_engine > 0 ? problem_engine - 1 : -1; }
  ~EngineScope() { t_engine = prev; }
};
int64_t gram_tc_min_rows() { return g_tc_min_rows.load(); }
bool use_tensor_gram(const GramDesc& d) {
  const int e = gram_engine();
  if (e == 0 || !gram_tc_supported(d)) return false;
  return e == 2 || d.m >= gram_tc_min_rows();
}
bool use_tensor_project(const ProjDesc& d) {
  const int e = gram_engine();
  if (e == 0 || !project_tc_supported(d)) return false;
  return e == 2 || d.m >= gram_tc_min_rows();
}
}  // namespace bcgs

struct bcgs_qr_s {
  int64_t m;
  int32_t n_max, s, variant, precision;
  char* Q;
  int64_t ldq;
  double* R;
  int32_t ldr;
  char* ws;
  size_t ws_bytes;
  cudaStream_t stream;
  Layout L;
  int32_t j;  // blocks ingested
  int32_t cur;
  int32_t finished;
  int32_t esz;
  int32_t fp32;
  int32_t sgram;  // Grams read the digit store (the current U and X blocks are split into it)
  int32_t flushed;  // a ragged last block was stepped: every block is final, finish does nothing
  cudaError_t last_cuda;
  // row-partitioned form: this process's rank among nranks and the all-gather
  // it calls once per synchronization (nranks = 1: no collective)
  int32_t rank, nranks;
  bcgs_allgather_fn allgather;
  void* ag_ctx;
  int32_t comm_failed;
  // one-call factorization: the next block of X (null when unknown or not to
  // be split ahead), and whether the current block's digits are already in the
  // store (split ahead on the side stream during the previous step's tail)
  const void* next_X;
  int64_t next_ldx;
  int32_t x_put;

  DevStatus* st() { return reinterpret_cast<DevStatus*>(ws + L.status); }
  DevStatus* st_side() { return reinterpret_cast<DevStatus*>(ws + L.status_side); }
  double* buf(size_t off) { return reinterpret_cast<double*>(ws + off); }
  void* U() { return ws + L.U; }
  void* V() { return ws + L.V; }
  // column block k (1-based) of Q
  char* Qblk(int k) { return Q + (size_t)(k - 1) * s * ldq * esz; }
  unsigned long long* amaxQ() { return reinterpret_cast<unsigned long long*>(ws + L.amaxQ); }
  unsigned long long* amaxU() { return reinterpret_cast<unsigned long long*>(ws + L.amaxU); }
  unsigned long long* rowmaxQ() { return reinterpret_cast<unsigned long long*>(ws + L.rowmaxQ); }
  // Q and U carry the column maxima their writers kept
  Seg Qseg(int ncols) { return seg(Q, ldq, ncols, fp32, amaxQ()); }
  Seg Useg(int w = 0) { return seg(U(), L.ldu, w ? w : s, fp32, amaxU()); }
  Seg Vseg(int w = 0) { return seg(V(), L.ldu, w ? w : s, fp32); }
  // columns [col0, ...) of Q, and the maxima to keep when writing them
  char* Qcol(int col0) { return Q + (size_t)col0 * ldq * esz; }
  MaxOut Qmax_at(int col0) {
    return MaxOut{sgram ? nullptr : amaxQ() + col0, L.store ? nullptr : rowmaxQ()};
  }
  bool delayed() const {
    return variant == BCGS_BCGSI_PLUS_P_1S || variant == BCGS_BCGSI_PLUS_P_2S || variant == BCGS_BCGSI_PLUS_1S;
  }
  // width of block column j (1-based): s, or the ragged rest of n_max
  int width(int j) const { return (int)((int64_t)j * s <= n_max ? s : n_max - (int64_t)(j - 1) * s); }
  // maxima to keep when writing block k of Q, or U: the column maxima feed the
  // on-the-fly Gram (not needed when the Grams read the store), the row maxima
  // of Q the on-the-fly projection (not needed with the store)
  MaxOut Qmax(int k) {
    return MaxOut{sgram ? nullptr : amaxQ() + (size_t)(k - 1) * s, L.store ? nullptr : rowmaxQ()};
  }
  MaxOut Umax() { return MaxOut{sgram ? nullptr : amaxU(), nullptr}; }
  int32_t* fexp() { return reinterpret_cast<int32_t*>(ws + L.fexp); }
  QStore qs() { return qstore_at(ws + L.qstore, m, n_max); }
};

namespace {

// bcgs_set_option(BCGS_OPT_DEBUG_SYNC, 1): synchronize after every launch and
// name the launch that failed on stderr (diagnostics only; off by default).
std::atomic<int> g_debug_sync{0};
bool debug_sync() { return g_debug_sync.load() != 0; }

int check(bcgs_qr_s* h, cudaError_t e, const char* what, int line) {
  if (e == cudaSuccess && debug_sync()) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    h->last_cuda = e;
    if (debug_sync()) fprintf(stderr, "bcgs: %s (bcgs_api.cu:%d): %s\n", what, line, cudaGetErrorString(e));
    return BCGS_ERR_CUDA;
  }
  return BCGS_OK;
}

#define TRY(expr)                                    \
  do {                                               \
    int rc_ = check(h, (expr), #expr, __LINE__);     \
    if (rc_ != BCGS_OK) return rc_;                  \
  } while (0)

cudaError_t gram(bcgs_qr_s* h, std::initializer_list<Seg> A, std::initializer_list<Seg> B,
                 double* G) {
  GramDesc d;
  memset(&d, 0, sizeof(d));
  d.nsa = 0;
  d.na = 0;
  for (const Seg& a : A) {
    if (a.ncols <= 0) continue;
    d.a[d.nsa++] = a;
    d.na += a.ncols;
  }
  d.nsb = 0;
  d.nb = 0;
  for (const Seg& b : B) {
    if (b.ncols <= 0) continue;
    d.b[d.nsb++] = b;
    d.nb += b.ncols;
  }
  d.m = h->m;
  d.block = h->j + 1;
  gram_partition(h->m, &d.chunk_rows, &d.nchunks);
  if (use_tensor_gram(d))
    return launch_gram_tc(d, h->buf(h->L.partial), G, h->L.ldg,
                          reinterpret_cast<unsigned long long*>(h->ws + h->L.amax), h->st(), h->stream);
  return launch_gram(d, h->buf(h->L.partial), G, h->L.ldg, h->st(), h->stream);
}

cudaError_t project(bcgs_qr_s* h, Seg v, int c, const double* C, int ldc, const double* T,
                    void* w, int64_t ldw, MaxOut wmax = MaxOut{nullptr, nullptr}, int sb = 0) {
  if (sb == 0) sb = h->s;
  ProjDesc d;
  memset(&d, 0, sizeof(d));
  d.q_rowmax = h->rowmaxQ();
  d.wmax = wmax;
  d.v = v;
  d.q = h->Qseg(c);
  d.C = C;
  d.ldc = ldc;
  d.T = T;
  d.ldt = sb;
  d.w = w;
  d.ldw = ldw;
  d.w_fp32 = h->fp32;
  d.m = h->m;
  d.s = sb;
  if (h->L.store && use_tensor_project(d) && project_store_supported(sb, 1)) {
    StoreProjDesc p;
    memset(&p, 0, sizeof(p));
    p.qs = h->qs();
    p.c = c;
    p.B = C;
    p.ldb = ldc;
    p.s = sb;
    p.nouts = 1;
    p.out[0] = ProjOut{reinterpret_cast<const double*>(v.p), v.ld, T, sb, reinterpret_cast<double*>(w),
                       ldw, wmax};
    p.m = h->m;
    p.block = h->j + 1;
    p.fexp = h->fexp();
    p.fp32 = h->fp32;
    return launch_project_store(p, h->st(), h->stream);
  }
  if (use_tensor_project(d)) return launch_project_tc(d, h->st(), h->stream);
  return launch_project(d, h->st(), h->stream);
}

// Digits of the freshly written columns [col0, col0 + sb) of Q into the store.
cudaError_t wrote_q_cols(bcgs_qr_s* h, int col0, int sb, int block) {
  if (!h->L.store) return cudaSuccess;
  return launch_qsplit(h->qs(), h->Qcol(col0), h->ldq, h->Q, h->ldq, h->m, col0, sb, h->fp32, h->st(), block,
                       h->stream);
}
// ... of the freshly written (full) block column k of Q.
cudaError_t wrote_q(bcgs_qr_s* h, int k) { return wrote_q_cols(h, (k - 1) * h->s, h->s, k); }

// With store Grams: digits of an m x s block (X or U) into store columns
// [k0, k0 + s), the columns Q fills next.
cudaError_t store_put(bcgs_qr_s* h, const void* src, int64_t ld, int k0, int sb = 0) {
  if (!h->sgram) return cudaSuccess;
  return launch_qsplit(h->qs(), src, ld, h->Q, h->ldq, h->m, k0, sb ? sb : h->s, h->fp32, h->st(), h->j + 1,
                       h->stream);
}

// A side stream of the calling host thread (one per device) with the two events
// that fork it from a factorization's stream and join it back.  Created on first
// use, never while the factorization's stream is being captured into a graph.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
struct SidePool {
  static constexpr int kDevices = 64;
  SideStream dev[kDevices];
  ~SidePool() {
    for (SideStream& d : dev) {
      if (d.join != nullptr) cudaEventDestroy(d.join);
      if (d.fork != nullptr) cudaEventDestroy(d.fork);
      if (d.s != nullptr) cudaStreamDestroy(d.s);
    }
  }
};
SideStream* side_stream(cudaStream_t main) {
  thread_local SidePool pool;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= SidePool::kDevices) return nullptr;
  SideStream& d = pool.dev[dev];
  if (d.join != nullptr) return &d;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(main, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
  if (d.s == nullptr && cudaStreamCreateWithFlags(&d.s, cudaStreamNonBlocking) != cudaSuccess) d.s = nullptr;
  if (d.s != nullptr && d.fork == nullptr && cudaEventCreateWithFlags(&d.fork, cudaEventDisableTiming) != cudaSuccess)
    d.fork = nullptr;
  if (d.fork != nullptr && cudaEventCreateWithFlags(&d.join, cudaEventDisableTiming) != cudaSuccess) d.join = nullptr;
  return d.join != nullptr ? &d : nullptr;
}

// Rows from which the next block's digit split runs ahead, during the tail
// (a single-CTA kernel that leaves the GPU's bandwidth idle).
constexpr int64_t kAheadMinRows = 1 << 17;

// G = A^T B: from the store (A = store columns [0, na), B = [b0, b0 + nb)) when
// the factorization keeps its Grams there, else from the segments.
// Row-partitioned form: G holds this rank's Gram of its rows; every rank sends
// its copy (NaN if its factorization has failed), receives all copies and adds
// them in rank order, so G becomes the Gram of the whole matrix, the same bits
// on every rank.
cudaError_t sum_over_ranks(bcgs_qr_s* h, double* G, int na, int nb) {
  const size_t elems = (size_t)h->L.ldg * nb;
  cudaError_t e = launch_poison_if_failed(G, (int64_t)elems, h->st(), h->stream);
  if (e != cudaSuccess) return e;
  double* recv = h->buf(h->L.comm_recv);
  if (h->allgather(h->ag_ctx, G, recv, elems * sizeof(double), h->stream) != 0) {
    h->comm_failed = 1;
    return cudaErrorUnknown;
  }
  return launch_rank_sum(recv, h->nranks, na, nb, h->L.ldg, G, h->st(), h->stream);
}

cudaError_t gram_local(bcgs_qr_s* h, int na, int b0, int nb, std::initializer_list<Seg> A,
                       std::initializer_list<Seg> B, double* G);

cudaError_t gram_cols(bcgs_qr_s* h, int na, int b0, int nb, std::initializer_list<Seg> A,
                      std::initializer_list<Seg> B, double* G) {
  const cudaError_t e = gram_local(h, na, b0, nb, A, B, G);
  if (e != cudaSuccess || h->nranks <= 1) return e;
  return sum_over_ranks(h, G, na, nb);
}

// The Gram of this process's rows only.
cudaError_t gram_local(bcgs_qr_s* h, int na, int b0, int nb, std::initializer_list<Seg> A,
                       std::initializer_list<Seg> B, double* G) {
  if (!h->sgram) return gram(h, A, B, G);
  // the store Gram takes at most 32 B columns per launch: wider B (the 2s
  // columns [U X] of 1S / 2S at s = 32) in groups of 32, each into its columns of G
  for (int j0 = 0; j0 < nb; j0 += 32) {
    GramStoreDesc d;
    memset(&d, 0, sizeof(d));
    d.qs = h->qs();
    d.na = na;
    d.b0 = b0 + j0;
    d.nb = nb - j0 < 32 ? nb - j0 : 32;
    gram_store_partition(h->m, &d.nchunks, &d.bpc);
    d.m = h->m;
    d.block = h->j + 1;
    const cudaError_t e = launch_gram_store(d, h->buf(h->L.partial), G + (size_t)j0 * h->L.ldg, h->L.ldg, h->st(),
                                            h->stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t tsqr(bcgs_qr_s* h, Seg a, void* q, int64_t ldq, double* R, int ldr, int block,
                 MaxOut qmax = MaxOut{nullptr, nullptr}) {
  // the plan of the block's width (a.ncols is s or the ragged rest)
  const TsqrPlan& tp = a.ncols == h->s ? h->L.tp : h->L.tp_last;
  if (h->nranks <= 1)
    return launch_tsqr(tp, a, q, ldq, h->fp32, R, ldr, h->buf(h->L.tsqr), h->st(), block, h->stream, qmax);
  // Row-partitioned TSQR: the local rows' TSQR gives Tq and R_loc; the ranks'
  // R_loc are gathered, stacked and factored again (the same bits on every
  // rank), [R_0; ...; R_{P-1}] = Qs R; this rank's rows of Q are Tq times its
  // s x s block of Qs.  The local factor carries no status word: a rank's rows
  // may be rank deficient while the whole block is not (and a NaN reaches the
  // stacked factor, which reports it).
  const int w = a.ncols, P = h->nranks;
  const TsqrPlan& tps = w == h->s ? h->L.tp_stack : h->L.tp_stack_last;
  double* Rloc = h->buf(h->L.Rloc);
  void* Tq = h->ws + h->L.Tq;
  cudaError_t e = launch_tsqr(tp, a, Tq, h->L.ldu, h->fp32, Rloc, w, h->buf(h->L.tsqr), nullptr, block, h->stream,
                              MaxOut{nullptr, nullptr});
  if (e != cudaSuccess) return e;
  e = launch_poison_if_failed(Rloc, (int64_t)w * w, h->st(), h->stream);
  if (e != cudaSuccess) return e;
  double* recv = h->buf(h->L.comm_recv);
  if (h->allgather(h->ag_ctx, Rloc, recv, (size_t)w * w * sizeof(double), h->stream) != 0) {
    h->comm_failed = 1;
    return cudaErrorUnknown;
  }
  double* stack = h->buf(h->L.stack);
  double* stackq = h->buf(h->L.stackq);
  e = launch_stack_r(recv, P, w, stack, h->st(), h->stream);
  if (e != cudaSuccess) return e;
  e = launch_tsqr(tps, seg(stack, (int64_t)P * w, w, 0), stackq, (int64_t)P * w, 0, R, ldr,
                  h->buf(h->L.tsqr_stack), h->st(), block, h->stream, MaxOut{nullptr, nullptr});
  if (e != cudaSuccess) return e;
  return launch_rows_times_small(h->m, w, Tq, h->L.ldu, stackq + (size_t)h->rank * w, P * w, q, ldq, h->fp32, qmax,
                                 h->st(), h->stream);
}
cudaError_t zero_umax(bcgs_qr_s* h, int sb = 0) { return launch_zero_u64(h->amaxU(), sb ? sb : h->s, h->stream); }

// Last-block branch of Alg. 2 (shared by BCGSI+P-1S and -2S):
// [Y_{1:q-1,q}; Omega_q] = [Q_{q-1} U_q]^T U_q, Y_qq, R column block q, Q_q.
int finish_p(bcgs_qr_s* h) {
  const int s = h->s, q = h->j;
  const int c = (q - 1) * s;
  double* G = h->buf(h->L.G);
  const int ldg = h->L.ldg;
  TRY(gram_cols(h, c + s, c, s, {h->Qseg(c), h->Useg()}, {h->Useg()}, G));
  TailDesc t;
  memset(&t, 0, sizeof(t));
  t.s = s;
  t.c = c;
  t.G = G;
  t.ldg = ldg;
  t.gy = 0;
  t.gom = c;
  t.S_prev = h->buf(h->L.S[h->cur]);
  t.Sd_prev = h->buf(h->L.Sd[h->cur]);
  t.Yd = h->buf(h->L.Yd);
  t.R = h->R;
  t.ldr = h->ldr;
  t.r_row0 = 0;
  t.r_col0 = c;
  t.has_next = 0;
  t.block = q;
  t.ldsm = h->n_max;
  ProjDesc probe;
  memset(&probe, 0, sizeof(probe));
  probe.q = h->Qseg(c);
  probe.m = h->m;
  probe.s = s;
  // U_q is in the store (columns [c, c + s)) when the Grams use it
  const bool folded = h->sgram && use_tensor_project(probe) && project_store_supported(s, 1);
  if (folded) {
    t.Bpair = h->buf(h->L.Bp);
    t.ldb = h->n_max;
  }
  TRY(launch_tail_1s2s(t, h->st(), h->stream));
  if (folded) {
    // Q_q = [Q_{1:q-1} U_q] [-Y Y_qq^{-1}; Y_qq^{-1}] from the digit store
    StoreProjDesc p;
    memset(&p, 0, sizeof(p));
    p.qs = h->qs();
    p.c = c + s;
    p.B = h->buf(h->L.Bp);
    p.ldb = h->n_max;
    p.s = s;
    p.nouts = 1;
    p.out[0] = ProjOut{nullptr, 0, nullptr, 0, reinterpret_cast<double*>(h->Qblk(q)), h->ldq, h->Qmax(q)};
    p.m = h->m;
    p.block = q;
    p.fexp = h->fexp();
    p.fp32 = h->fp32;
    TRY(launch_project_store(p, h->st(), h->stream));
  } else {
    TRY(project(h, h->Useg(), c, G, ldg, h->buf(h->L.Yd), h->Qblk(q), h->ldq, h->Qmax(q)));
  }
  TRY(wrote_q(h, q));
  return BCGS_OK;
}

// One block step of BCGSI+P-1S (Alg. 2), BCGSI+P-2S or BCGSI+1s for block
// j >= 3 (k = j - 1): the synchronization of block k, the tail, Q_k and U_{k+1}.
// BCGSI+1s is Alg. 2 without its first Cholesky line: U_{k+1} = X_{k+1} - Q_k S
// is not normalized (S_{k+1,k+1} stays the identity) and T is not formed.
int step_p(bcgs_qr_s* h, const void* X, int64_t ldx) {
  const int s = h->s, j = h->j + 1, k = j - 1;
  const int c = (k - 1) * s;
  const bool one_sync = h->variant == BCGS_BCGSI_PLUS_P_1S;
  const bool unnormalized = h->variant == BCGS_BCGSI_PLUS_1S;
  const Seg Xs = seg(X, ldx, s, h->fp32);
  double* G = h->buf(h->L.G);
  const int ldg = h->L.ldg;
  if (h->x_put) {
    // X_j's digits went into the store ahead (previous step): only its failure,
    // if any, is recorded now, where the split itself would have recorded it
    TRY(launch_merge_status(h->st(), h->st_side(), h->stream));
    h->x_put = 0;
  } else {
    TRY(store_put(h, X, ldx, c + s));
  }
  if (one_sync)
    TRY(gram_cols(h, c + 2 * s, c, 2 * s, {h->Qseg(c), h->Useg(), Xs}, {h->Useg(), Xs}, G));
  else
    TRY(gram_cols(h, c + s, c, 2 * s, {h->Qseg(c), h->Useg()}, {h->Useg(), Xs}, G));
  // X_{j+1}'s digits (store columns [c + 2s, c + 3s), which nothing reads before
  // the next Gram) are split on the side stream while the tail runs; the
  // factorization's stream waits for them before the projection.  Only for s a
  // multiple of 16: a split fills its 16-column chunk up with zero digits, so
  // with s = 8 the split of U_{k+1} at the end of this step would clear them.
  SideStream* side = nullptr;
  if (h->next_X != nullptr && h->sgram && s % 16 == 0 && h->m >= kAheadMinRows && h->width(j + 1) == s)
    side = side_stream(h->stream);
  if (side != nullptr) {
    TRY(cudaEventRecord(side->fork, h->stream));
    TRY(cudaStreamWaitEvent(side->s, side->fork, 0));
    TRY(launch_qsplit(h->qs(), h->next_X, h->next_ldx, h->Q, h->ldq, h->m, c + 2 * s, s, h->fp32, h->st_side(),
                      j + 1, side->s));
    TRY(cudaEventRecord(side->join, side->s));
    h->x_put = 1;
  }
  const int nxt = 1 - h->cur;
  TailDesc t;
  memset(&t, 0, sizeof(t));
  t.s = s;
  t.c = c;
  t.G = G;
  t.ldg = ldg;
  t.gy = 0;
  t.gz = s * ldg;
  t.gom = c;
  t.gp = c + s * ldg;
  t.gt = c + s + s * ldg;
  t.S_prev = h->buf(h->L.S[h->cur]);
  t.Sd_prev = h->buf(h->L.Sd[h->cur]);
  t.S_next = h->buf(h->L.S[nxt]);
  t.Sd_next = h->buf(h->L.Sd[nxt]);
  t.Yd = h->buf(h->L.Yd);
  t.R = h->R;
  t.ldr = h->ldr;
  t.r_row0 = 0;
  t.r_col0 = c;
  t.has_next = 1;
  t.chol_next = one_sync ? 1 : 0;
  t.block = k;
  t.ldsm = h->n_max;
  // Paired projection from the digit store: Q_k and the next block in one pass
  // over [Q_{1:k-1} U_k] (qstore.cu); the tail supplies its coefficients.
  ProjDesc probe;
  memset(&probe, 0, sizeof(probe));
  probe.q = h->Qseg(c);
  probe.m = h->m;
  probe.s = s;
  // [Q_{1:k-1} U_k] from the store: U_k is there when the Grams use it
  const bool paired = h->sgram && use_tensor_project(probe) && project_store_supported(s, 2);
  // s = 32 (past the paired kernel's tensor memory): the same coefficients,
  // applied by two single-output passes over [Q_{1:k-1} U_k]
  const bool two_pass = !paired && h->sgram && use_tensor_project(probe) && project_store_supported(s, 1);
  if (paired || two_pass) {
    t.Bpair = h->buf(h->L.Bp);
    t.ldb = h->n_max;
  }
  TRY(launch_tail_1s2s(t, h->st(), h->stream));
  if (side != nullptr) TRY(cudaStreamWaitEvent(h->stream, side->join, 0));
  if (paired || two_pass) {
    TRY(zero_umax(h));
    StoreProjDesc p;
    memset(&p, 0, sizeof(p));
    p.qs = h->qs();
    p.c = c + s;
    p.B = h->buf(h->L.Bp);
    p.ldb = h->n_max;
    p.s = s;
    p.nouts = 2;
    // Q_k from the folded coefficients [-Y Y_kk^{-1}; Y_kk^{-1}]: no FP64 epilogue
    p.out[0] = ProjOut{nullptr, 0, nullptr, 0, reinterpret_cast<double*>(h->Qblk(k)), h->ldq, h->Qmax(k)};
    if (one_sync)
      p.out[1] = ProjOut{reinterpret_cast<const double*>(X), ldx, h->buf(h->L.Sd[nxt]), s,
                         reinterpret_cast<double*>(h->U()), h->L.ldu, h->Umax()};
    else if (unnormalized)
      p.out[1] = ProjOut{reinterpret_cast<const double*>(X), ldx, nullptr, s,
                         reinterpret_cast<double*>(h->U()), h->L.ldu, h->Umax()};
    else
      p.out[1] = ProjOut{reinterpret_cast<const double*>(X), ldx, nullptr, s,
                         reinterpret_cast<double*>(h->V()), h->L.ldu, MaxOut{nullptr, nullptr}};
    p.m = h->m;
    p.block = k;
    p.fexp = h->fexp();
    p.fp32 = h->fp32;
    if (paired) {
      TRY(launch_project_store(p, h->st(), h->stream));
    } else {
      // Q_k with B[:, 0:s], then the next block with B[:, s:2s] (both read U_k's
      // digits, so Q_k's replace them only afterwards)
      StoreProjDesc p1 = p;
      p1.nouts = 1;
      TRY(launch_project_store(p1, h->st(), h->stream));
      StoreProjDesc p2 = p;
      p2.nouts = 1;
      p2.B = p.B + (size_t)s * p.ldb;
      p2.out[0] = p.out[1];
      TRY(launch_project_store(p2, h->st(), h->stream));
    }
    TRY(wrote_q(h, k));
    if (!one_sync && !unnormalized)
      TRY(tsqr(h, h->Vseg(), h->U(), h->L.ldu, h->buf(h->L.Sd[nxt]), s, k + 1, h->Umax()));
    TRY(store_put(h, h->U(), h->L.ldu, k * s));
    h->cur = nxt;
    return BCGS_OK;
  }
  // Q_k = (U_k - Q_{1:k-1} Y_{1:k-1,k}) Y_kk^{-1}
  TRY(project(h, h->Useg(), c, G, ldg, h->buf(h->L.Yd), h->Qblk(k), h->ldq, h->Qmax(k)));
  TRY(wrote_q(h, k));
  TRY(zero_umax(h));
  if (one_sync) {
    // U_{k+1} = (X_{k+1} - Q_{1:k} S_{1:k,k+1}) S_{k+1,k+1}^{-1}
    TRY(project(h, Xs, c + s, h->buf(h->L.S[nxt]), h->n_max, h->buf(h->L.Sd[nxt]), h->U(),
                h->L.ldu, h->Umax()));
  } else if (unnormalized) {
    // U_{k+1} = X_{k+1} - Q_{1:k} S_{1:k,k+1}  (BCGSI+1s: not normalized)
    TRY(project(h, Xs, c + s, h->buf(h->L.S[nxt]), h->n_max, nullptr, h->U(), h->L.ldu, h->Umax()));
  } else {
    // [U_{k+1}, S_{k+1,k+1}] = TSQR(X_{k+1} - Q_{1:k} S_{1:k,k+1})
    TRY(project(h, Xs, c + s, h->buf(h->L.S[nxt]), h->n_max, nullptr, h->V(), h->L.ldu));
    TRY(tsqr(h, h->Vseg(), h->U(), h->L.ldu, h->buf(h->L.Sd[nxt]), s, k + 1, h->Umax()));
  }
  TRY(store_put(h, h->U(), h->L.ldu, k * s));
  h->cur = nxt;
  return BCGS_OK;
}

// One BCGSI+ step (two projections, each followed by TSQR) for the block X
// (sb columns, block index j) against Q's first c final columns:
//   S = Q^T X;  [U, S_jj] = TSQR(X - Q S);  Y = Q^T U;  [Q_j, Y_jj] = TSQR(U - Q Y)
//   R_{1:c,j} = S + Y S_jj;  R_jj = Y_jj S_jj
int step_bcgsi(bcgs_qr_s* h, const void* X, int64_t ldx, int j, int c, int sb) {
  const Seg Xs = seg(X, ldx, sb, h->fp32);
  double* G = h->buf(h->L.G);
  double* G2 = h->buf(h->L.G2);
  const int ldg = h->L.ldg;
  TRY(store_put(h, X, ldx, c, sb));
  TRY(gram_cols(h, c, c, sb, {h->Qseg(c)}, {Xs}, G));
  TRY(project(h, Xs, c, G, ldg, nullptr, h->V(), h->L.ldu, MaxOut{nullptr, nullptr}, sb));
  TRY(zero_umax(h, sb));
  TRY(tsqr(h, h->Vseg(sb), h->U(), h->L.ldu, h->buf(h->L.Rt1), sb, j, h->Umax()));
  TRY(store_put(h, h->U(), h->L.ldu, c, sb));
  TRY(gram_cols(h, c, c, sb, {h->Qseg(c)}, {h->Useg(sb)}, G2));
  TRY(project(h, h->Useg(sb), c, G2, ldg, nullptr, h->V(), h->L.ldu, MaxOut{nullptr, nullptr}, sb));
  TRY(tsqr(h, h->Vseg(sb), h->Qcol(c), h->ldq, h->buf(h->L.Rt2), sb, j, h->Qmax_at(c)));
  TRY(wrote_q_cols(h, c, sb, j));
  TRY(launch_r_assemble(c, sb, G, ldg, G2, ldg, h->buf(h->L.Rt1), h->buf(h->L.Rt2), h->R, h->ldr, c, h->st(),
                        h->stream));
  return BCGS_OK;
}

// One BCGS-PIPI+ step (Alg. 1) for the block X (sb columns, block index j)
// against Q's first c final columns:
//   [S; T] = [Q X]^T X, S_jj = chol(T - S^T S), U = (X - Q S) S_jj^{-1}
//   [Y; Omega] = [Q U]^T U, Y_jj = chol(Omega - Y^T Y), Q_j = (U - Q Y) Y_jj^{-1}
//   R_{1:c,j} = S + Y S_jj;  R_jj = Y_jj S_jj
int step_pipi(bcgs_qr_s* h, const void* X, int64_t ldx, int j, int c, int sb) {
  const Seg Xs = seg(X, ldx, sb, h->fp32);
  double* G = h->buf(h->L.G);
  double* G2 = h->buf(h->L.G2);
  const int ldg = h->L.ldg;
  double* Skk = h->buf(h->L.Rt1);
  double* Ykk = h->buf(h->L.Rt2);
  TRY(store_put(h, X, ldx, c, sb));
  TRY(gram_cols(h, c + sb, c, sb, {h->Qseg(c), Xs}, {Xs}, G));
  TRY(launch_tail_pchol(c, sb, G, ldg, nullptr, 0, Skk, j, h->st(), h->stream));
  TRY(zero_umax(h, sb));
  TRY(project(h, Xs, c, G, ldg, Skk, h->U(), h->L.ldu, h->Umax(), sb));
  TRY(store_put(h, h->U(), h->L.ldu, c, sb));
  TRY(gram_cols(h, c + sb, c, sb, {h->Qseg(c), h->Useg(sb)}, {h->Useg(sb)}, G2));
  TRY(launch_tail_pchol(c, sb, G2, ldg, nullptr, 0, Ykk, j, h->st(), h->stream));
  TRY(project(h, h->Useg(sb), c, G2, ldg, Ykk, h->Qcol(c), h->ldq, h->Qmax_at(c), sb));
  TRY(wrote_q_cols(h, c, sb, j));
  TRY(launch_r_assemble(c, sb, G, ldg, G2, ldg, Skk, Ykk, h->R, h->ldr, c, h->st(), h->stream));
  return BCGS_OK;
}

// A ragged last block (sb = n_max mod s columns; the paper assumes n = q s):
// the delayed block of BCGSI+P-1S / -2S is finalized first (their last-block
// branch), then the ragged block takes one step of the variant of the same
// stability range whose step finalizes it at once: BCGS-PIPI+ for 1S and
// PIPI+ (and for BCGSI+1s, whose range it contains), BCGSI+ for BCGSI+ and 2S.  A first block that is already ragged
// (n_max < s) is TSQR alone.
int step_ragged(bcgs_qr_s* h, const void* X, int64_t ldx, int sb) {
  const int j = h->j + 1, c = h->j * h->s;
  if (j == 1) {
    TRY(tsqr(h, seg(X, ldx, sb, h->fp32), h->Q, h->ldq, h->R, h->ldr, 1, h->Qmax_at(0)));
    TRY(wrote_q_cols(h, 0, sb, 1));
    return BCGS_OK;
  }
  if (h->delayed() && h->j >= 2) {
    const int rc = finish_p(h);
    if (rc != BCGS_OK) return rc;
  }
  h->flushed = 1;  // after the ragged step every block is final: nothing left for finish
  if (h->variant == BCGS_BCGSI_PLUS_P_1S || h->variant == BCGS_BCGS_PIPI_PLUS || h->variant == BCGS_BCGSI_PLUS_1S)
    return step_pipi(h, X, ldx, j, c, sb);
  return step_bcgsi(h, X, ldx, j, c, sb);
}

int do_step(bcgs_qr_s* h, const void* X, int64_t ldx) {
  const int s = h->s, j = h->j + 1;
  if (h->width(j) < s) return step_ragged(h, X, ldx, h->width(j));
  const Seg Xs = seg(X, ldx, s, h->fp32);
  double* G = h->buf(h->L.G);
  const int ldg = h->L.ldg;
  if (j == 1) {
    // [Q_1, R_11] = TSQR(X_1)
    TRY(tsqr(h, Xs, h->Qblk(1), h->ldq, h->R, h->ldr, 1, h->Qmax(1)));
    TRY(wrote_q(h, 1));
    return BCGS_OK;
  }
  switch (h->variant) {
    case BCGS_BCGSI_PLUS:
      return step_bcgsi(h, X, ldx, j, (j - 1) * s, s);
    case BCGS_BCGSI_PLUS_P_1S:
      if (j == 2) {
        // [S_12; T_2] = [Q_1 X_2]^T X_2, S_22 = chol(T_2 - S_12^T S_12), U_2
        TRY(store_put(h, X, ldx, s));
        TRY(gram_cols(h, 2 * s, s, s, {h->Qseg(s), Xs}, {Xs}, G));
        TRY(launch_tail_pchol(s, s, G, ldg, h->buf(h->L.S[h->cur]), h->n_max, h->buf(h->L.Sd[h->cur]), 2,
                              h->st(), h->stream));
        TRY(zero_umax(h));
        TRY(project(h, Xs, s, h->buf(h->L.S[h->cur]), h->n_max, h->buf(h->L.Sd[h->cur]), h->U(),
                    h->L.ldu, h->Umax()));
        TRY(store_put(h, h->U(), h->L.ldu, s));
        return BCGS_OK;
      }
      return step_p(h, X, ldx);
    case BCGS_BCGSI_PLUS_P_2S:
      if (j == 2) {
        // S_12 = Q_1^T X_2, [U_2, S_22] = TSQR(X_2 - Q_1 S_12)
        TRY(store_put(h, X, ldx, s));
        TRY(gram_cols(h, s, s, s, {h->Qseg(s)}, {Xs}, G));
        TRY(launch_copy_small(s, s, G, ldg, h->buf(h->L.S[h->cur]), h->n_max, h->st(), h->stream));
        TRY(project(h, Xs, s, G, ldg, nullptr, h->V(), h->L.ldu));
        TRY(zero_umax(h));
        TRY(tsqr(h, h->Vseg(), h->U(), h->L.ldu, h->buf(h->L.Sd[h->cur]), s, 2, h->Umax()));
        TRY(store_put(h, h->U(), h->L.ldu, s));
        return BCGS_OK;
      }
      return step_p(h, X, ldx);
    case BCGS_BCGS_PIPI_PLUS:
      return step_pipi(h, X, ldx, j, (j - 1) * s, s);
    case BCGS_BCGSI_PLUS_1S:
      if (j == 2) {
        // S_12 = Q_1^T X_2, U_2 = X_2 - Q_1 S_12 (not normalized: S_22 = I)
        TRY(store_put(h, X, ldx, s));
        TRY(gram_cols(h, s, s, s, {h->Qseg(s)}, {Xs}, G));
        TRY(launch_copy_small(s, s, G, ldg, h->buf(h->L.S[h->cur]), h->n_max, h->st(), h->stream));
        TRY(zero_umax(h));
        TRY(project(h, Xs, s, G, ldg, nullptr, h->U(), h->L.ldu, h->Umax()));
        TRY(store_put(h, h->U(), h->L.ldu, s));
        return BCGS_OK;
      }
      return step_p(h, X, ldx);
  }
  return BCGS_ERR_INVALID_ARG;
}

// Row-partitioned form: a rank's slab needs s rows (its local TSQR), not n.
bool valid_local_shape(int64_t m, int32_t n, int32_t s) {
  return s >= 1 && s <= kMaxS && n >= 1 && n <= kMaxN && m >= s;
}

int init_handle(bcgs_qr_s* h, int64_t m, int32_t n_max, int32_t s, int variant, int precision,
                void* Q, int64_t ldq, double* R, int32_t ldr, void* workspace, size_t ws_bytes,
                void* stream, int32_t rank = 0, int32_t nranks = 1, bcgs_allgather_fn allgather = nullptr,
                void* ag_ctx = nullptr) {
  if (nranks < 1 || rank < 0 || rank >= nranks || (nranks > 1 && allgather == nullptr)) return BCGS_ERR_INVALID_ARG;
  if (nranks > 1 ? !valid_local_shape(m, n_max, s) : !valid_shape(m, n_max, s)) return BCGS_ERR_INVALID_ARG;
  if (variant < 0 || variant > 4 || precision < 0 || precision > 1) return BCGS_ERR_INVALID_ARG;
  if (Q == nullptr || R == nullptr || workspace == nullptr) return BCGS_ERR_INVALID_ARG;
  if (ldq < m || ldr < n_max) return BCGS_ERR_INVALID_ARG;
  if (((uintptr_t)workspace) % 256 != 0) return BCGS_ERR_WORKSPACE;
  memset(h, 0, sizeof(*h));
  make_layout(m, n_max, s, variant, precision, want_store(m, s, precision), &h->L, nranks);
  if (ws_bytes < h->L.total && h->L.store)  // sized without the store: run without it
    make_layout(m, n_max, s, variant, precision, 0, &h->L, nranks);
  if (ws_bytes < h->L.total) return BCGS_ERR_WORKSPACE;
  h->m = m;
  h->n_max = n_max;
  h->s = s;
  h->variant = variant;
  h->precision = precision;
  h->Q = reinterpret_cast<char*>(Q);
  h->ldq = ldq;
  h->R = R;
  h->ldr = ldr;
  h->ws = reinterpret_cast<char*>(workspace);
  h->ws_bytes = ws_bytes;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->fp32 = precision == BCGS_FP32_STORAGE ? 1 : 0;
  h->esz = h->fp32 ? 4 : 8;
  h->rank = rank;
  h->nranks = nranks;
  h->allgather = allgather;
  h->ag_ctx = ag_ctx;
  // Grams from the store need whole 8-column groups per block (a Gram with more
  // than 32 B columns runs as several launches of at most 32, gram_local)
  h->sgram = h->L.store && s % 8 == 0 && s <= 32;
  h->j = 0;
  h->cur = 0;
  h->finished = 0;
  TRY(launch_reset_status(h->st(), h->stream, h->st_side()));
  TRY(launch_zero_lower(n_max, R, ldr, h->stream));
  TRY(launch_zero_u64(h->amaxQ(), n_max, h->stream));
  TRY(launch_zero_u64(h->rowmaxQ(), m, h->stream));
  if (variant == BCGS_BCGSI_PLUS_1S)  // S_{k,k} = I for every block (no first normalization)
    for (int i = 0; i < 2; ++i) TRY(launch_set_identity(s, h->buf(h->L.Sd[i]), h->stream));
  return BCGS_OK;
}

// NVTX range over the host-side enqueue of one block step (tools show it
// against the kernels it launched)
struct StepRange {
  explicit StepRange(const char* name) { nvtxRangePushA(name); }
  ~StepRange() { nvtxRangePop(); }
};

int step_handle(bcgs_qr_s* h, const void* X, int64_t ldx) {
  if (h->finished || (int64_t)h->j * h->s >= h->n_max) return BCGS_ERR_STATE;
  static const char* kNames[5] = {"bcgs step (BCGSI+)", "bcgs step (BCGSI+P-1S)", "bcgs step (BCGSI+P-2S)",
                                  "bcgs step (BCGS-PIPI+)", "bcgs step (BCGSI+1s)"};
  StepRange range(kNames[h->variant]);
  if (X == nullptr || ldx < h->m) return BCGS_ERR_INVALID_ARG;
  const int rc = do_step(h, X, ldx);
  if (rc != BCGS_OK) return rc;
  h->j += 1;
  return BCGS_OK;
}

int finish_handle(bcgs_qr_s* h) {
  if (h->finished) return BCGS_OK;
  StepRange range("bcgs finish");
  if (h->j == 0) return BCGS_ERR_STATE;
  if (h->delayed() && h->j >= 2 && !h->flushed) {
    const int rc = finish_p(h);
    if (rc != BCGS_OK) return rc;
  }
  h->finished = 1;
  return BCGS_OK;
}

int read_status(const void* ws, cudaStream_t stream, int32_t* code, int32_t* block) {
  DevStatus hs;
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return BCGS_ERR_CUDA;
  e = cudaMemcpy(&hs, ws, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return BCGS_ERR_CUDA;
  *code = hs.code;
  *block = hs.block;
  return BCGS_OK;
}

// Internal streams of the batched form, created on first use per device and
// kept for the life of the process (streams and events only; no memory).
constexpr int kBatchLanes = 16;
struct BatchStreams {
  cudaStream_t lane[kBatchLanes];
  cudaEvent_t fork;
  cudaEvent_t join[kBatchLanes];
  std::mutex call;  // one batched call enqueues its fork, lanes and join at a time
};
std::mutex g_batch_mu;
BatchStreams* g_batch[64] = {nullptr};

int batch_streams(BatchStreams** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return BCGS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_batch_mu);
  if (g_batch[dev] == nullptr) {
    BatchStreams* bs = new (std::nothrow) BatchStreams;
    if (bs == nullptr) return BCGS_ERR_INVALID_ARG;
    for (int l = 0; l < kBatchLanes; ++l) {
      if (cudaStreamCreateWithFlags(&bs->lane[l], cudaStreamNonBlocking) != cudaSuccess)
        return BCGS_ERR_CUDA;
      if (cudaEventCreateWithFlags(&bs->join[l], cudaEventDisableTiming) != cudaSuccess)
        return BCGS_ERR_CUDA;
    }
    if (cudaEventCreateWithFlags(&bs->fork, cudaEventDisableTiming) != cudaSuccess) return BCGS_ERR_CUDA;
    g_batch[dev] = bs;
  }
  *out = g_batch[dev];
  return BCGS_OK;
}

// The two copy streams of bcgs_qr_factor_host (one per direction) and the
// events that order them against the caller's stream, one set per device.
struct CopyStreams {
  cudaStream_t h2d, d2h;
  cudaEvent_t start, in, out, done;
  std::mutex call;  // one host call enqueues its copies and events at a time
};
std::mutex g_copy_mu;
CopyStreams* g_copy[64] = {nullptr};

int copy_streams(CopyStreams** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return BCGS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_copy_mu);
  if (g_copy[dev] == nullptr) {
    CopyStreams* cs = new (std::nothrow) CopyStreams;
    if (cs == nullptr) return BCGS_ERR_INVALID_ARG;
    if (cudaStreamCreateWithFlags(&cs->h2d, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&cs->d2h, cudaStreamNonBlocking) != cudaSuccess)
      return BCGS_ERR_CUDA;
    cudaEvent_t* evs[4] = {&cs->start, &cs->in, &cs->out, &cs->done};
    for (cudaEvent_t* e : evs)
      if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return BCGS_ERR_CUDA;
    g_copy[dev] = cs;
  }
  *out = g_copy[dev];
  return BCGS_OK;
}

}  // namespace

namespace {
// One-call factorization; `ahead`: split each next block of X into the store
// while the current step's tail runs (on this thread's side stream).
int factor_impl(int64_t m, int32_t n, int32_t s, int variant, int precision, const void* X, int64_t ldx, void* Q,
                int64_t ldq, double* R, int32_t ldr, void* workspace, size_t ws_bytes, void* stream, bool ahead) {
  if (X == nullptr || ldx < m) return BCGS_ERR_INVALID_ARG;
  // in-place factorization (Q overlapping X) is not supported
  if (precision >= 0 && precision <= 1 &&
      overlaps(X, ldx, Q, ldq, m, n, precision == BCGS_FP32_STORAGE ? 4 : 8))
    return BCGS_ERR_INVALID_ARG;
  bcgs_qr_s hs;
  bcgs_qr_s* h = &hs;
  int rc = init_handle(h, m, n, s, variant, precision, Q, ldq, R, ldr, workspace, ws_bytes, stream);
  if (rc != BCGS_OK) return rc;
  const size_t esz = precision == BCGS_FP32_STORAGE ? 4 : 8;
  const char* Xc = reinterpret_cast<const char*>(X);
  const int q = (n + s - 1) / s;  // the last block may be ragged
  for (int k = 0; k < q; ++k) {
    h->next_X = ahead && k + 1 < q ? Xc + (size_t)(k + 1) * s * ldx * esz : nullptr;
    h->next_ldx = ldx;
    rc = step_handle(h, Xc + (size_t)k * s * ldx * esz, ldx);
    if (rc != BCGS_OK) return rc;
  }
  h->next_X = nullptr;
  return finish_handle(h);
}
}  // namespace

extern "C" {

const char* bcgs_status_string(int status) {
  switch (status) {
    case BCGS_OK: return "ok";
    case BCGS_ERR_INVALID_ARG: return "invalid argument";
    case BCGS_ERR_NOT_SPD: return "Cholesky breakdown (matrix not positive definite)";
    case BCGS_ERR_RANK_DEFICIENT: return "rank deficient block (zero R diagonal)";
    case BCGS_ERR_NONFINITE: return "non-finite value";
    case BCGS_ERR_WORKSPACE: return "workspace too small or misaligned";
    case BCGS_ERR_TIMEOUT: return "device wait timed out";
    case BCGS_ERR_STATE: return "call out of order";
    case BCGS_ERR_CUDA: return "CUDA runtime error";
    case BCGS_ERR_COMM: return "the all-gather callback of the row-partitioned form failed";
  }
  return "unknown status";
}

int bcgs_version(void) { return 100; }

int bcgs_set_option(int option, int64_t value) {
  switch (option) {
    case BCGS_OPT_GRAM_ENGINE:
      if (value < 0 || value > 2) return BCGS_ERR_INVALID_ARG;
      g_engine.store((int)value);
      return BCGS_OK;
    case BCGS_OPT_TC_MIN_ROWS:
      if (value < 1) return BCGS_ERR_INVALID_ARG;
      g_tc_min_rows.store(value);
      return BCGS_OK;
    case BCGS_OPT_DEBUG_SYNC:
      if (value < 0 || value > 1) return BCGS_ERR_INVALID_ARG;
      g_debug_sync.store((int)value);
      return BCGS_OK;
  }
  return BCGS_ERR_INVALID_ARG;
}

int64_t bcgs_get_option(int option) {
  switch (option) {
    case BCGS_OPT_GRAM_ENGINE: return g_engine.load();
    case BCGS_OPT_TC_MIN_ROWS: return g_tc_min_rows.load();
    case BCGS_OPT_DEBUG_SYNC: return g_debug_sync.load();
  }
  return -1;
}

int bcgs_qr_workspace_size(int64_t m, int32_t n_max, int32_t s, int variant, int precision,
                           size_t* bytes) {
  if (bytes == nullptr || !valid_shape(m, n_max, s)) return BCGS_ERR_INVALID_ARG;
  if (variant < 0 || variant > 4 || precision < 0 || precision > 1) return BCGS_ERR_INVALID_ARG;
  Layout L;
  make_layout(m, n_max, s, variant, precision, want_store(m, s, precision), &L);
  *bytes = L.total;
  return BCGS_OK;
}


int bcgs_qr_factor(int64_t m, int32_t n, int32_t s, int variant, int precision, const void* X,
                   int64_t ldx, void* Q, int64_t ldq, double* R, int32_t ldr, void* workspace,
                   size_t ws_bytes, void* stream) {
  return factor_impl(m, n, s, variant, precision, X, ldx, Q, ldq, R, ldr, workspace, ws_bytes, stream, true);
}

int bcgs_row_partition(int64_t m, int32_t nranks, int32_t rank, int64_t* row0, int64_t* rows) {
  if (m < 1 || nranks < 1 || rank < 0 || rank >= nranks || row0 == nullptr || rows == nullptr)
    return BCGS_ERR_INVALID_ARG;
  // whole 128-row blocks, as even as possible, the first nblk mod nranks ranks one more
  const int64_t nblk = ceil_div(m, kStoreRows);
  const int64_t base = nblk / nranks, extra = nblk % nranks;
  const int64_t b0 = (int64_t)rank * base + (rank < extra ? rank : extra);
  const int64_t nb = base + (rank < extra ? 1 : 0);
  const int64_t r0 = b0 * kStoreRows;
  int64_t r1 = (b0 + nb) * kStoreRows;
  if (r1 > m) r1 = m;
  *row0 = r0 < m ? r0 : m;
  *rows = r1 > r0 ? r1 - r0 : 0;
  return BCGS_OK;
}

int bcgs_qr_workspace_size_rows(int64_t m_local, int32_t n, int32_t s, int variant, int precision, int32_t nranks,
                                size_t* bytes) {
  if (bytes == nullptr || nranks < 1 || nranks > 4096) return BCGS_ERR_INVALID_ARG;
  if (nranks > 1 ? !valid_local_shape(m_local, n, s) : !valid_shape(m_local, n, s)) return BCGS_ERR_INVALID_ARG;
  if (variant < 0 || variant > 4 || precision < 0 || precision > 1) return BCGS_ERR_INVALID_ARG;
  Layout L;
  make_layout(m_local, n, s, variant, precision, want_store(m_local, s, precision), &L, nranks);
  *bytes = L.total;
  return BCGS_OK;
}

int bcgs_qr_factor_rows(int64_t m_local, int32_t n, int32_t s, int variant, int precision, const void* X, int64_t ldx,
                        void* Q, int64_t ldq, double* R, int32_t ldr, void* workspace, size_t ws_bytes, void* stream,
                        int32_t rank, int32_t nranks, bcgs_allgather_fn allgather, void* ctx) {
  if (X == nullptr || ldx < m_local || nranks > 4096) return BCGS_ERR_INVALID_ARG;
  if (precision >= 0 && precision <= 1 &&
      overlaps(X, ldx, Q, ldq, m_local, n, precision == BCGS_FP32_STORAGE ? 4 : 8))
    return BCGS_ERR_INVALID_ARG;
  bcgs_qr_s hs;
  bcgs_qr_s* h = &hs;
  int rc = init_handle(h, m_local, n, s, variant, precision, Q, ldq, R, ldr, workspace, ws_bytes, stream, rank,
                       nranks, allgather, ctx);
  if (rc != BCGS_OK) return rc;
  const size_t esz = precision == BCGS_FP32_STORAGE ? 4 : 8;
  const char* Xc = reinterpret_cast<const char*>(X);
  const int q = (n + s - 1) / s;
  for (int k = 0; k < q; ++k) {
    rc = step_handle(h, Xc + (size_t)k * s * ldx * esz, ldx);
    if (rc != BCGS_OK) return h->comm_failed ? BCGS_ERR_COMM : rc;
  }
  rc = finish_handle(h);
  return (rc != BCGS_OK && h->comm_failed) ? BCGS_ERR_COMM : rc;
}

int bcgs_qr_factor_host(int64_t m, int32_t n, int32_t s, int variant, int precision, const void* X_host,
                        int64_t ldxh, void* Q_host, int64_t ldqh, double* R_host, int32_t ldrh, void* Xd,
                        int64_t ldx, void* Qd, int64_t ldq, double* Rd, int32_t ldr, void* workspace,
                        size_t ws_bytes, void* stream) {
  if (X_host == nullptr || Q_host == nullptr || R_host == nullptr || Xd == nullptr) return BCGS_ERR_INVALID_ARG;
  if (ldxh < m || ldqh < m || ldx < m || ldrh < n) return BCGS_ERR_INVALID_ARG;
  if (precision >= 0 && precision <= 1 &&
      overlaps(Xd, ldx, Qd, ldq, m, n, precision == BCGS_FP32_STORAGE ? 4 : 8))
    return BCGS_ERR_INVALID_ARG;
  bcgs_qr_s hs;
  bcgs_qr_s* h = &hs;
  int rc = init_handle(h, m, n, s, variant, precision, Qd, ldq, Rd, ldr, workspace, ws_bytes, stream);
  if (rc != BCGS_OK) return rc;
  CopyStreams* cs = nullptr;
  rc = copy_streams(&cs);
  if (rc != BCGS_OK) return rc;
  // shared by every caller on this device: host threads enqueue one call at a time
  std::lock_guard<std::mutex> lk(cs->call);
  const size_t esz = precision == BCGS_FP32_STORAGE ? 4 : 8;
  const int q = (n + s - 1) / s;  // the last block may be ragged
  const cudaStream_t main = h->stream;
  const char* Xh = reinterpret_cast<const char*>(X_host);
  char* Qh = reinterpret_cast<char*>(Q_host);
  char* Xdc = reinterpret_cast<char*>(Xd);
  const char* Qdc = reinterpret_cast<const char*>(Qd);
  // block columns [k0, k1) of X to the device, of Q to the host (the last one may be ragged)
  auto ncols = [&](int k0, int k1) {
    const int64_t e = (int64_t)k1 * s < n ? (int64_t)k1 * s : n;
    return (size_t)(e - (int64_t)k0 * s);
  };
  auto h2d = [&](int k0, int k1) {
    return cudaMemcpy2DAsync(Xdc + (size_t)k0 * s * ldx * esz, (size_t)ldx * esz, Xh + (size_t)k0 * s * ldxh * esz,
                             (size_t)ldxh * esz, (size_t)m * esz, ncols(k0, k1), cudaMemcpyHostToDevice, cs->h2d);
  };
  auto d2h = [&](int k0, int k1) {
    return cudaMemcpy2DAsync(Qh + (size_t)k0 * s * ldqh * esz, (size_t)ldqh * esz, Qdc + (size_t)k0 * s * ldq * esz,
                             (size_t)ldq * esz, (size_t)m * esz, ncols(k0, k1), cudaMemcpyDeviceToHost, cs->d2h);
  };
  // the copies start after what `stream` already holds (Xd, Qd may still be in use)
  TRY(cudaEventRecord(cs->start, main));
  TRY(cudaStreamWaitEvent(cs->h2d, cs->start, 0));
  TRY(cudaStreamWaitEvent(cs->d2h, cs->start, 0));
  TRY(h2d(0, 1));
  TRY(cudaEventRecord(cs->in, cs->h2d));
  TRY(cudaStreamWaitEvent(main, cs->in, 0));
  const bool delayed = h->delayed();
  int sent = 0;  // Q blocks already on their way to the host
  for (int k = 0; k < q; ++k) {
    if (k + 1 < q) TRY(h2d(k + 1, k + 2));  // travels while block k is factored
    rc = step_handle(h, Xdc + (size_t)k * s * ldx * esz, ldx);
    if (rc != BCGS_OK) return rc;
    if (k + 1 < q) {
      TRY(cudaEventRecord(cs->in, cs->h2d));
      TRY(cudaStreamWaitEvent(main, cs->in, 0));
    }
    // a ragged last step finalizes every block (the delayed one first)
    const int final_blocks = (delayed && !h->flushed) ? (k > 1 ? k : 1) : k + 1;
    if (final_blocks > sent) {
      TRY(cudaEventRecord(cs->out, main));
      TRY(cudaStreamWaitEvent(cs->d2h, cs->out, 0));
      TRY(d2h(sent, final_blocks));
      sent = final_blocks;
    }
  }
  rc = finish_handle(h);
  if (rc != BCGS_OK) return rc;
  TRY(cudaEventRecord(cs->out, main));
  TRY(cudaStreamWaitEvent(cs->d2h, cs->out, 0));
  if (sent < q) TRY(d2h(sent, q));
  TRY(cudaMemcpy2DAsync(R_host, (size_t)ldrh * sizeof(double), Rd, (size_t)ldr * sizeof(double),
                        (size_t)n * sizeof(double), (size_t)n, cudaMemcpyDeviceToHost, cs->d2h));
  TRY(cudaEventRecord(cs->done, cs->d2h));
  TRY(cudaStreamWaitEvent(main, cs->done, 0));
  return BCGS_OK;
}

int bcgs_wait_selftest(void* workspace, size_t ws_bytes, int64_t cycles, void* stream) {
  if (workspace == nullptr || ws_bytes < 256 || cycles < 1 || cycles > 2000000000LL) return BCGS_ERR_INVALID_ARG;
  if (((uintptr_t)workspace) % 256 != 0) return BCGS_ERR_WORKSPACE;
  DevStatus* st = reinterpret_cast<DevStatus*>(workspace);
  const cudaStream_t sm = reinterpret_cast<cudaStream_t>(stream);
  if (launch_reset_status(st, sm) != cudaSuccess) return BCGS_ERR_CUDA;
  if (launch_wait_selftest(st, (long long)cycles, sm) != cudaSuccess) return BCGS_ERR_CUDA;
  return BCGS_OK;
}

int bcgs_qr_factor_status(const void* workspace, void* stream, int32_t* fail_block) {
  if (workspace == nullptr) return BCGS_ERR_INVALID_ARG;
  int32_t code = 0, block = 0;
  int rc = read_status(workspace, reinterpret_cast<cudaStream_t>(stream), &code, &block);
  if (rc != BCGS_OK) return rc;
  if (fail_block) *fail_block = code ? block : 0;
  return code;
}

int bcgs_qr_init(bcgs_qr_t* handle, int64_t m, int32_t n_max, int32_t s, int variant,
                 int precision, void* Q, int64_t ldq, double* R, int32_t ldr, void* workspace,
                 size_t ws_bytes, void* stream) {
  if (handle == nullptr) return BCGS_ERR_INVALID_ARG;
  *handle = nullptr;
  bcgs_qr_s* h = static_cast<bcgs_qr_s*>(malloc(sizeof(bcgs_qr_s)));
  if (h == nullptr) return BCGS_ERR_INVALID_ARG;
  const int rc = init_handle(h, m, n_max, s, variant, precision, Q, ldq, R, ldr, workspace,
                             ws_bytes, stream);
  if (rc != BCGS_OK) {
    free(h);
    return rc;
  }
  *handle = h;
  return BCGS_OK;
}

int bcgs_qr_step(bcgs_qr_t h, const void* X_block, int64_t ldx) {
  if (h == nullptr) return BCGS_ERR_INVALID_ARG;
  return step_handle(h, X_block, ldx);
}

int bcgs_qr_finish(bcgs_qr_t h) {
  if (h == nullptr) return BCGS_ERR_INVALID_ARG;
  return finish_handle(h);
}

int bcgs_qr_sync(bcgs_qr_t h, int32_t* n_final, int32_t* fail_block) {
  if (h == nullptr) return BCGS_ERR_INVALID_ARG;
  int32_t code = 0, block = 0;
  int rc = read_status(h->ws + h->L.status, h->stream, &code, &block);
  if (rc != BCGS_OK) return rc;
  if (n_final) {
    int64_t fin;
    if (h->finished || !h->delayed() || h->flushed) fin = (int64_t)h->j * h->s;
    else fin = (int64_t)(h->j <= 1 ? h->j : h->j - 1) * h->s;
    *n_final = code ? 0 : (int32_t)(fin < h->n_max ? fin : h->n_max);
  }
  if (fail_block) *fail_block = code ? block : 0;
  return code;
}

int bcgs_qr_set_stream(bcgs_qr_t h, void* stream) {
  if (h == nullptr) return BCGS_ERR_INVALID_ARG;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  return BCGS_OK;
}

int bcgs_qr_destroy(bcgs_qr_t h) {
  free(h);
  return BCGS_OK;
}

// ------------------------------------------------------------------ building blocks

int bcgs_gram_workspace_size(int64_t m, int32_t ka, int32_t kb, size_t* bytes) {
  if (bytes == nullptr || m < 1 || ka < 1 || kb < 1 || (int64_t)ka * kb > 65536)
    return BCGS_ERR_INVALID_ARG;
  *bytes = align256(sizeof(DevStatus)) + align256(gram_partial_doubles(m, ka, kb) * sizeof(double)) +
           ((size_t)ka + kb) * sizeof(unsigned long long);
  return BCGS_OK;
}

int bcgs_gram(int64_t m, int32_t ka, int32_t kb, const double* A, int64_t lda, const double* B,
              int64_t ldb, double* C, int32_t ldc, void* workspace, size_t ws_bytes, void* stream) {
  size_t need = 0;
  if (bcgs_gram_workspace_size(m, ka, kb, &need) != BCGS_OK) return BCGS_ERR_INVALID_ARG;
  if (!A || !B || !C || !workspace || lda < m || ldb < m || ldc < ka) return BCGS_ERR_INVALID_ARG;
  if (ws_bytes < need || ((uintptr_t)workspace) % 256 != 0) return BCGS_ERR_WORKSPACE;
  char* ws = reinterpret_cast<char*>(workspace);
  DevStatus* st = reinterpret_cast<DevStatus*>(ws);
  cudaStream_t sm = reinterpret_cast<cudaStream_t>(stream);
  if (launch_reset_status(st, sm) != cudaSuccess) return BCGS_ERR_CUDA;
  GramDesc d;
  memset(&d, 0, sizeof(d));
  d.a[0] = seg(A, lda, ka, 0);
  d.b[0] = seg(B, ldb, kb, 0);
  d.nsa = d.nsb = 1;
  d.na = ka;
  d.nb = kb;
  d.m = m;
  gram_partition(m, &d.chunk_rows, &d.nchunks);
  double* partial = reinterpret_cast<double*>(ws + align256(sizeof(DevStatus)));
  cudaError_t e;
  if (use_tensor_gram(d)) {
    auto* amax = reinterpret_cast<unsigned long long*>(
        ws + align256(sizeof(DevStatus)) + align256(gram_partial_doubles(m, ka, kb) * sizeof(double)));
    e = launch_gram_tc(d, partial, C, ldc, amax, st, sm);
  } else {
    e = launch_gram(d, partial, C, ldc, st, sm);
  }
  return e == cudaSuccess ? BCGS_OK : BCGS_ERR_CUDA;
}

int bcgs_project(int64_t m, int32_t c, int32_t s, const double* V, int64_t ldv, const double* Q,
                 int64_t ldq, const double* C, int32_t ldc, const double* T, int32_t ldt, double* W,
                 int64_t ldw, void* stream) {
  if (m < 1 || s < 1 || s > kMaxS || c < 0 || !V || !W || ldv < m || ldw < m)
    return BCGS_ERR_INVALID_ARG;
  if (c > 0 && (!Q || !C || ldq < m || ldc < c)) return BCGS_ERR_INVALID_ARG;
  if (T && ldt < s) return BCGS_ERR_INVALID_ARG;
  ProjDesc d;
  memset(&d, 0, sizeof(d));
  d.v = seg(V, ldv, s, 0);
  d.q = seg(Q, ldq, c, 0);
  d.C = C;
  d.ldc = ldc;
  d.T = T;
  d.ldt = ldt;
  d.w = W;
  d.ldw = ldw;
  d.w_fp32 = 0;
  d.m = m;
  d.s = s;
  cudaStream_t sm = reinterpret_cast<cudaStream_t>(stream);
  const cudaError_t e = use_tensor_project(d) ? launch_project_tc(d, nullptr, sm)
                                              : launch_project(d, nullptr, sm);
  return e == cudaSuccess ? BCGS_OK : BCGS_ERR_CUDA;
}

int bcgs_tsqr_workspace_size(int64_t m, int32_t s, size_t* bytes) {
  if (bytes == nullptr || s < 1 || s > kMaxS || m < s) return BCGS_ERR_INVALID_ARG;
  TsqrPlan p;
  tsqr_plan(m, s, &p);
  *bytes = align256(sizeof(DevStatus)) + p.doubles * sizeof(double);
  return BCGS_OK;
}

int bcgs_tsqr(int64_t m, int32_t s, const double* A, int64_t lda, double* Q, int64_t ldq, double* R,
              int32_t ldr, void* workspace, size_t ws_bytes, void* stream) {
  size_t need = 0;
  if (bcgs_tsqr_workspace_size(m, s, &need) != BCGS_OK) return BCGS_ERR_INVALID_ARG;
  if (!A || !Q || !R || !workspace || lda < m || ldq < m || ldr < s) return BCGS_ERR_INVALID_ARG;
  if (ws_bytes < need || ((uintptr_t)workspace) % 256 != 0) return BCGS_ERR_WORKSPACE;
  char* ws = reinterpret_cast<char*>(workspace);
  DevStatus* st = reinterpret_cast<DevStatus*>(ws);
  cudaStream_t sm = reinterpret_cast<cudaStream_t>(stream);
  if (launch_reset_status(st, sm) != cudaSuccess) return BCGS_ERR_CUDA;
  TsqrPlan p;
  tsqr_plan(m, s, &p);
  if (launch_tsqr(p, seg(A, lda, s, 0), Q, ldq, 0, R, ldr,
                  reinterpret_cast<double*>(ws + align256(sizeof(DevStatus))), st, 1,
                  sm) != cudaSuccess)
    return BCGS_ERR_CUDA;
  return BCGS_OK;
}

int bcgs_chol(int32_t s, const double* A, int32_t lda, double* R, int32_t ldr, void* workspace,
              size_t ws_bytes, void* stream) {
  if (s < 1 || s > kMaxS || !A || !R || !workspace || lda < s || ldr < s)
    return BCGS_ERR_INVALID_ARG;
  if (ws_bytes < sizeof(DevStatus) || ((uintptr_t)workspace) % 256 != 0) return BCGS_ERR_WORKSPACE;
  DevStatus* st = reinterpret_cast<DevStatus*>(workspace);
  cudaStream_t sm = reinterpret_cast<cudaStream_t>(stream);
  if (launch_reset_status(st, sm) != cudaSuccess) return BCGS_ERR_CUDA;
  return launch_chol(s, A, lda, R, ldr, 1, st, sm) == cudaSuccess ? BCGS_OK : BCGS_ERR_CUDA;
}

// Batched factorization: each problem gets its own slice of the workspace
// (status words at the start) and its kernels run in order on one of 16
// internal lanes forked from, and joined back into, the caller's stream, so
// independent problems overlap on the GPU.  The whole call can be captured
// into one CUDA graph by capturing the caller's stream.
int bcgs_qr_batched_workspace_size(int32_t count, const bcgs_problem* probs, size_t* bytes) {
  if (count < 0 || bytes == nullptr || (count > 0 && probs == nullptr)) return BCGS_ERR_INVALID_ARG;
  size_t total = align256((size_t)count * sizeof(DevStatus));
  for (int i = 0; i < count; ++i) {
    size_t b = 0;
    const bcgs_problem& p = probs[i];
    if (p.engine < 0 || p.engine > 3) return BCGS_ERR_INVALID_ARG;
    const EngineScope es(p.engine);  // the engine decides whether the workspace holds a digit store
    if (bcgs_qr_workspace_size(p.m, p.n, p.s, p.variant, p.precision, &b) != BCGS_OK)
      return BCGS_ERR_INVALID_ARG;
    total += align256(b);
  }
  *bytes = total;
  return BCGS_OK;
}

int bcgs_qr_factor_batched(int32_t count, const bcgs_problem* probs, void* workspace,
                           size_t ws_bytes, void* stream) {
  size_t need = 0;
  int rc = bcgs_qr_batched_workspace_size(count, probs, &need);
  if (rc != BCGS_OK) return rc;
  if (workspace == nullptr || ws_bytes < need || ((uintptr_t)workspace) % 256 != 0)
    return BCGS_ERR_WORKSPACE;
  // every problem is checked before anything is enqueued
  for (int i = 0; i < count; ++i) {
    const bcgs_problem& p = probs[i];
    if (p.X == nullptr || p.ldx < p.m ||
        overlaps(p.X, p.ldx, p.Q, p.ldq, p.m, p.n, p.precision == BCGS_FP32_STORAGE ? 4 : 8))
      return BCGS_ERR_INVALID_ARG;
  }
  cudaStream_t origin = reinterpret_cast<cudaStream_t>(stream);
  BatchStreams* bs = nullptr;
  rc = batch_streams(&bs);
  if (rc != BCGS_OK) return rc;
  // The lanes and events are shared by every caller on this device: calls from
  // several host threads enqueue one after the other (a wait takes the event as
  // recorded when the wait is enqueued, so nothing else needs ordering).
  std::lock_guard<std::mutex> lk(bs->call);
  // Fork: every lane waits for the work already queued on the caller's stream.
  if (cudaEventRecord(bs->fork, origin) != cudaSuccess) return BCGS_ERR_CUDA;
  for (int l = 0; l < kBatchLanes; ++l)
    if (cudaStreamWaitEvent(bs->lane[l], bs->fork, 0) != cudaSuccess) return BCGS_ERR_CUDA;
  // Problems go to lanes largest first (longest-processing-time order), each
  // to the lane with the least work so far; each lane runs its problems in turn.
  int* order = static_cast<int*>(malloc(sizeof(int) * (count > 0 ? count : 1)));
  double* work = static_cast<double*>(malloc(sizeof(double) * (count > 0 ? count : 1)));
  size_t* offs = static_cast<size_t*>(malloc(sizeof(size_t) * (count > 0 ? count : 1)));
  if (!order || !work || !offs) {
    free(order); free(work); free(offs);
    return BCGS_ERR_INVALID_ARG;
  }
  size_t off = align256((size_t)count * sizeof(DevStatus));
  for (int i = 0; i < count; ++i) {
    order[i] = i;
    work[i] = (double)probs[i].m * probs[i].n * probs[i].n;
    offs[i] = off;
    size_t b = 0;
    const EngineScope es(probs[i].engine);
    bcgs_qr_workspace_size(probs[i].m, probs[i].n, probs[i].s, probs[i].variant, probs[i].precision, &b);
    off += align256(b);
  }
  for (int i = 1; i < count; ++i) {  // insertion sort by decreasing work (stable)
    int v = order[i], j = i - 1;
    while (j >= 0 && work[order[j]] < work[v]) { order[j + 1] = order[j]; --j; }
    order[j + 1] = v;
  }
  double load[kBatchLanes] = {0};
  char* ws = reinterpret_cast<char*>(workspace);
  rc = BCGS_OK;
  for (int t = 0; t < count && rc == BCGS_OK; ++t) {
    const int i = order[t];
    int lane = 0;
    for (int l = 1; l < kBatchLanes; ++l)
      if (load[l] < load[lane]) lane = l;
    load[lane] += work[i] + 1e7;  // + a per-problem launch cost
    const bcgs_problem& p = probs[i];
    const EngineScope es(p.engine);
    size_t b = 0;
    bcgs_qr_workspace_size(p.m, p.n, p.s, p.variant, p.precision, &b);
    cudaStream_t ls = bs->lane[lane];
    // no run-ahead: every lane would share this thread's one side stream
    rc = factor_impl(p.m, p.n, p.s, p.variant, p.precision, p.X, p.ldx, p.Q, p.ldq, p.R, p.ldr, ws + offs[i],
                     align256(b), ls, false);
    if (rc == BCGS_OK &&
        cudaMemcpyAsync(ws + (size_t)i * sizeof(DevStatus), ws + offs[i], sizeof(DevStatus),
                        cudaMemcpyDeviceToDevice, ls) != cudaSuccess)
      rc = BCGS_ERR_CUDA;
  }
  free(order); free(work); free(offs);
  // Join: the caller's stream waits for every lane (also on failure, so that
  // nothing enqueued so far is left unordered).
  for (int l = 0; l < kBatchLanes; ++l) {
    if (cudaEventRecord(bs->join[l], bs->lane[l]) != cudaSuccess) return BCGS_ERR_CUDA;
    if (cudaStreamWaitEvent(origin, bs->join[l], 0) != cudaSuccess) return BCGS_ERR_CUDA;
  }
  return rc;
}

int bcgs_qr_batched_status(int32_t count, const void* workspace, void* stream, int32_t* codes,
                           int32_t* fail_blocks) {
  if (count < 0 || workspace == nullptr) return BCGS_ERR_INVALID_ARG;
  cudaStream_t sm = reinterpret_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(sm) != cudaSuccess) return BCGS_ERR_CUDA;
  int first = BCGS_OK;
  const char* ws = reinterpret_cast<const char*>(workspace);
  for (int i = 0; i < count; ++i) {
    int32_t cb[2] = {0, 0};
    if (cudaMemcpy(cb, ws + (size_t)i * sizeof(DevStatus), sizeof(cb), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return BCGS_ERR_CUDA;
    if (codes) codes[i] = cb[0];
    if (fail_blocks) fail_blocks[i] = cb[0] ? cb[1] : 0;
    if (first == BCGS_OK && cb[0] != 0) first = cb[0];
  }
  return first;
}

}  // extern "C"
