// Tall-skinny Gram reduction C = [A_1 ... ]^T [B_1 ...]: one synchronization
// point of the paper (Sec. 3: the product of two tall-thin matrices is the only
// operation with global communication; Alg. 2's sync step computes
// [Q_k U_{k+1}]^T [U_{k+1} X_{k+2}] and X_{k+2}^T X_{k+2}).
//
// GB300 form: the m rows are cut into a fixed number of chunks (a function of m
// only); one CTA streams one chunk through shared memory and accumulates its
// partial product in FP64 registers; a second kernel adds the chunk partials in
// chunk order.  The result is therefore bitwise reproducible for a given shape.
#include "bcgs_internal.cuh"

namespace bcgs {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxOutPerThread = 64;
constexpr int kMaxOutPerCta = kThreads * kMaxOutPerThread;  // 16384

template <typename T>
__device__ __forceinline__ double ld_elem(const void* base, int64_t idx) {
  return (double)__ldg(reinterpret_cast<const T*>(base) + idx);
}

struct ColMap {
  // Prefix column offsets of the segments (exclusive), for a column -> segment lookup.
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

// grid = (nchunks, ngroups); group g owns A columns [g*na_g, min((g+1)*na_g, na)).
template <typename T, int NPT>
__global__ void __launch_bounds__(kThreads)
gram_partial_kernel(GramDesc d, ColMap cm, int32_t na_g, int32_t tr, double* __restrict__ partial,
                    const DevStatus* st) {
  if (failed(st)) return;
  extern __shared__ double smem[];
  const int chunk = blockIdx.x;
  const int g = blockIdx.y;
  const int col0 = g * na_g;
  const int ncol_a = min(na_g, d.na - col0);
  const int nb = d.nb;
  const int ldas = ncol_a + 1;  // odd strides keep the row-major tiles conflict-light
  const int ldbs = nb + 1;
  double* As = smem;                 // [tr][ldas]
  double* Bs = smem + tr * ldas;     // [tr][ldbs]
  const int64_t r_begin = (int64_t)chunk * d.chunk_rows;
  const int64_t r_end = min(r_begin + d.chunk_rows, d.m);
  const int nout = ncol_a * nb;

  double acc[NPT];
#pragma unroll
  for (int u = 0; u < NPT; ++u) acc[u] = 0.0;

  const int tile_elems = tr * (ncol_a + nb);
  for (int64_t r0 = r_begin; r0 < r_end; r0 += tr) {
    __syncthreads();
    for (int e = threadIdx.x; e < tile_elems; e += kThreads) {
      const int col = e / tr;
      const int r = e - col * tr;
      const int64_t row = r0 + r;
      double v = 0.0;
      if (col < ncol_a) {
        const int ca = col0 + col;
        const int sg = find_seg<kMaxSegA>(cm.a_off, d.nsa, ca);
        if (row < r_end) v = ld_elem<T>(d.a[sg].p, row + (int64_t)(ca - cm.a_off[sg]) * d.a[sg].ld);
        As[r * ldas + col] = v;
      } else {
        const int cb = col - ncol_a;
        const int sg = find_seg<kMaxSegB>(cm.b_off, d.nsb, cb);
        if (row < r_end) v = ld_elem<T>(d.b[sg].p, row + (int64_t)(cb - cm.b_off[sg]) * d.b[sg].ld);
        Bs[r * ldbs + cb] = v;
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NPT; ++u) {
      const int o = threadIdx.x + u * kThreads;
      if (o < nout) {
        const int i = o / nb;
        const int j = o - i * nb;
        double a = acc[u];
        for (int r = 0; r < tr; ++r) a = fma(As[r * ldas + i], Bs[r * ldbs + j], a);
        acc[u] = a;
      }
    }
  }
  // partial layout: [chunk][i (global A column)][j]
  double* out = partial + (size_t)chunk * ((size_t)d.na * nb) + (size_t)col0 * nb;
#pragma unroll
  for (int u = 0; u < NPT; ++u) {
    const int o = threadIdx.x + u * kThreads;
    if (o < nout) out[o] = acc[u];
  }
}

// G[i + j*ldg] = sum over chunks in a fixed order that depends on nchunks only:
// warp w of a CTA adds the chunks c = w, w + 8, ... in turn, then the eight
// warp sums are added as a fixed tree.  One CTA per 32 consecutive outputs (each
// warp load is 256 contiguous bytes of one chunk), so the FP64 additions spread
// over many SMs instead of one long chain per output.
constexpr int kReduceWarps = 8;
__global__ void __launch_bounds__(32 * kReduceWarps)
gram_reduce_kernel(const double* __restrict__ partial, int32_t nchunks, int32_t na, int32_t nb,
                   double* __restrict__ G, int32_t ldg, const DevStatus* st) {
  if (failed(st)) return;  // the same for every thread: nothing sets it during this kernel
  __shared__ double part[kReduceWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nout = na * nb;
  const int o = blockIdx.x * 32 + lane;
  double sum = 0.0;
  if (o < nout)
    for (int c = w; c < nchunks; c += kReduceWarps) sum += __ldcg(partial + (size_t)c * nout + o);
  part[w][lane] = sum;
  __syncthreads();
  if (w == 0 && o < nout) {
    const double t = ((part[0][lane] + part[1][lane]) + (part[2][lane] + part[3][lane])) +
                     ((part[4][lane] + part[5][lane]) + (part[6][lane] + part[7][lane]));
    const int i = o / nb;
    const int j = o - i * nb;
    G[i + (size_t)j * ldg] = t;
  }
}

// G = the sum over ranks, in rank order, of the gathered copies of the local
// Grams (rank-major; each column-major with leading dimension ld over nb
// columns): the cross-rank part of one synchronization of the row-partitioned
// form (Sec. 3: each process holds a block of rows and the Gram is summed over
// the processes).  A fixed order makes the sum, and so the replicated tail
// after it, the same on every rank and on every run.
__global__ void rank_sum_kernel(const double* __restrict__ recv, int32_t nranks, int32_t na, int32_t nb,
                                int32_t ld, double* __restrict__ G, const DevStatus* st) {
  if (failed(st)) return;
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= na * nb) return;
  const int i = o % na, j = o / na;
  const size_t per = (size_t)ld * nb;
  double sum = recv[i + (size_t)j * ld];
  for (int r = 1; r < nranks; ++r) sum += recv[(size_t)r * per + i + (size_t)j * ld];
  G[i + (size_t)j * ld] = sum;
}

// p[0 .. n) = NaN when the factorization has failed: a rank that stopped
// working sends NaN, so the failure reaches every rank through the next sum
// instead of a stale buffer being added in.
__global__ void poison_kernel(double* p, int64_t n, const DevStatus* st) {
  if (!failed(st)) return;
  for (int64_t e = threadIdx.x + (int64_t)blockIdx.x * blockDim.x; e < n; e += (int64_t)blockDim.x * gridDim.x)
    p[e] = __longlong_as_double(0x7FF8000000000000LL);
}

template <typename T>
cudaError_t launch_gram_t(const GramDesc& d, double* partial, double* G, int ldg, DevStatus* st,
                          cudaStream_t stream) {
  ColMap cm;
  cm.a_off[0] = 0;
  for (int k = 0; k < kMaxSegA; ++k) cm.a_off[k + 1] = cm.a_off[k] + (k < d.nsa ? d.a[k].ncols : 0);
  cm.b_off[0] = 0;
  for (int k = 0; k < kMaxSegB; ++k) cm.b_off[k + 1] = cm.b_off[k] + (k < d.nsb ? d.b[k].ncols : 0);
  // Columns of A per CTA group so that one CTA holds at most kMaxOutPerCta outputs.
  int na_g = d.na;
  if ((int64_t)d.na * d.nb > kMaxOutPerCta) na_g = kMaxOutPerCta / d.nb;
  const int ngroups = (int)ceil_div(d.na, na_g);
  const int ncol_a = na_g;
  // Rows per shared-memory tile: as many of 16 / 8 / 4 as fit in 160 KB.
  int tr = 16;
  auto smem_bytes = [&](int t) { return (size_t)t * ((ncol_a + 1) + (d.nb + 1)) * sizeof(double); };
  while (tr > 4 && smem_bytes(tr) > 160 * 1024) tr /= 2;
  const size_t smem = smem_bytes(tr);
  const int nout = ncol_a * d.nb;
  const int npt_need = (nout + kThreads - 1) / kThreads;
  dim3 grid(d.nchunks, ngroups);
  const double esz = sizeof(T);
  const int slot = prof_begin(stream);
#define BCGS_GRAM_CASE(NPT)                                                                    \
  if (npt_need <= NPT) {                                                                       \
    auto kern = gram_partial_kernel<T, NPT>;                                                   \
    cudaError_t e = ensure_dyn_smem(kern, smem);                                               \
    if (e != cudaSuccess) return e;                                                            \
    kern<<<grid, kThreads, smem, stream>>>(d, cm, na_g, tr, partial, st);                      \
  } else
  BCGS_GRAM_CASE(1) BCGS_GRAM_CASE(2) BCGS_GRAM_CASE(4) BCGS_GRAM_CASE(8) BCGS_GRAM_CASE(16)
  BCGS_GRAM_CASE(32) BCGS_GRAM_CASE(64) { return cudaErrorInvalidValue; }
#undef BCGS_GRAM_CASE
  prof_end(slot, kProfGramPartial, stream, 2.0 * (double)d.m * d.na * d.nb,
           (double)d.m * (d.na + d.nb) * esz + (double)d.nchunks * d.na * d.nb * 8.0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  note_launch(1);
  return launch_gram_reduce(partial, d.nchunks, d.na, d.nb, G, ldg, st, stream);
}

}  // namespace

cudaError_t launch_gram_reduce(const double* partial, int32_t nchunks, int32_t na, int32_t nb,
                               double* G, int32_t ldg, const DevStatus* st, cudaStream_t stream) {
  const int nout_all = na * nb;
  const int slot2 = prof_begin(stream);
  gram_reduce_kernel<<<(nout_all + 31) / 32, 32 * kReduceWarps, 0, stream>>>(partial, nchunks, na, nb, G, ldg,
                                                                              st);
  prof_end(slot2, kProfGramReduce, stream, (double)nchunks * nout_all,
           (double)nchunks * nout_all * 8.0 + nout_all * 8.0);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_rank_sum(const double* recv, int32_t nranks, int32_t na, int32_t nb, int32_t ld, double* G,
                            const DevStatus* st, cudaStream_t stream) {
  const int n = na * nb;
  if (n <= 0) return cudaSuccess;
  rank_sum_kernel<<<(n + 255) / 256, 256, 0, stream>>>(recv, nranks, na, nb, ld, G, st);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_poison_if_failed(double* p, int64_t n, const DevStatus* st, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  int64_t grid = (n + 255) / 256;
  if (grid > 256) grid = 256;
  poison_kernel<<<(unsigned)grid, 256, 0, stream>>>(p, n, st);
  note_launch(1);
  return cudaGetLastError();
}

void gram_partition(int64_t m, int64_t* chunk_rows, int32_t* nchunks) {
  // About two chunks per SM of a 152-SM GB300 for large m; at least 64 rows each.
  const int64_t target = 304;
  int64_t cr = round_up(ceil_div(m, target), 16);
  if (cr < 64) cr = 64;
  *chunk_rows = cr;
  *nchunks = (int32_t)ceil_div(m, cr);
}

size_t gram_partial_doubles(int64_t m, int32_t na, int32_t nb) {
  int64_t cr;
  int32_t nc;
  gram_partition(m, &cr, &nc);
  return (size_t)nc * (size_t)na * (size_t)nb;
}

cudaError_t launch_gram(const GramDesc& d, double* partial, double* G, int ldg, DevStatus* st,
                        cudaStream_t stream) {
  if (d.na <= 0 || d.nb <= 0) return cudaSuccess;
  const bool f32 = d.a[0].fp32 != 0;
  return f32 ? launch_gram_t<float>(d, partial, G, ldg, st, stream)
             : launch_gram_t<double>(d, partial, G, ldg, st, stream);
}

}  // namespace bcgs
