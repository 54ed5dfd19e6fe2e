// TSQR: the unconditionally stable intraorthogonalization of an m x s block
// (Sec. 1; [Q_1, R_11] = TSQR(X_1) in Alg. 1 and Alg. 2; BCGSI+P-2S and BCGSI+
// use it for every block).  The paper took TSQR from Trilinos (Sec. 4) and fixes
// no tree; this is a fixed-shape tree on one GPU:
//
//   level 0     one CTA per row tile of mt rows: Householder QR in shared
//               memory, reflectors kept in the workspace, the s x s R factor
//               written into its parent's stacked matrix;
//   level l>=1  one CTA per node: Householder QR of `fan` stacked R factors;
//   root        diag(R) made >= 0 (signs D), R written out;
//   apply       top-down, each node forms H [B; 0] for the coefficient block B
//               it receives from its parent (the root starts from B = D), and
//               the leaves write the explicit Q rows.
//
// The Householder step per column follows the oracle's convention
// (beta = -sign(a_jj) ||a_j||, v_j = 1, tau = (beta - a_jj) / beta), so the
// sign-normalized factors agree with a plain Householder QR up to rounding.
#include <type_traits>

#include "bcgs_internal.cuh"
#include "dfloat.cuh"

namespace bcgs {

namespace {

constexpr int kTsqrThreads = 256;
constexpr int kWarps = kTsqrThreads / 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum over r = r0, r0 + 32, ... < rows of a[r] b[r], in four interleaved
// accumulators (a fixed order: the result depends on the shape only)
__device__ __forceinline__ double dot4(const double* a, const double* b, int r0, int rows) {
  double w0 = 0.0, w1 = 0.0, w2 = 0.0, w3 = 0.0;
  int r = r0;
  for (; r + 96 < rows; r += 128) {
    w0 = fma(a[r], b[r], w0);
    w1 = fma(a[r + 32], b[r + 32], w1);
    w2 = fma(a[r + 64], b[r + 64], w2);
    w3 = fma(a[r + 96], b[r + 96], w3);
  }
  for (; r < rows; r += 32) w0 = fma(a[r], b[r], w0);
  return (w0 + w1) + (w2 + w3);
}

// The sums over r = r0, r0 + 32, ... < rows of a[r] b0[r] and a[r] b1[r] (b1
// may be null: its sum is 0), with two interleaved accumulators each, then one
// warp reduce-scatter for both (lanes 0..15 finish b0's, 16..31 b1's): five FP64
// additions per lane for the pair instead of five per column, on GB300's scarce
// FP64 pipe.  Every lane gets both sums; the order depends on the shape only.
__device__ __forceinline__ void dot2_pair(const double* a, const double* b0, const double* b1, int r0, int rows,
                                          int lane, double& s0, double& s1) {
  double p0 = 0.0, q0 = 0.0, p1 = 0.0, q1 = 0.0;
  int r = r0;
  if (b1 != nullptr) {
    for (; r + 32 < rows; r += 64) {
      const double x = a[r], y = a[r + 32];
      p0 = fma(x, b0[r], p0);
      q0 = fma(y, b0[r + 32], q0);
      p1 = fma(x, b1[r], p1);
      q1 = fma(y, b1[r + 32], q1);
    }
    for (; r < rows; r += 32) {
      const double x = a[r];
      p0 = fma(x, b0[r], p0);
      p1 = fma(x, b1[r], p1);
    }
  } else {
    for (; r + 32 < rows; r += 64) {
      p0 = fma(a[r], b0[r], p0);
      q0 = fma(a[r + 32], b0[r + 32], q0);
    }
    for (; r < rows; r += 32) p0 = fma(a[r], b0[r], p0);
  }
  p0 += q0;
  p1 += q1;
  const bool upper = lane >= 16;
  double keep = upper ? p1 : p0;
  const double give = upper ? p0 : p1;
  keep += __shfl_xor_sync(0xffffffffu, give, 16);
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o);
  s0 = __shfl_sync(0xffffffffu, keep, 0);
  s1 = __shfl_sync(0xffffffffu, keep, 16);
}

// In-place Householder QR of the rows x s column-major matrix A (ld = rows) in
// shared memory.  On return A holds R in its upper triangle and v_j below the
// diagonal (v_j has an implicit 1 at row j); tau[j] the reflector scalars.
__device__ void block_householder(double* A, int rows, int s, double* tau) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  // reflector of column j by one warp: v_j below the diagonal, beta on it, tau[j]
  auto reflect = [&](int j) {
    double* aj = A + (size_t)j * rows;
    const double sum = warp_sum(dot4(aj, aj, j + 1 + lane, rows));
    const double x0 = aj[j];
    const double alpha = sqrt(fma(x0, x0, sum));
    double t = 0.0, beta = 0.0, denom = 1.0;
    if (alpha != 0.0) {
      beta = x0 >= 0.0 ? -alpha : alpha;
      denom = x0 - beta;
      t = (beta - x0) / beta;
    }
    if (alpha != 0.0) {
      const double rden = 1.0 / denom;  // one FP64 division per column
      for (int r = j + 1 + lane; r < rows; r += 32) aj[r] *= rden;
    }
    __syncwarp();
    if (lane == 0) {
      tau[j] = t;
      if (alpha != 0.0) aj[j] = beta;
    }
  };
  if (warp == 0) reflect(0);
  __syncthreads();
  for (int j = 0; j < s; ++j) {
    // reflector j is final; apply it to the columns l > j.  Warp 0 takes column
    // j + 1 first and forms reflector j + 1 at once (look-ahead), while the other
    // warps finish their columns with reflector j: one barrier per column.
    // Each warp takes a pair of columns (l0, l0 + 1), sharing the loads of v_j and
    // one reduction (dot2_pair).
    const double* aj = A + (size_t)j * rows;
    const double t = tau[j];
    const int npairs = (s - j) / 2;  // ceil((s - j - 1) / 2)
    for (int pr = warp; pr < npairs; pr += kWarps) {
      const int l0 = j + 1 + 2 * pr;
      double* a0 = A + (size_t)l0 * rows;
      double* a1 = l0 + 1 < s ? a0 + rows : nullptr;
      if (t != 0.0) {
        double s0, s1;
        dot2_pair(aj, a0, a1, j + 1 + lane, rows, lane, s0, s1);
        const double w0 = (s0 + a0[j]) * t;
        const double w1 = a1 != nullptr ? (s1 + a1[j]) * t : 0.0;
        __syncwarp();  // every lane has read a0[j], a1[j] before lane 0 updates them
        if (lane == 0) {
          a0[j] -= w0;
          if (a1 != nullptr) a1[j] -= w1;
        }
        if (a1 != nullptr) {
          for (int r = j + 1 + lane; r < rows; r += 32) {
            const double v = aj[r];
            a0[r] = fma(-v, w0, a0[r]);
            a1[r] = fma(-v, w1, a1[r]);
          }
        } else {
          for (int r = j + 1 + lane; r < rows; r += 32) a0[r] = fma(-aj[r], w0, a0[r]);
        }
        __syncwarp();
      }
      if (l0 == j + 1) reflect(l0);
    }
    __syncthreads();
  }
}

// E <- H_0 H_1 ... H_{s-1} E for reflectors stored as by block_householder
// (pairs of columns of E per warp, as there).
__device__ void block_apply_q(const double* V, const double* tau, double* E, int rows, int s) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int nwarps = blockDim.x / 32;
  const int npairs = (s + 1) / 2;
  for (int j = s - 1; j >= 0; --j) {
    const double t = tau[j];
    if (t != 0.0) {
      const double* vj = V + (size_t)j * rows;
      for (int pr = warp; pr < npairs; pr += nwarps) {
        double* e0 = E + (size_t)(2 * pr) * rows;
        double* e1 = 2 * pr + 1 < s ? e0 + rows : nullptr;
        double s0, s1;
        dot2_pair(vj, e0, e1, j + 1 + lane, rows, lane, s0, s1);
        const double w0 = (s0 + e0[j]) * t;
        const double w1 = e1 != nullptr ? (s1 + e1[j]) * t : 0.0;
        __syncwarp();
        if (lane == 0) {
          e0[j] -= w0;
          if (e1 != nullptr) e1[j] -= w1;
        }
        if (e1 != nullptr) {
          for (int r = j + 1 + lane; r < rows; r += 32) {
            const double v = vj[r];
            e0[r] = fma(-v, w0, e0[r]);
            e1[r] = fma(-v, w1, e1[r]);
          }
        } else {
          for (int r = j + 1 + lane; r < rows; r += 32) e0[r] = fma(-vj[r], w0, e0[r]);
        }
        __syncwarp();
      }
    }
    __syncthreads();
  }
}

// Root: make diag(R) >= 0 and write R (s x s, ldr) and the signs D into bout (s x s).
__device__ void finish_root(const double* A, int rows, int s, double* R, int ldr, double* bout,
                            DevStatus* st, int block) {
  __shared__ int bad_rank, bad_fin;
  if (threadIdx.x == 0) { bad_rank = 0; bad_fin = 0; }
  __syncthreads();
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    const int i = e % s, j = e / s;
    const double d = A[i + (size_t)i * rows] < 0.0 ? -1.0 : 1.0;
    double v = i <= j ? d * A[i + (size_t)j * rows] : 0.0;
    R[i + (size_t)j * ldr] = v;
    bout[i + (size_t)j * s] = (i == j) ? d : 0.0;
    if (!isfinite(v)) bad_fin = 1;
    if (i == j && v == 0.0) bad_rank = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (bad_fin) set_failure(st, BCGS_ERR_NONFINITE, block);
    else if (bad_rank) set_failure(st, BCGS_ERR_RANK_DEFICIENT, block);
  }
}

template <typename T>
__global__ void __launch_bounds__(kTsqrThreads)
tsqr_leaf_factor(TsqrPlan p, Seg a, double* work, double* R, int32_t ldr, DevStatus* st,
                 int32_t block) {
  if (failed(st)) return;
  extern __shared__ double sm[];
  __shared__ double tau[64];
  const int mt = p.mt, s = p.s;
  double* A = sm;  // mt x s
  const int t = blockIdx.x;
  const int64_t row0 = (int64_t)t * mt;
  const int rows_here = (int)(p.m - row0 < (int64_t)mt ? p.m - row0 : (int64_t)mt);
  const T* src = reinterpret_cast<const T*>(a.p);
  for (int e = threadIdx.x; e < mt * s; e += kTsqrThreads) {
    const int r = e % mt, j = e / mt;
    A[e] = r < rows_here ? (double)src[row0 + r + (int64_t)j * a.ld] : 0.0;
  }
  __syncthreads();
  block_householder(A, mt, s, tau);
  double* H = work + p.off_h + (size_t)t * mt * s;
  for (int e = threadIdx.x; e < mt * s; e += kTsqrThreads) H[e] = A[e];
  double* tg = work + p.off_tau[0] + (size_t)t * s;
  for (int j = threadIdx.x; j < s; j += kTsqrThreads) tg[j] = tau[j];
  // WY triangle of the leaf: H_0 ... H_{s-1} = I - V T V^T (forward, columnwise)
  {
    double* VV = A + (size_t)mt * s;  // s x s: (V^T V)_{ij} for i < j
    double* Tl = VV + (size_t)s * s;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    // (V^T V)_ij = v_i[j] + sum_{r > j} v_i[r] v_j[r]  (v_j[j] = 1, v_j[r < j] = 0):
    // for each j the entries i < j in pairs (i, i + 1), one task per warp
    int task = 0;
    for (int j = 1; j < s; ++j) {
      const double* vj = A + (size_t)j * mt;
      for (int i = 0; i < j; i += 2, ++task) {
        if (task % kWarps != warp) continue;
        const double* vi = A + (size_t)i * mt;
        const double* vi1 = i + 1 < j ? vi + mt : nullptr;
        double d0, d1;
        dot2_pair(vj, vi, vi1, j + 1 + lane, mt, lane, d0, d1);
        if (lane == 0) {
          VV[i + (size_t)j * s] = d0 + vi[j];
          if (vi1 != nullptr) VV[i + 1 + (size_t)j * s] = d1 + vi1[j];
        }
      }
    }
    __syncthreads();
    // T(i, j) = -tau_j sum_{l = i}^{j-1} T(i, l) (V^T V)(l, j), T(j, j) = tau_j:
    // column by column, the rows of a column in parallel
    for (int j = 0; j < s; ++j) {
      for (int i = threadIdx.x; i < s; i += kTsqrThreads) {
        double x = 0.0;
        if (i < j)
          for (int l = i; l < j; ++l) x = fma(Tl[i + (size_t)l * s], VV[l + (size_t)j * s], x);
        Tl[i + (size_t)j * s] = i < j ? -tau[j] * x : (i == j ? tau[j] : 0.0);
      }
      __syncthreads();
    }
    double* tw = work + p.off_t0 + (size_t)t * s * s;
    for (int e = threadIdx.x; e < s * s; e += kTsqrThreads) tw[e] = Tl[e];
  }
  if (p.nlevels == 1) {
    finish_root(A, mt, s, R, ldr, work + p.off_b[0], st, block);
    return;
  }
  // R_t -> parent's stacked matrix, rows [(t % fan) s, +s)
  const int fan = p.fan, ldp = fan * s;
  double* P = work + p.off_lvl[1] + (size_t)(t / fan) * ldp * s;
  const int rbase = (t % fan) * s;
  for (int e = threadIdx.x; e < s * s; e += kTsqrThreads) {
    const int i = e % s, j = e / s;
    P[rbase + i + (size_t)j * ldp] = i <= j ? A[i + (size_t)j * mt] : 0.0;
  }
}

__global__ void __launch_bounds__(kTsqrThreads)
tsqr_node_factor(TsqrPlan p, int32_t level, double* work, double* R, int32_t ldr, DevStatus* st,
                 int32_t block) {
  if (failed(st)) return;
  extern __shared__ double sm[];
  __shared__ double tau[64];
  const int s = p.s, fan = p.fan, rows = fan * s;
  const int n = blockIdx.x;
  const int nchild = min(fan, p.nodes[level - 1] - n * fan);
  // only the nchild stacked factors: the rows past them are zero and would
  // change nothing but the work (compact in shared memory, ld = re)
  const int re = nchild * s;
  double* A = sm;
  double* G = work + p.off_lvl[level] + (size_t)n * rows * s;
  for (int e = threadIdx.x; e < re * s; e += kTsqrThreads) {
    const int r = e % re, j = e / re;
    A[e] = G[r + (size_t)j * rows];
  }
  __syncthreads();
  block_householder(A, re, s, tau);
  for (int e = threadIdx.x; e < re * s; e += kTsqrThreads) {
    const int r = e % re, j = e / re;
    G[r + (size_t)j * rows] = A[e];
  }
  double* tg = work + p.off_tau[level] + (size_t)n * s;
  for (int j = threadIdx.x; j < s; j += kTsqrThreads) tg[j] = tau[j];
  if (level == p.nlevels - 1) {
    finish_root(A, re, s, R, ldr, work + p.off_b[level], st, block);
    return;
  }
  double* P = work + p.off_lvl[level + 1] + (size_t)(n / fan) * rows * s;
  const int rbase = (n % fan) * s;
  for (int e = threadIdx.x; e < s * s; e += kTsqrThreads) {
    const int i = e % s, j = e / s;
    P[rbase + i + (size_t)j * rows] = i <= j ? A[i + (size_t)j * re] : 0.0;
  }
}

__global__ void __launch_bounds__(kTsqrThreads)
tsqr_node_apply(TsqrPlan p, int32_t level, double* work, const DevStatus* st) {
  if (failed(st)) return;
  extern __shared__ double sm[];
  __shared__ double tau[64];
  const int s = p.s, fan = p.fan, rows = fan * s;
  const int n = blockIdx.x;
  const int nchild = min(fan, p.nodes[level - 1] - n * fan);
  const int re = nchild * s;  // the rows tsqr_node_factor factored (compact, ld = re)
  double* V = sm;
  double* E = sm + (size_t)re * s;
  const double* G = work + p.off_lvl[level] + (size_t)n * rows * s;
  const double* B = work + p.off_b[level] + (size_t)n * s * s;
  for (int e = threadIdx.x; e < re * s; e += kTsqrThreads) {
    const int r = e % re, j = e / re;
    V[e] = G[r + (size_t)j * rows];
    E[e] = r < s ? B[r + (size_t)j * s] : 0.0;
  }
  for (int j = threadIdx.x; j < s; j += kTsqrThreads) tau[j] = work[p.off_tau[level] + (size_t)n * s + j];
  __syncthreads();
  block_apply_q(V, tau, E, re, s);
  for (int e = threadIdx.x; e < nchild * s * s; e += kTsqrThreads) {
    const int g = e / (s * s), rem = e % (s * s);
    const int i = rem % s, j = rem / s;
    work[p.off_b[level - 1] + (size_t)(n * fan + g) * s * s + i + (size_t)j * s] =
        E[g * s + i + (size_t)j * re];
  }
}

template <typename T>
__global__ void __launch_bounds__(kTsqrThreads)
tsqr_leaf_apply(TsqrPlan p, const double* work, void* q, int64_t ldq, const DevStatus* st, MaxOut qmax) {
  if (failed(st)) return;
  extern __shared__ double sm[];
  const int mt = p.mt, s = p.s;
  const int t = blockIdx.x;
  // E = H_0 ... H_{s-1} [B; 0] = [B; 0] - V (T (V_top^T B))  (compact WY: one row-wise
  // product instead of s reflector sweeps with reductions)
  double* V = sm;                     // mt x s (reflectors below the diagonal)
  double* Bs = V + (size_t)mt * s;    // s x s coefficient block from the parent
  double* Tl = Bs + (size_t)s * s;    // s x s WY triangle
  double* W = Tl + (size_t)s * s;     // s x s: V_top^T B, then M = T W
  double* E = W + (size_t)s * s;      // mt x s output (for the maxima)
  const double* H = work + p.off_h + (size_t)t * mt * s;
  const double* B = work + p.off_b[0] + (size_t)t * s * s;
  const double* Tg = work + p.off_t0 + (size_t)t * s * s;
  for (int e = threadIdx.x; e < mt * s; e += kTsqrThreads) V[e] = H[e];
  for (int e = threadIdx.x; e < s * s; e += kTsqrThreads) {
    Bs[e] = B[e];
    Tl[e] = Tg[e];
  }
  __syncthreads();
  // W = V_top^T B: V_top(i, l) = 1 (i = l), V(i, l) (i > l), 0 (i < l)
  for (int e = threadIdx.x; e < s * s; e += kTsqrThreads) {
    const int l = e % s, c = e / s;
    double x = Bs[l + (size_t)c * s];
    for (int i = l + 1; i < s; ++i) x = fma(V[i + (size_t)l * mt], Bs[i + (size_t)c * s], x);
    E[e] = x;  // scratch until W is final
  }
  __syncthreads();
  // M = T W (T upper triangular)
  for (int e = threadIdx.x; e < s * s; e += kTsqrThreads) {
    const int l = e % s, c = e / s;
    double x = 0.0;
    for (int i = l; i < s; ++i) x = fma(Tl[l + (size_t)i * s], E[i + (size_t)c * s], x);
    W[e] = x;
  }
  __syncthreads();
  const int64_t row0 = (int64_t)t * mt;
  const int rows_here = (int)(p.m - row0 < (int64_t)mt ? p.m - row0 : (int64_t)mt);
  T* dst = reinterpret_cast<T*>(q);
  for (int r = threadIdx.x; r < mt; r += kTsqrThreads) {
    for (int c0 = 0; c0 < s; c0 += 16) {
      const int nc = s - c0 < 16 ? s - c0 : 16;
      double e[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) e[c] = (c < nc && r < s) ? Bs[r + (size_t)(c0 + c) * s] : 0.0;
      const int lmax = r < s ? r + 1 : s;  // V(r, l) = 0 for l > r
      for (int l = 0; l < lmax; ++l) {
        const double v = l == r ? 1.0 : V[r + (size_t)l * mt];
#pragma unroll
        for (int c = 0; c < 16; ++c)
          if (c < nc) e[c] = fma(-v, W[l + (size_t)(c0 + c) * s], e[c]);
      }
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c < nc) {
          E[r + (size_t)(c0 + c) * mt] = e[c];
          if (r < rows_here) dst[row0 + r + (int64_t)(c0 + c) * ldq] = (T)e[c];
        }
    }
  }
  __syncthreads();
  // maxima of the written Q block (of the stored values)
  if (qmax.col != nullptr) {
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int j = warp; j < s; j += kWarps) {
      unsigned long long mx = 0ull;
      for (int r = lane; r < rows_here; r += 32) mx = umax64(mx, abs_bits64((double)(T)E[r + (size_t)j * mt]));
      warp_max_to(mx, qmax.col + j);
    }
  }
  if (qmax.row != nullptr) {
    for (int r = threadIdx.x; r < rows_here; r += kTsqrThreads) {
      unsigned long long mx = 0ull;
      for (int j = 0; j < s; ++j) mx = umax64(mx, abs_bits64((double)(T)E[r + (size_t)j * mt]));
      qmax.row[row0 + r] = umax64(qmax.row[row0 + r], mx);
    }
  }
}

// The ranks' s x s R factors, gathered rank-major (each column-major, ld s),
// stacked into one (nranks s) x s column-major matrix: the cross-rank level of
// the row-partitioned TSQR (Sec. 3, Sec. 4: TSQR reduces the R factors of the
// row blocks).
__global__ void stack_r_kernel(const double* __restrict__ recv, int32_t nranks, int32_t s, double* __restrict__ out,
                               const DevStatus* st) {
  if (failed(st)) return;
  const int ld = nranks * s;
  for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < nranks * s * s; e += blockDim.x * gridDim.x) {
    const int r = e / (s * s), rem = e - r * s * s, i = rem % s, j = rem / s;
    out[(r * s + i) + (size_t)j * ld] = recv[e];
  }
}

// W = A B, A m x s (storage type T, lda), B s x s FP64 (ldb), W m x s (T, ldw):
// one thread per row, B in shared memory; the maxima of the stored W.  Used to
// turn a rank's local TSQR factor into its rows of the global Q (the local Q
// times the rank's s x s block of the stacked factor's Q).
template <typename T>
__global__ void __launch_bounds__(256) rows_times_small_kernel(int64_t m, int32_t s, const T* __restrict__ A,
                                                               int64_t lda, const double* __restrict__ B,
                                                               int32_t ldb, T* __restrict__ W, int64_t ldw,
                                                               MaxOut wmax, const DevStatus* st) {
  if (failed(st)) return;
  __shared__ double Bs[64 * 64];
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) Bs[e] = B[(e % s) + (size_t)(e / s) * ldb];
  __syncthreads();
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = r < m;
  unsigned long long rmax = 0ull;
  for (int c0 = 0; c0 < s; c0 += 16) {
    const int nc = s - c0 < 16 ? s - c0 : 16;
    double e[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) e[c] = 0.0;
    if (live)
      for (int l = 0; l < s; ++l) {
        const double a = (double)A[r + (int64_t)l * lda];
#pragma unroll
        for (int c = 0; c < 16; ++c)
          if (c < nc) e[c] = fma(a, Bs[l + (c0 + c) * s], e[c]);
      }
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      if (c >= nc) break;
      const T v = (T)e[c];
      if (live) W[r + (int64_t)(c0 + c) * ldw] = v;
      const unsigned long long b = live ? abs_bits64((double)v) : 0ull;
      rmax = umax64(rmax, b);
      if (wmax.col != nullptr) warp_max_to(b, wmax.col + c0 + c);
    }
  }
  if (live && wmax.row != nullptr) wmax.row[r] = umax64(wmax.row[r], rmax);
}

// ------------------------------------------------------------ double-float tiles
// FP32-storage blocks: the tile arithmetic of the leaves (the column updates,
// V^T V and the explicit-Q product) runs in double-float (dfloat.cuh).  Column
// norms, the reflector scalars, the WY triangle and the tree levels stay FP64;
// the column norms, computed in FP64, do not overflow float's range.
// dot2_pair in double-float: the sums of a[r] b0[r] and a[r] b1[r] (b1 may be
// null), one accumulator each, then one warp reduce-scatter for both.
__device__ __forceinline__ void dot2_pair_df(const df* a, const df* b0, const df* b1, int r0, int rows, int lane,
                                             df& s0, df& s1) {
  df p0{0.f, 0.f}, p1{0.f, 0.f};
  if (b1 != nullptr) {
    for (int r = r0; r < rows; r += 32) {
      const df x = a[r];
      p0 = df_fma(x, b0[r], p0);
      p1 = df_fma(x, b1[r], p1);
    }
  } else {
    for (int r = r0; r < rows; r += 32) p0 = df_fma(a[r], b0[r], p0);
  }
  const bool upper = lane >= 16;
  df keep = upper ? p1 : p0;
  const df give = upper ? p0 : p1;
  keep = df_add(keep, df{__shfl_xor_sync(0xffffffffu, give.hi, 16), __shfl_xor_sync(0xffffffffu, give.lo, 16)});
#pragma unroll
  for (int o = 8; o > 0; o >>= 1)
    keep = df_add(keep, df{__shfl_xor_sync(0xffffffffu, keep.hi, o), __shfl_xor_sync(0xffffffffu, keep.lo, o)});
  s0 = df{__shfl_sync(0xffffffffu, keep.hi, 0), __shfl_sync(0xffffffffu, keep.lo, 0)};
  s1 = df{__shfl_sync(0xffffffffu, keep.hi, 16), __shfl_sync(0xffffffffu, keep.lo, 16)};
}

// block_householder in double-float (the same steps, look-ahead and barriers);
// the column's sum of squares, beta, tau and 1 / (x0 - beta) in FP64.
__device__ void block_householder_df(df* A, int rows, int s, double* tau) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int nwarps = blockDim.x / 32;
  auto reflect = [&](int j) {
    df* aj = A + (size_t)j * rows;
    double ssq = 0.0;
    for (int r = j + 1 + lane; r < rows; r += 32) {
      const double v = df_dbl(aj[r]);
      ssq = fma(v, v, ssq);
    }
    const double sum = warp_sum(ssq);
    const double x0 = df_dbl(aj[j]);
    const double alpha = sqrt(fma(x0, x0, sum));
    double t = 0.0, beta = 0.0, denom = 1.0;
    if (alpha != 0.0) {
      beta = x0 >= 0.0 ? -alpha : alpha;
      denom = x0 - beta;
      t = (beta - x0) / beta;
    }
    if (alpha != 0.0) {
      const df rden = df_from(1.0 / denom);
      for (int r = j + 1 + lane; r < rows; r += 32) aj[r] = df_mul(aj[r], rden);
    }
    __syncwarp();
    if (lane == 0) {
      tau[j] = t;
      if (alpha != 0.0) aj[j] = df_from(beta);
    }
  };
  if (warp == 0) reflect(0);
  __syncthreads();
  for (int j = 0; j < s; ++j) {
    const df* aj = A + (size_t)j * rows;
    const double t = tau[j];
    // pairs of columns per warp, as in block_householder
    const int npairs = (s - j) / 2;
    const df td = df_from(t);
    for (int pr = warp; pr < npairs; pr += nwarps) {
      const int l0 = j + 1 + 2 * pr;
      df* a0 = A + (size_t)l0 * rows;
      df* a1 = l0 + 1 < s ? a0 + rows : nullptr;
      if (t != 0.0) {
        df s0, s1;
        dot2_pair_df(aj, a0, a1, j + 1 + lane, rows, lane, s0, s1);
        const df w0 = df_mul(df_add(s0, a0[j]), td);
        const df w1 = a1 != nullptr ? df_mul(df_add(s1, a1[j]), td) : df{0.f, 0.f};
        __syncwarp();  // every lane has read a0[j], a1[j] before lane 0 updates them
        if (lane == 0) {
          a0[j] = df_add(a0[j], df_neg(w0));
          if (a1 != nullptr) a1[j] = df_add(a1[j], df_neg(w1));
        }
        const df nw0 = df_neg(w0), nw1 = df_neg(w1);
        if (a1 != nullptr) {
          for (int r = j + 1 + lane; r < rows; r += 32) {
            const df v = aj[r];
            a0[r] = df_fma(v, nw0, a0[r]);
            a1[r] = df_fma(v, nw1, a1[r]);
          }
        } else {
          for (int r = j + 1 + lane; r < rows; r += 32) a0[r] = df_fma(aj[r], nw0, a0[r]);
        }
        __syncwarp();
      }
      if (l0 == j + 1) reflect(l0);
    }
    __syncthreads();
  }
}

// tsqr_leaf_factor for an FP32 block: the tile in double-float, the reflectors
// kept as double-float pairs (8 bytes, in the same workspace slots), tau, the
// WY triangle and the R factor in FP64.
constexpr int kDfThreads = 512;  // twice the FP64 kernels' warps: the double-float chains need more in flight

__global__ void __launch_bounds__(kDfThreads)
tsqr_leaf_factor_df(TsqrPlan p, Seg a, double* work, double* R, int32_t ldr, DevStatus* st, int32_t block) {
  if (failed(st)) return;
  extern __shared__ double sm[];
  __shared__ double tau[64];
  const int mt = p.mt, s = p.s;
  df* A = reinterpret_cast<df*>(sm);  // mt x s
  const int t = blockIdx.x;
  const int64_t row0 = (int64_t)t * mt;
  const int rows_here = (int)(p.m - row0 < (int64_t)mt ? p.m - row0 : (int64_t)mt);
  const float* src = reinterpret_cast<const float*>(a.p);
  for (int e = threadIdx.x; e < mt * s; e += kDfThreads) {
    const int r = e % mt, j = e / mt;
    A[e] = df{r < rows_here ? src[row0 + r + (int64_t)j * a.ld] : 0.0f, 0.0f};
  }
  __syncthreads();
  block_householder_df(A, mt, s, tau);
  df* H = reinterpret_cast<df*>(work + p.off_h) + (size_t)t * mt * s;
  for (int e = threadIdx.x; e < mt * s; e += kDfThreads) H[e] = A[e];
  double* tg = work + p.off_tau[0] + (size_t)t * s;
  for (int j = threadIdx.x; j < s; j += kDfThreads) tg[j] = tau[j];
  double* VV = sm + (size_t)mt * s;  // s x s: (V^T V)_{ij} for i < j, later the root's R
  double* Tl = VV + (size_t)s * s;
  {
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    int task = 0;
    for (int j = 1; j < s; ++j) {
      const df* vj = A + (size_t)j * mt;
      for (int i = 0; i < j; i += 2, ++task) {
        if (task % (kDfThreads / 32) != warp) continue;
        const df* vi = A + (size_t)i * mt;
        const df* vi1 = i + 1 < j ? vi + mt : nullptr;
        df d0, d1;
        dot2_pair_df(vj, vi, vi1, j + 1 + lane, mt, lane, d0, d1);
        if (lane == 0) {
          VV[i + (size_t)j * s] = df_dbl(df_add(d0, vi[j]));
          if (vi1 != nullptr) VV[i + 1 + (size_t)j * s] = df_dbl(df_add(d1, vi1[j]));
        }
      }
    }
    __syncthreads();
    for (int j = 0; j < s; ++j) {
      for (int i = threadIdx.x; i < s; i += kDfThreads) {
        double x = 0.0;
        if (i < j)
          for (int l = i; l < j; ++l) x = fma(Tl[i + (size_t)l * s], VV[l + (size_t)j * s], x);
        Tl[i + (size_t)j * s] = i < j ? -tau[j] * x : (i == j ? tau[j] : 0.0);
      }
      __syncthreads();
    }
    double* tw = work + p.off_t0 + (size_t)t * s * s;
    for (int e = threadIdx.x; e < s * s; e += kDfThreads) tw[e] = Tl[e];
  }
  if (p.nlevels == 1) {
    // the R factor (upper triangle of the tile) in FP64, then the root's signs
    __syncthreads();
    for (int e = threadIdx.x; e < s * s; e += kDfThreads) {
      const int i = e % s, j = e / s;
      VV[e] = df_dbl(A[i + (size_t)j * mt]);
    }
    __syncthreads();
    finish_root(VV, s, s, R, ldr, work + p.off_b[0], st, block);
    return;
  }
  const int fan = p.fan, ldp = fan * s;
  double* P = work + p.off_lvl[1] + (size_t)(t / fan) * ldp * s;
  const int rbase = (t % fan) * s;
  for (int e = threadIdx.x; e < s * s; e += kDfThreads) {
    const int i = e % s, j = e / s;
    P[rbase + i + (size_t)j * ldp] = i <= j ? df_dbl(A[i + (size_t)j * mt]) : 0.0;
  }
}

// tsqr_leaf_apply for an FP32 block: E = [B; 0] - V (T (V_top^T B)) entirely
// in double-float (one thread per row and 16-column group for the mt x s
// product), each result rounded once to float; the maxima of the stored values
// from registers.
__global__ void __launch_bounds__(kDfThreads)
tsqr_leaf_apply_df(TsqrPlan p, const double* work, void* q, int64_t ldq, const DevStatus* st, MaxOut qmax) {
  if (failed(st)) return;
  extern __shared__ double sm[];
  const int mt = p.mt, s = p.s;
  const int t = blockIdx.x;
  df* V = reinterpret_cast<df*>(sm);                  // mt x s
  double* Bs = sm + (size_t)mt * s;                   // s x s coefficient block from the parent, then W
  double* Tl = Bs + (size_t)s * s;                    // s x s WY triangle, then M = T W
  double* W = Tl + (size_t)s * s;                     // s x s: B in double-float
  df* Md = reinterpret_cast<df*>(W + (size_t)s * s);  // s x s: T in double-float
  const df* H = reinterpret_cast<const df*>(work + p.off_h) + (size_t)t * mt * s;
  const double* B = work + p.off_b[0] + (size_t)t * s * s;
  const double* Tg = work + p.off_t0 + (size_t)t * s * s;
  for (int e = threadIdx.x; e < mt * s; e += kDfThreads) V[e] = H[e];
  for (int e = threadIdx.x; e < s * s; e += kDfThreads) {
    Bs[e] = B[e];
    Tl[e] = Tg[e];
  }
  __syncthreads();
  // W = V_top^T B and M = T W in double-float too (no FP64 work in this kernel:
  // GB300's FP64 rate would make these s^3 products its slowest part); B and T
  // go to double-float once, into the s x s slots of W (as Bd) and Md (as Td)
  df* Bd = reinterpret_cast<df*>(W);
  df* Td = Md;
  for (int e = threadIdx.x; e < s * s; e += kDfThreads) {
    Bd[e] = df_from(Bs[e]);
    Td[e] = df_from(Tl[e]);
  }
  __syncthreads();
  df* Wd = reinterpret_cast<df*>(Bs);  // B itself is read again below from Bd
  for (int e = threadIdx.x; e < s * s; e += kDfThreads) {
    const int l = e % s, c = e / s;
    df x = Bd[l + (size_t)c * s];
    for (int i = l + 1; i < s; ++i) x = df_fma(V[i + (size_t)l * mt], Bd[i + (size_t)c * s], x);
    Wd[e] = x;
  }
  __syncthreads();
  df* Mw = reinterpret_cast<df*>(Tl);  // T is read from Td
  for (int e = threadIdx.x; e < s * s; e += kDfThreads) {
    const int l = e % s, c = e / s;
    df x{0.0f, 0.0f};
    for (int i = l; i < s; ++i) x = df_fma(Td[l + (size_t)i * s], Wd[i + (size_t)c * s], x);
    Mw[e] = x;
  }
  __syncthreads();
  const int64_t row0 = (int64_t)t * mt;
  const int rows_here = (int)(p.m - row0 < (int64_t)mt ? p.m - row0 : (int64_t)mt);
  float* dst = reinterpret_cast<float*>(q);
  const int ngr = (s + 15) / 16;
  // mt is a multiple of 32, so each warp's lanes share one column group (the
  // column maxima are warp reductions)
  for (int w = threadIdx.x; w < mt * ngr; w += kDfThreads) {
    const int r = w % mt, c0 = (w / mt) * 16;
    const int nc = s - c0 < 16 ? s - c0 : 16;
    df e[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) e[c] = (c < nc && r < s) ? Bd[r + (size_t)(c0 + c) * s] : df{0.0f, 0.0f};
    const int lmax = r < s ? r + 1 : s;  // V(r, l) = 0 for l > r
    for (int l = 0; l < lmax; ++l) {
      const df nv = l == r ? df{-1.0f, 0.0f} : df_neg(V[r + (size_t)l * mt]);
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c < nc) e[c] = df_fma(nv, Mw[l + (size_t)(c0 + c) * s], e[c]);
    }
    const bool live = r < rows_here;
    unsigned long long rmax = 0ull;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      if (c < nc) {
        const float f = __fadd_rn(e[c].hi, e[c].lo);
        if (live) dst[row0 + r + (int64_t)(c0 + c) * ldq] = f;
        const unsigned long long b = live ? abs_bits64((double)f) : 0ull;
        rmax = umax64(rmax, b);
        if (qmax.col != nullptr) warp_max_to(b, qmax.col + c0 + c);
      }
    }
    if (live && qmax.row != nullptr) atomicMax(qmax.row + row0 + r, rmax);
  }
}

// block_apply_q in double-float.
__device__ void block_apply_q_df(const df* V, const double* tau, df* E, int rows, int s) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int nwarps = blockDim.x / 32;
  const int npairs = (s + 1) / 2;
  for (int j = s - 1; j >= 0; --j) {
    const double t = tau[j];
    if (t != 0.0) {
      const df td = df_from(t);
      const df* vj = V + (size_t)j * rows;
      for (int pr = warp; pr < npairs; pr += nwarps) {
        df* e0 = E + (size_t)(2 * pr) * rows;
        df* e1 = 2 * pr + 1 < s ? e0 + rows : nullptr;
        df s0, s1;
        dot2_pair_df(vj, e0, e1, j + 1 + lane, rows, lane, s0, s1);
        const df w0 = df_mul(df_add(s0, e0[j]), td);
        const df w1 = e1 != nullptr ? df_mul(df_add(s1, e1[j]), td) : df{0.f, 0.f};
        __syncwarp();
        if (lane == 0) {
          e0[j] = df_add(e0[j], df_neg(w0));
          if (e1 != nullptr) e1[j] = df_add(e1[j], df_neg(w1));
        }
        const df nw0 = df_neg(w0), nw1 = df_neg(w1);
        if (e1 != nullptr) {
          for (int r = j + 1 + lane; r < rows; r += 32) {
            const df v = vj[r];
            e0[r] = df_fma(v, nw0, e0[r]);
            e1[r] = df_fma(v, nw1, e1[r]);
          }
        } else {
          for (int r = j + 1 + lane; r < rows; r += 32) e0[r] = df_fma(vj[r], nw0, e0[r]);
        }
        __syncwarp();
      }
    }
    __syncthreads();
  }
}

// tsqr_node_factor for the tree of an FP32 block: the stacked R factors (FP64)
// factored in double-float; the reflectors go back into the level's slots as
// double-float pairs (read only by tsqr_node_apply_df), tau and the R factor
// passed up in FP64.  Dynamic shared memory: the node matrix plus s x s doubles.
__global__ void __launch_bounds__(kDfThreads)
tsqr_node_factor_df(TsqrPlan p, int32_t level, double* work, double* R, int32_t ldr, DevStatus* st,
                    int32_t block) {
  if (failed(st)) return;
  extern __shared__ double sm[];
  __shared__ double tau[64];
  const int s = p.s, fan = p.fan, rows = fan * s;
  const int n = blockIdx.x;
  const int nchild = min(fan, p.nodes[level - 1] - n * fan);
  const int re = nchild * s;
  df* A = reinterpret_cast<df*>(sm);
  double* Rb = sm + (size_t)rows * s;  // s x s: the root's R in FP64
  double* G = work + p.off_lvl[level] + (size_t)n * rows * s;
  for (int e = threadIdx.x; e < re * s; e += kDfThreads) {
    const int r = e % re, j = e / re;
    A[e] = df_from(G[r + (size_t)j * rows]);
  }
  __syncthreads();
  block_householder_df(A, re, s, tau);
  df* Gd = reinterpret_cast<df*>(G);
  for (int e = threadIdx.x; e < re * s; e += kDfThreads) {
    const int r = e % re, j = e / re;
    Gd[r + (size_t)j * rows] = A[e];
  }
  double* tg = work + p.off_tau[level] + (size_t)n * s;
  for (int j = threadIdx.x; j < s; j += kDfThreads) tg[j] = tau[j];
  if (level == p.nlevels - 1) {
    for (int e = threadIdx.x; e < s * s; e += kDfThreads) {
      const int i = e % s, j = e / s;
      Rb[e] = df_dbl(A[i + (size_t)j * re]);
    }
    __syncthreads();
    finish_root(Rb, s, s, R, ldr, work + p.off_b[level], st, block);
    return;
  }
  double* P = work + p.off_lvl[level + 1] + (size_t)(n / fan) * rows * s;
  const int rbase = (n % fan) * s;
  for (int e = threadIdx.x; e < s * s; e += kDfThreads) {
    const int i = e % s, j = e / s;
    P[rbase + i + (size_t)j * rows] = i <= j ? df_dbl(A[i + (size_t)j * re]) : 0.0;
  }
}

// tsqr_node_apply for the tree of an FP32 block, in double-float; the children's
// coefficient blocks go out in FP64.
__global__ void __launch_bounds__(kDfThreads)
tsqr_node_apply_df(TsqrPlan p, int32_t level, double* work, const DevStatus* st) {
  if (failed(st)) return;
  extern __shared__ double sm[];
  __shared__ double tau[64];
  const int s = p.s, fan = p.fan, rows = fan * s;
  const int n = blockIdx.x;
  const int nchild = min(fan, p.nodes[level - 1] - n * fan);
  const int re = nchild * s;
  df* V = reinterpret_cast<df*>(sm);
  df* E = V + (size_t)re * s;
  const df* Gd = reinterpret_cast<const df*>(work + p.off_lvl[level] + (size_t)n * rows * s);
  const double* B = work + p.off_b[level] + (size_t)n * s * s;
  for (int e = threadIdx.x; e < re * s; e += kDfThreads) {
    const int r = e % re, j = e / re;
    V[e] = Gd[r + (size_t)j * rows];
    E[e] = df_from(r < s ? B[r + (size_t)j * s] : 0.0);
  }
  for (int j = threadIdx.x; j < s; j += kDfThreads) tau[j] = work[p.off_tau[level] + (size_t)n * s + j];
  __syncthreads();
  block_apply_q_df(V, tau, E, re, s);
  for (int e = threadIdx.x; e < nchild * s * s; e += kDfThreads) {
    const int g = e / (s * s), rem = e % (s * s);
    const int i = rem % s, j = rem / s;
    work[p.off_b[level - 1] + (size_t)(n * fan + g) * s * s + i + (size_t)j * s] =
        df_dbl(E[g * s + i + (size_t)j * re]);
  }
}

template <typename T>
cudaError_t launch_tsqr_t(const TsqrPlan& p, Seg a, void* q, int64_t ldq, double* R, int32_t ldr,
                          double* work, DevStatus* st, int32_t block, cudaStream_t stream, MaxOut qmax) {
  const size_t leaf_f = (size_t)p.mt * p.s * sizeof(double);
  const size_t ss = (size_t)p.s * p.s * sizeof(double);
  const size_t node_f = (size_t)p.fan * p.s * p.s * sizeof(double);
  // FP32 blocks: the leaves in double-float (their E buffer holds floats)
  constexpr bool kDf = std::is_same<T, float>::value;
  const size_t apply_f = kDf ? leaf_f + 4 * ss : 2 * leaf_f + 3 * ss;
  cudaError_t e;
  e = kDf ? ensure_dyn_smem(tsqr_leaf_factor_df, leaf_f + 2 * ss) : ensure_dyn_smem(tsqr_leaf_factor<T>, leaf_f + 2 * ss);
  if (e != cudaSuccess) return e;
  e = kDf ? ensure_dyn_smem(tsqr_leaf_apply_df, apply_f) : ensure_dyn_smem(tsqr_leaf_apply<T>, apply_f);
  if (e != cudaSuccess) return e;
  e = kDf ? ensure_dyn_smem(tsqr_node_factor_df, node_f + ss) : ensure_dyn_smem(tsqr_node_factor, node_f);
  if (e != cudaSuccess) return e;
  e = kDf ? ensure_dyn_smem(tsqr_node_apply_df, 2 * node_f) : ensure_dyn_smem(tsqr_node_apply, 2 * node_f);
  if (e != cudaSuccess) return e;
  const int slot = prof_begin(stream);
  if (kDf)
    tsqr_leaf_factor_df<<<p.nodes[0], kDfThreads, leaf_f + 2 * ss, stream>>>(p, a, work, R, ldr, st, block);
  else
    tsqr_leaf_factor<T><<<p.nodes[0], kTsqrThreads, leaf_f + 2 * ss, stream>>>(p, a, work, R, ldr, st, block);
  for (int l = 1; l < p.nlevels; ++l)
    if (kDf)
      tsqr_node_factor_df<<<p.nodes[l], kDfThreads, node_f + ss, stream>>>(p, l, work, R, ldr, st, block);
    else
      tsqr_node_factor<<<p.nodes[l], kTsqrThreads, node_f, stream>>>(p, l, work, R, ldr, st, block);
  for (int l = p.nlevels - 1; l >= 1; --l)
    if (kDf)
      tsqr_node_apply_df<<<p.nodes[l], kDfThreads, 2 * node_f, stream>>>(p, l, work, st);
    else
      tsqr_node_apply<<<p.nodes[l], kTsqrThreads, 2 * node_f, stream>>>(p, l, work, st);
  if (kDf)
    tsqr_leaf_apply_df<<<p.nodes[0], kDfThreads, apply_f, stream>>>(p, work, q, ldq, st, qmax);
  else
    tsqr_leaf_apply<T><<<p.nodes[0], kTsqrThreads, apply_f, stream>>>(p, work, q, ldq, st, qmax);
  // Householder QR and explicit Q of the m x s block: 2 m s^2 flops each.
  prof_end(slot, kProfTsqr, stream, 4.0 * (double)p.m * p.s * p.s,
           2.0 * (double)p.m * p.s * sizeof(T) + 2.0 * (double)p.nodes[0] * p.mt * p.s * 8.0);
  note_launch(2 * p.nlevels);
  return cudaGetLastError();
}

}  // namespace

void tsqr_plan(int64_t m, int32_t s, TsqrPlan* p) {
  p->m = m;
  p->s = s;
  // Leaf tiles of at most about 8192 doubles (64 KB of shared memory), and no
  // taller than needed for about two tiles per SM of a 152-SM GB300: a tile's
  // Householder runs its columns one after the other on the FP64 pipe of one
  // SM, so a few tall tiles would leave most SMs idle on large blocks.  At
  // least 2s rows (a fan-in of two), a multiple of 32.
  const int64_t cap = round_up(8192 / s, 32) > 1024 ? 1024 : round_up(8192 / s, 32);
  int64_t mt = cap;
  const int64_t spread = round_up(ceil_div(m, 304), 32);
  if (mt > spread) mt = spread;
  if (mt < round_up(2 * s, 32)) mt = round_up(2 * s, 32);
  // On small blocks every tree level is a pair of latency-bound launches (about
  // 27 + 16 us measured, whatever the node size), so taller leaves pay when they
  // save a level.  Estimated time of leaf height h (us, measured on GB300: 35 us
  // for a leaf's chain of reflectors plus its FP64 work at 2 DFMA per cycle and
  // SM, 2.07 GHz; the whole leaf level at the FP64 rate of 152 SMs; 43 us per
  // level): the h from the one above up to the cap with the smallest estimate.
  auto levels_of = [&](int64_t h) {
    const int64_t f = h / s < 2 ? 2 : h / s;
    int64_t nodes = ceil_div(m, h);
    int lv = 0;
    while (nodes > 1) {
      nodes = ceil_div(nodes, f);
      ++lv;
    }
    return lv;
  };
  auto estimate = [&](int64_t h) {
    const double one_leaf = 35.0 + (double)h * s * s / 2070.0;
    const double all_leaves = (double)m * s * s / (152.0 * 2070.0);
    return (one_leaf > all_leaves ? one_leaf : all_leaves) + 43.0 * levels_of(h);
  };
  for (int64_t h = mt + 32; h <= cap && h <= round_up(m, 32); h += 32)
    if (estimate(h) < estimate(mt)) mt = h;
  if (mt > round_up(m, 32)) mt = round_up(m, 32) < s ? s : round_up(m, 32);
  p->mt = (int32_t)mt;
  int fan = (int)(mt / s);
  if (fan < 2) fan = 2;
  p->fan = fan;
  int lvl = 0;
  p->nodes[0] = (int32_t)ceil_div(m, mt);
  while (p->nodes[lvl] > 1 && lvl < 31) {
    p->nodes[lvl + 1] = (int32_t)ceil_div(p->nodes[lvl], fan);
    ++lvl;
  }
  p->nlevels = lvl + 1;
  size_t off = 0;
  p->off_h = off;
  off += (size_t)p->nodes[0] * mt * s;
  p->off_t0 = off;
  off += (size_t)p->nodes[0] * s * s;
  for (int l = 0; l < p->nlevels; ++l) {
    p->off_tau[l] = off;
    off += round_up((size_t)p->nodes[l] * s, 32);
    p->off_b[l] = off;
    off += (size_t)p->nodes[l] * s * s;
    if (l >= 1) {
      p->off_lvl[l] = off;
      off += (size_t)p->nodes[l] * fan * s * s;
    } else {
      p->off_lvl[l] = 0;
    }
  }
  p->doubles = round_up(off, 32);
}

cudaError_t launch_stack_r(const double* recv, int32_t nranks, int32_t s, double* out, const DevStatus* st,
                           cudaStream_t stream) {
  stack_r_kernel<<<(nranks * s * s + 255) / 256, 256, 0, stream>>>(recv, nranks, s, out, st);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_rows_times_small(int64_t m, int32_t s, const void* A, int64_t lda, const double* B, int32_t ldb,
                                    void* W, int64_t ldw, int32_t fp32, MaxOut wmax, const DevStatus* st,
                                    cudaStream_t stream) {
  if (m <= 0) return cudaSuccess;
  if (s < 1 || s > 64) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)ceil_div(m, 256);
  if (fp32)
    rows_times_small_kernel<float><<<grid, 256, 0, stream>>>(m, s, reinterpret_cast<const float*>(A), lda, B, ldb,
                                                              reinterpret_cast<float*>(W), ldw, wmax, st);
  else
    rows_times_small_kernel<double><<<grid, 256, 0, stream>>>(m, s, reinterpret_cast<const double*>(A), lda, B, ldb,
                                                               reinterpret_cast<double*>(W), ldw, wmax, st);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_tsqr(const TsqrPlan& p, Seg a, void* q, int64_t ldq, int32_t q_fp32, double* R,
                        int32_t ldr, double* work, DevStatus* st, int32_t block,
                        cudaStream_t stream, MaxOut qmax) {
  if (p.m <= 0) return cudaSuccess;
  (void)q_fp32;
  return a.fp32 ? launch_tsqr_t<float>(p, a, q, ldq, R, ldr, work, st, block, stream, qmax)
                : launch_tsqr_t<double>(p, a, q, ldq, R, ldr, work, st, block, stream, qmax);
}

}  // namespace bcgs
