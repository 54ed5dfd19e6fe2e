// The small FP64 tail of a block step (one CTA; all operands are at most
// (n+s) x s).  After the synchronization of block k (Alg. 2's sync step, which
// returns [Y_{1:k-1,k} Z_{k-1}; Omega_k P_k] and, under BCGSI+P-1S, T_{k+1}):
//
//   Y_kk          = chol(Omega_k - Y_{1:k-1,k}^T Y_{1:k-1,k})       (Alg. 2)
//   R_{1:k-1,k}   = S_{1:k-1,k} + Y_{1:k-1,k} S_kk,  R_kk = Y_kk S_kk
//   S_{1:k,k+1}   = [Z_{k-1}; Y_kk^{-T} (P_k - Y_{1:k-1,k}^T Z_{k-1})]   (eq. (1))
//   S_{k+1,k+1}   = chol(T_{k+1} - S_{1:k,k+1}^T S_{1:k,k+1})      (BCGSI+P-1S only)
//
// A pivot that is not > 0 sets BCGS_ERR_NOT_SPD (BCGS_ERR_NONFINITE for NaN/Inf)
// with the block index; every later kernel then does nothing.
#include "bcgs_internal.cuh"

namespace bcgs {

namespace {

constexpr int kTailThreads = 1024;
constexpr int kMaxS = 64;

// C (s x s, smem, ld s) = A^T B over `rows` rows; A, B column-major (lda, ldb).
// With s^2 <= blockDim / 2 each entry takes g = blockDim / s^2 threads: thread
// part p adds the rows p, p + g, ... and the g sums are added in part order (a
// fixed order: the result depends on the shape and blockDim only), so the FP64
// chains are g times shorter.  Called by every thread of the CTA.
__device__ void small_tn(int rows, int s, const double* A, int lda, const double* B, int ldb,
                         double* C) {
  __shared__ double red[kTailThreads];
  const int ss = s * s;
  const int g = (int)blockDim.x / ss;
  if (g < 2) {
    for (int e = threadIdx.x; e < ss; e += blockDim.x) {
      const int i = e % s, j = e / s;
      const double* a = A + (size_t)i * lda;
      const double* b = B + (size_t)j * ldb;
      double acc = 0.0;
      for (int r = 0; r < rows; ++r) acc = fma(a[r], b[r], acc);
      C[e] = acc;
    }
    return;
  }
  const int e = threadIdx.x % ss, part = threadIdx.x / ss;
  double acc = 0.0;
  if (part < g) {
    const int i = e % s, j = e / s;
    const double* a = A + (size_t)i * lda;
    const double* b = B + (size_t)j * ldb;
    for (int r = part; r < rows; r += g) acc = fma(a[r], b[r], acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < ss) {
    double t = red[threadIdx.x];
    for (int p = 1; p < g; ++p) t += red[threadIdx.x + p * ss];
    C[threadIdx.x] = t;
  }
  __syncthreads();
}

// Upper Cholesky factor of the s x s matrix M (smem, ld s, upper triangle read)
// into Rc (smem, ld s).  Returns 0, BCGS_ERR_NOT_SPD or BCGS_ERR_NONFINITE
// (uniform across the block).  The pivot's reciprocal square root r gives
// R_jj = d r and the row's entries (M_ji - dot) r: one FP64 function call on
// the serial chain of each column and a multiplication, not a division, per
// entry (GB300's FP64 divide is a long dependent sequence on a slow pipe).
__device__ int small_chol(int s, const double* M, double* Rc) {
  __shared__ int code;
  __shared__ double rinv;
  if (threadIdx.x == 0) code = 0;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) Rc[e] = 0.0;
  __syncthreads();
  for (int j = 0; j < s; ++j) {
    if (threadIdx.x == 0) {
      double dot = 0.0;
      for (int l = 0; l < j; ++l) dot = fma(Rc[l + j * s], Rc[l + j * s], dot);
      const double d = M[j + j * s] - dot;
      if (!isfinite(d)) code = BCGS_ERR_NONFINITE;
      else if (!(d > 0.0)) code = BCGS_ERR_NOT_SPD;
      const double r = code ? 1.0 : rsqrt(d);
      rinv = r;
      Rc[j + j * s] = code ? 1.0 : d * r;
    }
    __syncthreads();
    if (code) return code;
    const double r = rinv;
    for (int i = j + 1 + threadIdx.x; i < s; i += blockDim.x) {
      double dot = 0.0;
      for (int l = 0; l < j; ++l) dot = fma(Rc[l + j * s], Rc[l + i * s], dot);
      Rc[j + i * s] = (M[j + i * s] - dot) * r;
    }
    __syncthreads();
  }
  return 0;
}

// dyn: 4 s^2 doubles of dynamic shared memory.
__device__ void tail_1s2s_body(const TailDesc& d, DevStatus* st, double* dyn) {
  const int s = d.s, c = d.c;
  double* Ms = dyn;
  double* Yd = dyn + s * s;
  double* Sd = dyn + 2 * s * s;
  double* Wb = dyn + 3 * s * s;
  const double* G = d.G;
  const int ldg = d.ldg;
  const double* Yg = G + d.gy;           // c x s  (Y_{1:k-1,k})
  const double* Zg = G + d.gz;           // c x s  (Z_{k-1})
  const double* Omg = G + d.gom;         // s x s  (Omega_k)
  const double* Pg = G + d.gp;           // s x s  (P_k)
  const double* Tg = G + d.gt;           // s x s  (T_{k+1})

  // Y_kk = chol(Omega - Y^T Y)
  small_tn(c, s, Yg, ldg, Yg, ldg, Ms);
  __syncthreads();
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    const int i = e % s, j = e / s;
    Ms[e] = Omg[i + (size_t)j * ldg] - Ms[e];
  }
  __syncthreads();
  int code = small_chol(s, Ms, Yd);
  if (code) {
    if (threadIdx.x == 0) set_failure(st, code, d.block);
    return;
  }
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    Sd[e] = d.Sd_prev[e];
    d.Yd[e] = Yd[e];
  }
  // reciprocals of Y_kk's diagonal for the triangular solves below: their
  // serial chains then multiply instead of dividing
  __shared__ double rdiag[kMaxS];
  for (int i = threadIdx.x; i < s; i += blockDim.x) rdiag[i] = 1.0 / Yd[i + i * s];
  __syncthreads();
  // R_{1:k-1,k} = S + Y S_kk ; R_kk = Y_kk S_kk
  for (int e = threadIdx.x; e < (c + s) * s; e += blockDim.x) {
    const int i = e % (c + s), j = e / (c + s);
    double v;
    if (i < c) {
      double t = 0.0;
      for (int l = 0; l <= j; ++l) t = fma(Yg[i + (size_t)l * ldg], Sd[l + j * s], t);
      v = d.S_prev[i + (size_t)j * d.ldsm] + t;
    } else {
      const int ii = i - c;
      double t = 0.0;
      for (int l = ii; l <= j; ++l) t = fma(Yd[ii + l * s], Sd[l + j * s], t);
      v = t;
    }
    d.R[(d.r_row0 + i) + (size_t)(d.r_col0 + j) * d.ldr] = v;
  }
  if (d.Bpair != nullptr) {
    // Q_k = (U_k - Q_{1:k-1} Y) Y_kk^{-1} = [Q_{1:k-1} U_k] [-Y Yi; Yi], Yi = Y_kk^{-1}
    // (upper triangular, by back substitution; Y_kk is close to the identity
    // once U_k has been normalized, so the explicit inverse costs no accuracy).
    __syncthreads();
    double* Yi = Sd;  // S_kk is no longer needed
    for (int j = threadIdx.x; j < s; j += blockDim.x) {
      for (int i = s - 1; i >= 0; --i) {
        double x = i == j ? 1.0 : 0.0;
        for (int l = i + 1; l <= j; ++l) x = fma(-Yd[i + l * s], Yi[l + j * s], x);
        Yi[i + j * s] = i > j ? 0.0 : x * rdiag[i];
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < (c + s) * s; e += blockDim.x) {
      const int i = e % (c + s), j = e / (c + s);
      double v;
      if (i < c) {
        double t = 0.0;
        for (int l = 0; l <= j; ++l) t = fma(Yg[i + (size_t)l * ldg], Yi[l + j * s], t);
        v = -t;
      } else {
        v = Yi[(i - c) + j * s];
      }
      d.Bpair[i + (size_t)j * d.ldb] = v;
    }
  }
  if (!d.has_next) return;
  // S_{1:k,k+1} = [Z; Y_kk^{-T} (P - Y^T Z)]
  small_tn(c, s, Yg, ldg, Zg, ldg, Ms);
  __syncthreads();
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    const int i = e % s, j = e / s;
    Ms[e] = Pg[i + (size_t)j * ldg] - Ms[e];
  }
  __syncthreads();
  // forward substitution with Y_kk^T (lower): W_i = (M_i - sum_{l<i} Yd_li W_l) / Yd_ii
  for (int j = threadIdx.x; j < s; j += blockDim.x) {
    for (int i = 0; i < s; ++i) {
      double dot = 0.0;
      for (int l = 0; l < i; ++l) dot = fma(Yd[l + i * s], Wb[l + j * s], dot);
      Wb[i + j * s] = (Ms[i + j * s] - dot) * rdiag[i];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < (c + s) * s; e += blockDim.x) {
    const int i = e % (c + s), j = e / (c + s);
    d.S_next[i + (size_t)j * d.ldsm] = i < c ? Zg[i + (size_t)j * ldg] : Wb[(i - c) + j * s];
  }
  if (d.Bpair != nullptr) {
    // Coefficients of the paired projection (Q_k and the next block in one pass
    // over [Q_{1:k-1} U_k]): Q_{1:k} S_{1:k,k+1} = Q_{1:k-1} Z + Q_k W
    //   = Q_{1:k-1} (Z - Y M) + U_k M  with  M = Y_kk^{-1} W, since
    // Q_k = (U_k - Q_{1:k-1} Y) Y_kk^{-1}.
    __syncthreads();
    // M = Y_kk^{-1} W by back substitution (into Ms), column by column
    for (int j = threadIdx.x; j < s; j += blockDim.x) {
      for (int i = s - 1; i >= 0; --i) {
        double x = Wb[i + j * s];
        for (int l = i + 1; l < s; ++l) x = fma(-Yd[i + l * s], Ms[l + j * s], x);
        Ms[i + j * s] = x * rdiag[i];
      }
    }
    __syncthreads();
    double* B = d.Bpair + (size_t)s * d.ldb;
    for (int e = threadIdx.x; e < (c + s) * s; e += blockDim.x) {
      const int i = e % (c + s), jj = e / (c + s);
      double v;
      if (i < c) {
        double t = 0.0;
        for (int l = 0; l < s; ++l) t = fma(Yg[i + (size_t)l * ldg], Ms[l + jj * s], t);
        v = Zg[i + (size_t)jj * ldg] - t;
      } else {
        v = Ms[(i - c) + jj * s];
      }
      B[i + (size_t)jj * d.ldb] = v;
    }
  }
  if (!d.chol_next) return;
  __syncthreads();
  // S_{k+1,k+1} = chol(T - S^T S), S = S_{1:k,k+1} ((c+s) x s, just written)
  __threadfence_block();
  small_tn(c + s, s, d.S_next, d.ldsm, d.S_next, d.ldsm, Ms);
  __syncthreads();
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    const int i = e % s, j = e / s;
    Ms[e] = Tg[i + (size_t)j * ldg] - Ms[e];
  }
  __syncthreads();
  code = small_chol(s, Ms, Wb);
  if (code) {
    if (threadIdx.x == 0) set_failure(st, code, d.block + 1);
    return;
  }
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) d.Sd_next[e] = Wb[e];
}

__global__ void __launch_bounds__(kTailThreads) tail_1s2s_kernel(TailDesc d, DevStatus* st) {
  if (failed(st)) return;
  extern __shared__ double dyn[];
  tail_1s2s_body(d, st, dyn);
}

// Pythagorean Cholesky of one block (Alg. 1; the startup of BCGSI+P-1S is its
// c = s case): G = [S; T] = [Q_{1:k} V]^T V with S = G[0:c, :], T = G[c:c+s, :],
// R_kk = chol(T - S^T S).  S is copied to S_out (ld ldsm) when S_out is set.
__global__ void __launch_bounds__(kTailThreads)
tail_pchol_kernel(int32_t c, int32_t s, const double* G, int32_t ldg, double* S_out, int32_t ldsm,
                  double* Rkk, int32_t block, DevStatus* st) {
  if (failed(st)) return;
  extern __shared__ double dyn[];
  double* Ms = dyn;
  double* Rc = dyn + s * s;
  small_tn(c, s, G, ldg, G, ldg, Ms);
  __syncthreads();
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    const int i = e % s, j = e / s;
    Ms[e] = G[(c + i) + (size_t)j * ldg] - Ms[e];
  }
  if (S_out != nullptr)
    for (int e = threadIdx.x; e < c * s; e += blockDim.x) {
      const int i = e % c, j = e / c;
      S_out[i + (size_t)j * ldsm] = G[i + (size_t)j * ldg];
    }
  __syncthreads();
  const int code = small_chol(s, Ms, Rc);
  if (code) {
    if (threadIdx.x == 0) set_failure(st, code, block);
    return;
  }
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) Rkk[e] = Rc[e];
}

__global__ void copy_small_kernel(int32_t rows, int32_t cols, const double* A, int32_t lda,
                                  double* B, int32_t ldb, const DevStatus* st) {
  if (failed(st)) return;
  for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < rows * cols; e += blockDim.x * gridDim.x) {
    const int i = e % rows, j = e / rows;
    B[i + (size_t)j * ldb] = A[i + (size_t)j * lda];
  }
}

// BCGSI+: R_{1:k,k+1} = S + Y S_kk, R_{k+1,k+1} = Y_kk S_kk (as in Alg. 1).
__global__ void r_assemble_kernel(int32_t c, int32_t s, const double* S, int32_t lds, const double* Y,
                                  int32_t ldy, const double* Sd, const double* Yd, double* R,
                                  int32_t ldr, int32_t col0, const DevStatus* st) {
  if (failed(st)) return;
  for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < (c + s) * s; e += blockDim.x * gridDim.x) {
    const int i = e % (c + s), j = e / (c + s);
    double v;
    if (i < c) {
      double t = 0.0;
      for (int l = 0; l <= j; ++l) t = fma(Y[i + (size_t)l * ldy], Sd[l + (size_t)j * s], t);
      v = S[i + (size_t)j * lds] + t;
    } else {
      const int ii = i - c;
      double t = 0.0;
      for (int l = ii; l <= j; ++l) t = fma(Yd[ii + (size_t)l * s], Sd[l + (size_t)j * s], t);
      v = t;
    }
    R[i + (size_t)(col0 + j) * ldr] = v;
  }
}

__global__ void __launch_bounds__(kTailThreads)
chol_kernel(int32_t s, const double* A, int32_t lda, double* R, int32_t ldr, int32_t block,
            DevStatus* st) {
  if (failed(st)) return;
  extern __shared__ double dyn[];
  double* Ms = dyn;
  double* Rc = dyn + s * s;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    const int i = e % s, j = e / s;
    Ms[e] = A[i + (size_t)j * lda];
  }
  __syncthreads();
  const int code = small_chol(s, Ms, Rc);
  if (code) {
    if (threadIdx.x == 0) set_failure(st, code, block);
    return;
  }
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    const int i = e % s, j = e / s;
    R[i + (size_t)j * ldr] = Rc[e];
  }
}

__global__ void zero_kernel(int32_t n, double* R, int32_t ldr) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = threadIdx.x + (int64_t)blockIdx.x * blockDim.x; e < total;
       e += (int64_t)blockDim.x * gridDim.x) {
    const int64_t i = e % n, j = e / n;
    R[i + j * ldr] = 0.0;
  }
}

// A = I (s x s, ld s): BCGSI+1s's S_{k+1,k+1}, the first intraorthogonalization
// it does not perform (Sec. 2).
__global__ void identity_kernel(int32_t s, double* A) {
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) A[e] = (e % s) == (e / s) ? 1.0 : 0.0;
}

__global__ void zero_u64_words(unsigned long long* p, int64_t n) {
  for (int64_t i = threadIdx.x + (int64_t)blockIdx.x * blockDim.x; i < n; i += (int64_t)blockDim.x * gridDim.x)
    p[i] = 0ull;
}

__global__ void reset_status_kernel(DevStatus* st, DevStatus* st2) {
  if (threadIdx.x == 0) {
    st->code = 0;
    st->block = 0;
    if (st2 != nullptr) {
      st2->code = 0;
      st2->block = 0;
    }
  }
}

// A failure recorded in `side` (work run ahead on another stream) becomes the
// factorization's failure, unless one is already recorded; `side` is cleared.
__global__ void merge_status_kernel(DevStatus* st, DevStatus* side) {
  if (threadIdx.x == 0 && side->code != 0) {
    set_failure(st, side->code, side->block);
    side->code = 0;
    side->block = 0;
  }
}

}  // namespace

cudaError_t launch_tail_1s2s(const TailDesc& d, DevStatus* st, cudaStream_t stream) {
  if (d.s > kMaxS) return cudaErrorInvalidValue;
  const size_t smem = 4 * (size_t)d.s * d.s * sizeof(double);
  cudaError_t e = ensure_dyn_smem(tail_1s2s_kernel, (size_t)(smem));
  if (e != cudaSuccess) return e;
  const int slot = prof_begin(stream);
  tail_1s2s_kernel<<<1, kTailThreads, smem, stream>>>(d, st);
  prof_end(slot, kProfTail, stream, 8.0 * (double)(d.c + d.s) * d.s * d.s, 0.0);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_tail_pchol(int32_t c, int32_t s, const double* G, int32_t ldg, double* S_out,
                              int32_t ldsm, double* Rkk, int32_t block, DevStatus* st, cudaStream_t stream) {
  if (s > kMaxS || c < 0) return cudaErrorInvalidValue;
  const size_t smem = 2 * (size_t)s * s * sizeof(double);
  cudaError_t e = ensure_dyn_smem(tail_pchol_kernel, (size_t)(smem));
  if (e != cudaSuccess) return e;
  const int slot = prof_begin(stream);
  tail_pchol_kernel<<<1, kTailThreads, smem, stream>>>(c, s, G, ldg, S_out, ldsm, Rkk, block, st);
  note_launch(1);
  prof_end(slot, kProfTail, stream, 2.0 * (double)c * s * s + (double)s * s * s / 3.0, 0.0);
  return cudaGetLastError();
}

cudaError_t launch_copy_small(int32_t rows, int32_t cols, const double* A, int32_t lda, double* B,
                              int32_t ldb, DevStatus* st, cudaStream_t stream) {
  copy_small_kernel<<<1, 256, 0, stream>>>(rows, cols, A, lda, B, ldb, st);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_r_assemble(int32_t c, int32_t s, const double* S, int32_t lds, const double* Y,
                              int32_t ldy, const double* Sd, const double* Yd, double* R,
                              int32_t ldr, int32_t col0, DevStatus* st, cudaStream_t stream) {
  const int total = (c + s) * s;
  r_assemble_kernel<<<(total + 255) / 256, 256, 0, stream>>>(c, s, S, lds, Y, ldy, Sd, Yd, R, ldr,
                                                             col0, st);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_chol(int32_t s, const double* A, int32_t lda, double* R, int32_t ldr,
                        int32_t block, DevStatus* st, cudaStream_t stream) {
  if (s > kMaxS) return cudaErrorInvalidValue;
  const size_t smem = 2 * (size_t)s * s * sizeof(double);
  cudaError_t e = ensure_dyn_smem(chol_kernel, (size_t)(smem));
  if (e != cudaSuccess) return e;
  chol_kernel<<<1, kTailThreads, smem, stream>>>(s, A, lda, R, ldr, block, st);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_zero_lower(int32_t n, double* R, int32_t ldr, cudaStream_t stream) {
  const int64_t total = (int64_t)n * n;
  int grid = (int)((total + 255) / 256);
  if (grid > 1024) grid = 1024;
  if (grid < 1) grid = 1;
  zero_kernel<<<grid, 256, 0, stream>>>(n, R, ldr);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_zero_u64(unsigned long long* p, int64_t n, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  int64_t grid = (n + 255) / 256;
  if (grid > 1024) grid = 1024;
  zero_u64_words<<<(unsigned)grid, 256, 0, stream>>>(p, n);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_set_identity(int32_t s, double* A, cudaStream_t stream) {
  identity_kernel<<<1, 256, 0, stream>>>(s, A);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_reset_status(DevStatus* st, cudaStream_t stream, DevStatus* st2) {
  reset_status_kernel<<<1, 32, 0, stream>>>(st, st2);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_merge_status(DevStatus* st, DevStatus* side, cudaStream_t stream) {
  merge_status_kernel<<<1, 32, 0, stream>>>(st, side);
  note_launch(1);
  return cudaGetLastError();
}

}  // namespace bcgs
