// Projection plus triangular-solve normalization
//     W = (V - Q C) T^{-1}
// (Alg. 1 and Alg. 2: U_{k+1} = (X_{k+1} - Q_k S_{1:k,k+1}) S_{k+1,k+1}^{-1} and
//  Q_{k+1} = (U_{k+1} - Q_k Y_{1:k,k+1}) Y_{k+1,k+1}^{-1}).
//
// Row-local: row r of W needs only row r of V and Q.  One thread owns one row;
// a warp reads 32 consecutive rows of each column of Q (coalesced), C is staged
// through shared memory in chunks, and the s-wide triangular solve runs in
// registers by forward substitution over columns.
#include "bcgs_internal.cuh"

namespace bcgs {

namespace {

constexpr int kProjThreads = 128;

template <typename T>
__device__ __forceinline__ double ldv(const void* p, int64_t i) {
  return (double)__ldg(reinterpret_cast<const T*>(p) + i);
}
template <typename T>
__device__ __forceinline__ void stv(void* p, int64_t i, double v) {
  reinterpret_cast<T*>(p)[i] = (T)v;
}

// Column maxima of the written W (one warp max and atomic per column and warp).
template <typename T, int S>
__device__ __forceinline__ void column_max_out(const ProjDesc& d, const double* w, bool live) {
  if (d.wmax.col == nullptr) return;
#pragma unroll
  for (int j = 0; j < S; ++j)
    if (j < d.s) warp_max_to(live ? abs_bits64((double)(T)w[j]) : 0ull, d.wmax.col + j);
}

template <typename T, int S>
__global__ void __launch_bounds__(kProjThreads)
project_kernel(ProjDesc d, const DevStatus* st) {
  // rows of C staged per pass (keeps static shared memory under 48 KB)
  constexpr int kCChunk = S >= 64 ? 16 : 64;
  if (failed(st)) return;
  __shared__ double Cs[kCChunk * S];
  __shared__ double Ts[S * S];
  const int s = d.s;
  const int c = d.q.ncols;
  const int64_t r = (int64_t)blockIdx.x * kProjThreads + threadIdx.x;
  const bool live = r < d.m;

  double acc[S];
#pragma unroll
  for (int j = 0; j < S; ++j) acc[j] = 0.0;

  for (int i0 = 0; i0 < c; i0 += kCChunk) {
    const int ni = min(kCChunk, c - i0);
    __syncthreads();
    for (int e = threadIdx.x; e < ni * s; e += kProjThreads) {
      const int i = e % ni, j = e / ni;
      Cs[i * S + j] = d.C[(i0 + i) + (int64_t)j * d.ldc];
    }
    __syncthreads();
    if (live) {
      for (int i = 0; i < ni; ++i) {
        const double q = ldv<T>(d.q.p, r + (int64_t)(i0 + i) * d.q.ld);
#pragma unroll
        for (int j = 0; j < S; ++j)
          if (j < s) acc[j] = fma(q, Cs[i * S + j], acc[j]);
      }
    }
  }
  if (d.T != nullptr) {
    __syncthreads();
    for (int e = threadIdx.x; e < s * s; e += kProjThreads) {
      const int i = e % s, j = e / s;
      Ts[i * S + j] = d.T[i + (int64_t)j * d.ldt];
    }
    __syncthreads();
  }
  double* w = acc;  // reuse the registers: w_j = v_j - (Q C)_j
  if (live) {
#pragma unroll
    for (int j = 0; j < S; ++j) {
      if (j < s) w[j] = ldv<T>(d.v.p, r + (int64_t)j * d.v.ld) - acc[j];
    }
    if (d.T != nullptr) {
      // w T^{-1}: w_j = (v_j - sum_{l<j} w_l t_lj) / t_jj
#pragma unroll
      for (int j = 0; j < S; ++j) {
        if (j < s) {
          double x = w[j];
#pragma unroll
          for (int l = 0; l < S; ++l)
            if (l < j) x = fma(-w[l], Ts[l * S + j], x);
          w[j] = x / Ts[j * S + j];
        }
      }
    }
#pragma unroll
    for (int j = 0; j < S; ++j)
      if (j < s) stv<T>(d.w, r + (int64_t)j * d.ldw, w[j]);
    if (d.wmax.row != nullptr) {
      unsigned long long mx = 0ull;
#pragma unroll
      for (int j = 0; j < S; ++j)
        if (j < s) mx = umax64(mx, abs_bits64((double)(T)w[j]));
      d.wmax.row[r] = umax64(d.wmax.row[r], mx);
    }
  }
  // every thread of the warp takes part in the column maxima (dead rows give 0)
  column_max_out<T, S>(d, w, live);
}

template <typename T>
cudaError_t launch_t(const ProjDesc& d, DevStatus* st, cudaStream_t stream) {
  const unsigned grid = (unsigned)ceil_div(d.m, kProjThreads);
  if (grid == 0) return cudaSuccess;
  const int slot = prof_begin(stream);
#define BCGS_PROJ_CASE(SV) \
  if (d.s <= SV) { project_kernel<T, SV><<<grid, kProjThreads, 0, stream>>>(d, st); } else
  BCGS_PROJ_CASE(1) BCGS_PROJ_CASE(2) BCGS_PROJ_CASE(4) BCGS_PROJ_CASE(8) BCGS_PROJ_CASE(16)
  BCGS_PROJ_CASE(32) BCGS_PROJ_CASE(64) { return cudaErrorInvalidValue; }
#undef BCGS_PROJ_CASE
  prof_end(slot, kProfProject, stream, 2.0 * (double)d.m * d.q.ncols * d.s + (double)d.m * d.s * d.s,
           (double)d.m * (d.q.ncols + 2.0 * d.s) * sizeof(T));
  note_launch(1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_project(const ProjDesc& d, DevStatus* st, cudaStream_t stream) {
  return d.w_fp32 ? launch_t<float>(d, st, stream) : launch_t<double>(d, st, stream);
}

}  // namespace bcgs
