// bcgs_gram_noalloc: the Gram product C = A^T B for callers that cannot hand the
// library any device memory of its own.
//
// Some callers cannot call cudaMalloc or provide a workspace: a host framework
// that owns every device allocation through its own pool (an allocation made
// behind its back fragments or exhausts that pool, and cudaMalloc / cudaFree may
// synchronize the device), or a latency-bound loop that must not reach the
// allocator at all once it is running.  For them the chunk partial sums of the
// Gram reduction live in a fixed array compiled into the library instead of in
// a caller workspace.  The array is allocated when the library's device code is
// loaded on a GPU and every GPU that loads the library keeps it until the process
// exits.
#include <string.h>

#include <mutex>

#include "bcgs_internal.cuh"

namespace bcgs {
namespace {

// The array: 2^20 doubles (8 MiB) of chunk partials, then 65544 words for the
// column maxima of the tensor-core engine (ka * kb <= 65536 implies
// ka + kb <= 65537).
constexpr size_t kNoAllocPartials = BCGS_GRAM_NOALLOC_MAX_PARTIALS;
constexpr size_t kNoAllocAmax = 65544;

static __device__ __align__(256) double g_gram_partials[kNoAllocPartials + kNoAllocAmax];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double* g_partials_ptr[kMaxDevices] = {nullptr};

// Device address of g_gram_partials on the current device, looked up once per
// device.  In host code the symbol g_gram_partials names a host-side shadow, not
// device memory, so it must never be passed to a kernel directly.  The address
// is kept for the life of the process: after cudaDeviceReset (or anything else
// that rebuilds the device's context) it is stale, so the entry point must not be
// used across such a reset.
int partials_on_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BCGS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (g_partials_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_gram_partials) != cudaSuccess || p == nullptr)
      return BCGS_ERR_CUDA;
    g_partials_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_ptr[dev];
  return BCGS_OK;
}

}  // namespace
}  // namespace bcgs

using namespace bcgs;

extern "C" int bcgs_gram_noalloc(int64_t m, int32_t ka, int32_t kb, const double* A, int64_t lda,
                                 const double* B, int64_t ldb, double* C, int32_t ldc,
                                 void* stream) {
  if (m < 1 || ka < 1 || kb < 1 || (int64_t)ka * kb > 65536) return BCGS_ERR_INVALID_ARG;
  if (!A || !B || !C || lda < m || ldb < m || ldc < ka) return BCGS_ERR_INVALID_ARG;
  GramDesc d;
  memset(&d, 0, sizeof(d));
  d.a[0].p = A;
  d.a[0].ld = lda;
  d.a[0].ncols = ka;
  d.b[0].p = B;
  d.b[0].ld = ldb;
  d.b[0].ncols = kb;
  d.nsa = d.nsb = 1;
  d.na = ka;
  d.nb = kb;
  d.m = m;
  gram_partition(m, &d.chunk_rows, &d.nchunks);
  // Every partial slot of this call is written before it is read (a CTA of the
  // tensor engine that meets a non-finite column or a wait that runs out writes
  // NaN into its slots), so the array needs no clearing between calls and a
  // failure shows as NaN in C, never as an earlier call's sums.  Sizes beyond the
  // array's capacity are refused.
  if ((size_t)d.nchunks * (size_t)ka * (size_t)kb > kNoAllocPartials) return BCGS_ERR_WORKSPACE;
  double* partials = nullptr;
  const int rc = partials_on_current_device(&partials);
  if (rc != BCGS_OK) return rc;
  // No status word: a null status pointer makes the kernels skip the check;
  // non-finite input and a timed-out wait come back as NaN entries of C.
  cudaError_t e;
  if (use_tensor_gram(d)) {
    auto* amax = reinterpret_cast<unsigned long long*>(partials + kNoAllocPartials);
    e = launch_gram_tc(d, partials, C, ldc, amax, nullptr, reinterpret_cast<cudaStream_t>(stream));
  } else {
    e = launch_gram(d, partials, C, ldc, nullptr, reinterpret_cast<cudaStream_t>(stream));
  }
  return e == cudaSuccess ? BCGS_OK : BCGS_ERR_CUDA;
}
