// Launch counter and optional per-kernel-class event timing.
//
// Every launcher calls note_launch(); when profiling is enabled, the Gram,
// projection, TSQR and tail launchers also bracket their kernels with CUDA
// events recorded on the stream the kernels run on, together with the
// algorithmic flops and bytes of that launch.  bcgs_profile_read resolves the
// events after the caller has synchronized.
#include <atomic>
#include <mutex>
#include <vector>

#include "bcgs_internal.cuh"

namespace bcgs {

namespace {
std::atomic<int64_t> g_launches{0};
std::atomic<int> g_enabled{0};
struct Pending {
  int cls;
  cudaEvent_t a, b;
  double flops, bytes;
};
struct ClassTotals {
  int64_t launches = 0;
  double ms = 0, flops = 0, bytes = 0;
};
std::mutex g_mu;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free;
ClassTotals g_tot[kProfClasses];

cudaEvent_t get_event() {
  if (!g_free.empty()) {
    cudaEvent_t e = g_free.back();
    g_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {
struct SmemEntry {
  const void* kernel;
  int dev;
  size_t bytes;  // dynamic shared memory the kernel may launch with now
};
std::mutex g_smem_mu;
std::vector<SmemEntry> g_smem;
}  // namespace

// Without the opt-in a kernel may take 48 KB minus its static shared memory of
// dynamic shared memory; above that, raise MaxDynamicSharedMemorySize once.
cudaError_t ensure_dyn_smem_ptr(const void* kernel, size_t bytes) {
  if (bytes == 0) return cudaSuccess;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
  std::lock_guard<std::mutex> lk(g_smem_mu);
  SmemEntry* hit = nullptr;
  for (auto& e : g_smem)
    if (e.kernel == kernel && e.dev == dev) {
      hit = &e;
      break;
    }
  if (hit == nullptr) {
    cudaFuncAttributes a;
    cudaError_t err = cudaFuncGetAttributes(&a, kernel);
    if (err != cudaSuccess) return err;
    const size_t def = a.sharedSizeBytes < 48 * 1024 ? 48 * 1024 - a.sharedSizeBytes : 0;
    g_smem.push_back({kernel, dev, def});
    hit = &g_smem.back();
  }
  if (hit->bytes >= bytes) return cudaSuccess;
  cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (err != cudaSuccess) return err;
  hit->bytes = bytes;
  return cudaSuccess;
}

int prof_begin(cudaStream_t stream) {
  if (!g_enabled.load(std::memory_order_relaxed)) return -1;
  std::lock_guard<std::mutex> lk(g_mu);
  Pending p;
  p.cls = -1;
  p.a = get_event();
  p.b = get_event();
  p.flops = p.bytes = 0;
  if (!p.a || !p.b) return -1;
  cudaEventRecord(p.a, stream);
  g_pending.push_back(p);
  return (int)g_pending.size() - 1;
}

void prof_end(int slot, int cls, cudaStream_t stream, double flops, double bytes) {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (slot >= (int)g_pending.size()) return;
  Pending& p = g_pending[slot];
  p.cls = cls;
  p.flops = flops;
  p.bytes = bytes;
  cudaEventRecord(p.b, stream);
}

}  // namespace bcgs

using namespace bcgs;

extern "C" {

int64_t bcgs_launch_count(void) { return g_launches.load(); }

int bcgs_profile_enable(int enable) {
  g_enabled.store(enable ? 1 : 0);
  return BCGS_OK;
}

int bcgs_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& p : g_pending) {
    g_free.push_back(p.a);
    g_free.push_back(p.b);
  }
  g_pending.clear();
  for (auto& t : g_tot) t = ClassTotals();
  return BCGS_OK;
}

int bcgs_profile_read(int cls, int64_t* launches, double* total_ms, double* flops, double* bytes) {
  if (cls < 0 || cls >= kProfClasses) return BCGS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& p : g_pending) {
    if (p.cls >= 0) {
      float ms = 0.f;
      if (cudaEventSynchronize(p.b) != cudaSuccess) return BCGS_ERR_CUDA;
      if (cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) return BCGS_ERR_CUDA;
      ClassTotals& t = g_tot[p.cls];
      t.launches += 1;
      t.ms += ms;
      t.flops += p.flops;
      t.bytes += p.bytes;
    }
    g_free.push_back(p.a);
    g_free.push_back(p.b);
  }
  g_pending.clear();
  const ClassTotals& t = g_tot[cls];
  if (launches) *launches = t.launches;
  if (total_ms) *total_ms = t.ms;
  if (flops) *flops = t.flops;
  if (bytes) *bytes = t.bytes;
  return BCGS_OK;
}

}  // extern "C"
