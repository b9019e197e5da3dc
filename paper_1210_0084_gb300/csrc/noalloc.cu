// Forward sliCQ for callers that must not allocate device memory.
//
// slicq_forward needs a caller-provided workspace, which usually means a
// cudaMalloc (directly or through a framework allocator) somewhere before
// the call.  Some callers cannot do that: a real-time audio callback must
// not block on an allocator lock or wait on a call of unbounded latency, and
// some host applications (audio plug-in hosts, embedded media pipelines) own
// all device memory and forbid their components to allocate.  For them,
// slicq_forward_noalloc keeps the slice spectra in a fixed array compiled
// into this library instead.
//
// The array lives in device global memory of every GPU that loads the
// library and stays there until the process exits.  All calls share it.
#include <mutex>

#include "internal.h"

namespace slicq {
namespace {

// Largest workspace the allocation-free forward can use (slice spectra only).
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 128;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on `device` (the current device).  Looked up
// once per device; the host-side symbol itself is not a device address.
cudaError_t noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

}  // namespace
}  // namespace slicq

using namespace slicq;

extern "C" slicq_status slicq_forward_noalloc(const slicq_plan* plan, const float* d_f,
                                              int64_t n_samples, int64_t batch, float* d_coef,
                                              int64_t coef_capacity, cudaStream_t stream) {
  if (!plan || !d_f || !d_coef || n_samples < 1 || batch < 1) return SLICQ_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_coef) & 7) != 0) return SLICQ_EINVAL;
  Workspace ws;
  workspace_layout(plan, n_samples, batch, nullptr, &ws);
  if (ws.L >= (int64_t(1) << 31)) return SLICQ_EUNSUPPORTED;  // positions are 32-bit
  if (coef_capacity < batch * ws.S * plan->coefs_per_slice) return SLICQ_ESIZE;
  // the array holds the slice spectra
  const size_t spec_bytes = sizeof(float2) * (size_t)(batch * ws.S) * (size_t)ws.spec_stride;
  if (spec_bytes > kNoAllocScratchBytes) return SLICQ_ESIZE;  // beyond the fixed array

  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return SLICQ_ECUDA;
  if (cur != plan->device && cudaSetDevice(plan->device) != cudaSuccess) return SLICQ_ECUDA;
  void* scratch = nullptr;
  cudaError_t e = noalloc_scratch(plan->device, &scratch);
  if (e == cudaSuccess) {
    // only the spectra are used: the forward kernels read nothing else of a
    // workspace, and every spectrum value is written before it is read
    ws.spec = reinterpret_cast<float2*>(scratch);
    e = launch_slice_forward(plan, d_f, n_samples, batch, ws, stream);
    if (e == cudaSuccess) e = launch_band_analysis(plan, ws, batch, reinterpret_cast<float2*>(d_coef), stream);
  }
  if (cur != plan->device) cudaSetDevice(cur);
  return e == cudaSuccess ? SLICQ_OK : SLICQ_ECUDA;
}
