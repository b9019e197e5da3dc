// Self-test of the bounded device waits: one CTA waits, with the same wait
// the split-precision band kernels use for their tensor-core products, on
// an mbarrier that nothing completes.  The wait gives up after the given
// number of SM clocks and the kernel reports it; nothing faults or hangs.
#include "internal.h"
#include "tc_dft.cuh"

namespace {

__global__ void wait_timeout_kernel(long long limit, int* gave_up) {
  __shared__ __align__(8) unsigned long long bar;
  const uint32_t addr = slicq::smem_addr(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(addr) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  // nothing arrives on the barrier: phase 0 never completes
  const bool done = threadIdx.x == 0 && slicq::tc_wait(addr, 0, limit);
  if (__syncthreads_or(done) == 0 && threadIdx.x == 0) *gave_up = 1;
}

}  // namespace

extern "C" slicq_status slicq_selftest_wait(int device, int64_t limit_cycles) {
  if (limit_cycles < 1) return SLICQ_EINVAL;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return SLICQ_ECUDA;
  if (cur != device && cudaSetDevice(device) != cudaSuccess) return SLICQ_ECUDA;
  int* d = nullptr;
  int h = 0;
  slicq_status st = SLICQ_ECUDA;
  if (cudaMalloc(&d, sizeof(int)) == cudaSuccess && cudaMemset(d, 0, sizeof(int)) == cudaSuccess) {
    wait_timeout_kernel<<<1, 128>>>((long long)limit_cycles, d);
    if (cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess &&
        cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess)
      st = h ? SLICQ_ETIMEOUT : SLICQ_OK;
  }
  cudaFree(d);
  if (cur != device) cudaSetDevice(cur);
  return st;
}
