// Test hooks for the fault paths, exercised without faulting the GPU: a bounded device-side
// wait that runs out (an mbarrier that nothing arrives at) and reports through the context's
// status word, and host-side injection of workspace allocation failures.
#include "ozg_context.h"
#include "ozg_device.cuh"

namespace ozg {
namespace {

// One thread waits on an mbarrier that no thread arrives at.  The wait is bounded at `limit`
// clock cycles; when it runs out the thread raises the timeout status (sticky until ozg_sync),
// as every wait of the GEMM kernels does, and the kernel returns normally.
__global__ void debug_wait_kernel(int* status, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
    const long long t0 = clock64();
    while (!mbar_try_wait(&bar, 0)) {
      if (clock64() - t0 > limit) {
        atomicExch(status, kDevTimeout);
        break;
      }
    }
  }
}

}  // namespace
}  // namespace ozg

extern "C" int ozg_debug_wait(ozg_ctx* c, long long cycles) {
  if (!c || cycles < 1000 || cycles > 4000000000ll) return OZG_ERR_INVALID;
  cudaSetDevice(c->device);
  { ozg::debug_wait_kernel<<<1, 32, 0, c->stream>>>(c->dflags, cycles); ozg::note_launch(); }
  return cudaGetLastError() == cudaSuccess ? OZG_OK : OZG_ERR_CUDA;
}

extern "C" int ozg_debug_fail_allocs(ozg_ctx* c, int n) {
  if (!c || n < 0) return OZG_ERR_INVALID;
  c->fail_allocs = n;
  return OZG_OK;
}
