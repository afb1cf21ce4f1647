// selftest.cu -- the failure path of the library's bounded device waits, exercised
// without a fault: one thread waits on an mbarrier that nothing arrives on, gives up
// after a short limit, and records the timeout in the device status word exactly as
// the product kernels do when a TMA copy or an MMA never completes.  The host then
// reports CHASE_ERR_TIMEOUT and the CUDA context stays usable.
#include "common.cuh"
#include "kernels.h"

namespace chase {

namespace {

__global__ void wait_timeout_kernel(long long limit_cycles, DevStatus* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  // phase 0 needs one arrival, which never comes: the wait must run out
  const long long t0 = clock64();
  bool done = false;
  while (!done) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(b)
        : "memory");
    done = ok != 0;
    if (!done && clock64() - t0 > limit_cycles) break;
  }
  if (!done) atomicOr(&status->timeout, 16);
}

}  // namespace

int selftest_wait_timeout(cudaStream_t st, double seconds, DevStatus* dst, int* launches) {
  int dev = 0, khz = 0;
  CHASE_CUDA_TRY(cudaGetDevice(&dev));
  CHASE_CUDA_TRY(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
  const long long limit = (long long)(seconds * (double)khz * 1e3);
  wait_timeout_kernel<<<1, 32, 0, st>>>(limit > 0 ? limit : 1, dst);
  if (launches) ++*launches;
  CHASE_CUDA_TRY(cudaGetLastError());
  return 0;
}

}  // namespace chase
