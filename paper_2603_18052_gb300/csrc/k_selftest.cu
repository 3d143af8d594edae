// Failure-detection self test: a bounded wait that runs out (see
// lb_selftest_wait_timeout in lb.h).  The wait is the one the tensor-core
// kernels use on their mbarriers: try_wait in a loop with a clock64 limit.
#include "lb_internal.cuh"

#include <cstdint>

namespace lb {
namespace {

__global__ void selftest_wait_kernel(long long cycles, unsigned int* err) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  // phase 0 never completes: nothing arrives on the barrier
  const long long t0 = clock64();
  bool done = false;
  while (!done) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(b), "r"(0u)
        : "memory");
    done = ok != 0;
    if (!done && clock64() - t0 > cycles) break;
  }
  if (!done) atomicOr(err, ERR_TIMEOUT);
}

}  // namespace
}  // namespace lb

extern "C" lb_status lb_selftest_wait_timeout(lb_ctx* c, long long cycles, void* stream) {
  if (c == nullptr) return LB_EINVAL;
  if (cycles < 1000) cycles = 1000;
  if (cycles > 4000000000LL) cycles = 4000000000LL;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  lb::count_launch();
  lb::selftest_wait_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(cycles, c->err_dev);
  const cudaError_t e = cudaGetLastError();
  if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
  return e == cudaSuccess ? LB_OK : LB_ECUDA;
}
