// watchdog.cu -- self-test of the bounded device waits.
//
// Every wait inside the library's kernels (the mbarrier waits of the
// tcgen05 update) is bounded in SM clock cycles; when a bound runs out the
// kernel records kStTimeout in the plan's status word and returns, and the
// host reports PEVC_ERR_TIMEOUT with the context still usable.  This kernel
// runs one such wait on an mbarrier whose only arrival can be withheld, so
// that the timeout path is exercised without any fault, trap or endless loop:
// with the arrival withheld the wait gives up after `cycles` clock cycles.
#include "common.cuh"
#include "tc.cuh"

namespace pevc {

namespace {

__global__ void k_watchdog_probe(unsigned* __restrict__ status, int withhold, long long cycles) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!withhold) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(&bar)));
    if (!mbar_wait_cycles(&bar, 0u, cycles)) atomicOr(status, kStTimeout);
  }
}

}  // namespace

cudaError_t launch_watchdog_probe(unsigned* status, int withhold, long long cycles, cudaStream_t s) {
  k_watchdog_probe<<<1, 32, 0, s>>>(status, withhold, cycles);
  return cudaGetLastError();
}

}  // namespace pevc
