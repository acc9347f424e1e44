// Failure-path self-test of the bounded waits: one thread waits on an
// mbarrier that nothing arrives on, for `budget` SM clock cycles, then
// records CWTH_ERR_TIMEOUT in the status word exactly as direct_mma_kernel
// does when a TMA or MMA stage never completes.  The wait is bounded, so
// nothing faults or hangs; the host reads the word through cwth_sync.
#include "cwth_internal.h"
#include "sm100.cuh"

namespace cwth {
namespace {

__global__ void wait_selftest_kernel(int* status, long long budget) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        sm100::mbar_init(&bar, 1);
        sm100::fence_mbar_init();
        if (!sm100::mbar_wait(&bar, 0, budget)) atomicExch(status, (int)CWTH_ERR_TIMEOUT);
    }
}

}  // namespace

cudaError_t direct_wait_selftest(int* status, long long budget, cudaStream_t st) {
    wait_selftest_kernel<<<1, 32, 0, st>>>(status, budget);
    return cudaGetLastError();
}

}  // namespace cwth
