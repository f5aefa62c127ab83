// poisson_selftest_wait: exercises the bounded mbarrier wait of the solve kernels and the
// plan's status word without a fault, a trap or a hang.
#include <cuda_runtime.h>

#include "../../include/poisson.h"
#include "solver.h"
#include "tma.cuh"

namespace {

// One thread waits on an mbarrier that expects one arrival and never gets it; the wait
// gives up after `polls` polls, records the timeout bit in *status and the kernel returns.
__global__ void k_wait_selftest(int *status, long long polls) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    gsp::mbar_init(&bar, 1);
    gsp::fence_mbar_init();
    gsp::mbar_wait(&bar, 0, status, polls);
}

}  // namespace

namespace gsp {
cudaError_t launch_wait_selftest(const DevicePlan &p, long long polls, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(p.status, polls);
    return cudaGetLastError();
}
}  // namespace gsp
