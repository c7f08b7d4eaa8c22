// A check of the failure path of the bounded waits, runnable on any GPU.
//
// Every mbarrier wait of the fused kernels gives up after a time limit, sets
// a bit in the grid's error word and returns, so that a copy that never
// lands is reported (TS_ERR_TIMEOUT at the next syncing call) instead of
// hanging the GPU.  This kernel runs the same bounded wait on an mbarrier
// that nothing completes -- no copy is in flight and nothing else waits --
// and takes the same error path, so a host can see that path work without
// any fault: the wait runs out after limit_ns and the kernel returns.
#include "internal.h"
#include "mbar.cuh"

namespace ts {

namespace {

__global__ void wait_timeout_kernel(uint64_t limit_ns, int *err)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);   // one arrival expected; none ever comes
        fence_mbar_init();
    }
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0, limit_ns);
    if (!__all_sync(0xffffffffu, ok) && threadIdx.x == 0) atomicOr(err, ERRBIT_WAIT_TIMEOUT);
}

}  // namespace

cudaError_t launch_wait_timeout_check(int *err, uint64_t limit_ns, cudaStream_t st)
{
    wait_timeout_kernel<<<1, 32, 0, st>>>(limit_ns, err);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace ts
