// map_smoother_wait_selftest: the device-error path of the solve kernels
// exercised without a fault or a hang.  One CTA waits on a shared-memory
// mbarrier that nothing arrives on (the poll-limited wait of the bulk copies)
// and on a grid-barrier counter that nothing advances (the spin-limited wait of
// the single-launch solves); both run out, and each is reported through
// report_event exactly as in a solve.
#include <cuda_runtime.h>

#include "scan.cuh"
#include "handle.h"

namespace {

__global__ void __launch_bounds__(32) k_wait_selftest(unsigned long long* stats, int polls)
{
    using namespace mapk;
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    // no arrival and no transaction is ever posted on this barrier
    const bool ok = mbar_wait_bounded(&bar, 0, polls);
    if (!__syncthreads_and(ok) && threadIdx.x == 0) report_event(stats, EV_TIMEOUT);
    // a barrier target that the one CTA cannot reach (its own arrival adds 1)
    const GridSync gs{stats + EV_SELFTEST, ~0ull >> 1};
    grid_sync(gs, 1, stats, polls);
}

}  // namespace

extern "C" map_status map_smoother_wait_selftest(map_smoother* h, int polls, void* stream)
{
    if (!h) return MAP_ERR_INVALID_ARG;
    if (polls < 1 || polls > (1 << 20)) return mapk::fail(*h, MAP_ERR_INVALID_ARG, "polls must be 1..1048576");
    k_wait_selftest<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(h->d_stats, polls);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mapk::cuda_fail(*h, e, "wait self-test launch");
    return MAP_OK;
}
