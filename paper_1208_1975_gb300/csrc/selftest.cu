// Diagnostic: exercises the bounded device-side wait used by the TMA-ring kernels and the
// sticky status path, without any fault: one CTA waits on an mbarrier that nothing ever
// arrives on, gives up after `limit_ns`, records BRS_ERR_TIMEOUT and returns normally.
#include "brs_internal.cuh"

namespace {

__global__ void wait_unsignalled_kernel(unsigned long long limit_ns, int* status)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
    if (!ok && threadIdx.x == 0)
        set_status(status, BRS_ERR_TIMEOUT);
}

}  // namespace

extern "C" int brsmooth_selftest_wait(brs_ctx* c, long long limit_ns, void* stream)
{
    cudaGetLastError();
    if (!c || !c->dev_status || limit_ns < 0 || limit_ns > 1000000000ll)
        return BRS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    c->last_stream = s;
    wait_unsignalled_kernel<<<1, 32, 0, s>>>((unsigned long long)limit_ns, c->dev_status);
    return brs_cuda_status(cudaGetLastError());
}
