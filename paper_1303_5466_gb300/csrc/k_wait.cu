// k_wait.cu -- a check of the bounded device-side waits: one CTA enters the group barrier the
// cooperative kernels use (CPQR, the sweep), with a target that needs two arrivals, so the
// wait can only end by its iteration limit.  It must come back with DEV_TIMEOUT in the status
// word, the kernel must return, and the context must stay usable.
#include "k_common.cuh"
#include "rs.h"
#include "rs_host.h"

namespace rs {

__global__ void __launch_bounds__(32) wait_check_kernel(unsigned int* ctr, int* status, long long limit)
{
    // one arrival (this CTA) against a target of two: nothing else ever arrives
    group_sync(ctr, 2u, status, limit);
}

cudaError_t launch_wait_check(cudaStream_t st, unsigned int* ctr, int* status, long long limit)
{
    count_launches(1);
    wait_check_kernel<<<1, 32, 0, st>>>(ctr, status, limit);
    return cudaGetLastError();
}

}  // namespace rs

using namespace rs;

extern "C" int rs_wait_check(int64_t limit, void* stream)
{
    if (limit < 1) return fail(RS_E_INVALID, "limit must be >= 1");
    const cudaStream_t st = (cudaStream_t)stream;
    DevMem ctr, status;
    RS_CUDA(ctr.alloc(sizeof(unsigned int)));
    RS_CUDA(status.alloc(sizeof(int)));
    RS_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(unsigned int), st));
    RS_CUDA(cudaMemsetAsync(status.p, 0, sizeof(int), st));
    RS_CUDA(launch_wait_check(st, ctr.as<unsigned int>(), status.as<int>(), (long long)limit));
    RS_CUDA(cudaStreamSynchronize(st));
    int s = 0;
    RS_CUDA(cudaMemcpy(&s, status.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (s & DEV_TIMEOUT) return fail(RS_E_TIMEOUT, "the device-side wait ended by its iteration limit");
    return fail(RS_E_CUDA, "a wait that cannot complete returned without DEV_TIMEOUT");
}
