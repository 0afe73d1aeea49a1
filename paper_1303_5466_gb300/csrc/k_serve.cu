// k_serve.cu -- job-list kernels of the serving scheduler: one launch carries the same stage
// of the inverse apply for every in-flight request, whatever its operator, level or nrhs.
// The per-request arithmetic is that of the per-level kernels (shared matvec body, same copy
// and axpby expressions), so a request's result does not depend on its batch.
#include "k_matvec.cuh"

namespace rs {

// Last job whose start (member `start`) is <= t; jobs are sorted by start.
template <class J>
__device__ __forceinline__ int find_job(const J* __restrict__ jobs, int nj, int64_t t, int64_t J::*start)
{
    int lo = 0, hi = nj - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].*start <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) mv_jobs_kernel(const MvJob* __restrict__ jobs, int nj)
{
    __shared__ double part[256 * 8];
    const int64_t t = blockIdx.x;
    const int j = find_job(jobs, nj, t, &MvJob::blk_start);
    const MvJob J = jobs[j];
    const int64_t lt = t - J.blk_start;
    const int pi = find_block(J.blk0, J.np, lt);
    const MatvecProb P = J.probs[pi];
    const int row0 = (int)(lt - J.blk0[pi]) * J.rb;
    const double* A = J.A + P.a_off;
    const double* x = J.x + P.x_off * J.nrhs;
    double* y = J.y + P.y_off * J.nrhs;
    if (J.rb == 16) matvec_block<double, 16>(P, row0, A, x, y, J.nrhs, part);
    else if (J.rb == 32) matvec_block<double, 32>(P, row0, A, x, y, J.nrhs, part);
    else matvec_block<double, 64>(P, row0, A, x, y, J.nrhs, part);
}

__global__ void __launch_bounds__(256) copy_jobs_kernel(const CopyJob* __restrict__ jobs, int nj, int64_t total)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int j = find_job(jobs, nj, e, &CopyJob::e_start);
    const CopyJob J = jobs[j];
    const int64_t l = e - J.e_start;
    if (J.mode == COPY_AXPBY) {
        J.out[l] = fma(J.a, J.in[l], J.b * J.out[l]);
        return;
    }
    const int64_t p = l / J.nrhs;
    const int c = (int)(l - p * J.nrhs);
    switch (J.mode) {
        case COPY_GATHER_ROWS: J.out[l] = J.in[J.idx[p] * J.nrhs + c]; break;
        case COPY_SCATTER_ROWS: J.out[J.idx[p] * J.nrhs + c] = J.in[l]; break;
        case COPY_GATHER_CM: J.out[l] = J.in[(int64_t)c * J.N + J.idx[p]]; break;
        default: J.out[(int64_t)c * J.N + J.idx[p]] = J.in[l]; break;   // COPY_SCATTER_CM
    }
}

cudaError_t launch_mv_jobs(cudaStream_t st, const MvJob* jobs, int nj, int64_t blocks)
{
    if (nj <= 0 || blocks <= 0) return cudaSuccess;
    count_launches(1);
    mv_jobs_kernel<<<(unsigned)blocks, 256, 0, st>>>(jobs, nj);
    return cudaGetLastError();
}

cudaError_t launch_copy_jobs(cudaStream_t st, const CopyJob* jobs, int nj, int64_t total)
{
    if (nj <= 0 || total <= 0) return cudaSuccess;
    count_launches(1);
    copy_jobs_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(jobs, nj, total);
    return cudaGetLastError();
}

}  // namespace rs
