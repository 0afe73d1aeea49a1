// k_krylov.cu -- vector kernels of the preconditioned BiCGstab (Sec. 5.4): conjugated dot
// products with a fixed summation order (per-block partial sums, then one block adds them),
// and the three-term linear combinations of the recurrence.
#include <algorithm>

#include "k_common.cuh"

namespace rs {

constexpr int KR_NT = 256;
constexpr int KR_BLOCKS = 608;          // 4 per SM on 152 SMs; partial sums per dot product

template <class T>
__global__ void __launch_bounds__(KR_NT) dot_partial_kernel(int64_t n, const T* __restrict__ a,
                                                           const T* __restrict__ b, T* __restrict__ part)
{
    __shared__ T red[KR_NT];
    T s = 0;
    for (int64_t i = (int64_t)blockIdx.x * KR_NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * KR_NT)
        s = fma_(conj_(a[i]), b[i], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = KR_NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

template <class T>
__global__ void __launch_bounds__(KR_NT) dot_final_kernel(int np, const T* __restrict__ part, T* __restrict__ out)
{
    __shared__ T red[KR_NT];
    T s = 0;
    for (int i = threadIdx.x; i < np; i += KR_NT) s = s + part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = KR_NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// y = c0 x0 + c1 x1 + c2 x2 (x1, x2 may be NULL; any of them may be y)
template <class T>
__global__ void __launch_bounds__(KR_NT) lincomb_kernel(int64_t n, T c0, const T* x0, T c1, const T* x1, T c2,
                                                        const T* x2, T* y)
{
    for (int64_t i = (int64_t)blockIdx.x * KR_NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * KR_NT) {
        T v = c0 * x0[i];
        if (x1) v = fma_(c1, x1[i], v);
        if (x2) v = fma_(c2, x2[i], v);
        y[i] = v;
    }
}

template <class T>
cudaError_t launch_dot(cudaStream_t st, int64_t n, const T* a, const T* b, T* part, T* out)
{
    count_launches(2);
    dot_partial_kernel<T><<<KR_BLOCKS, KR_NT, 0, st>>>(n, a, b, part);
    dot_final_kernel<T><<<1, KR_NT, 0, st>>>(KR_BLOCKS, part, out);
    return cudaGetLastError();
}

int dot_partials() { return KR_BLOCKS; }

template <class T>
cudaError_t launch_lincomb(cudaStream_t st, int64_t n, T c0, const T* x0, T c1, const T* x1, T c2, const T* x2,
                           T* y)
{
    if (n <= 0) return cudaSuccess;
    count_launches(1);
    const int64_t want = (n + KR_NT - 1) / KR_NT;
    lincomb_kernel<T><<<(unsigned)std::min<int64_t>(want, 8 * KR_BLOCKS), KR_NT, 0, st>>>(n, c0, x0, c1, x1, c2,
                                                                                           x2, y);
    return cudaGetLastError();
}

#define RS_INST_KR(T)                                                                                  \
    template cudaError_t launch_dot<T>(cudaStream_t, int64_t, const T*, const T*, T*, T*);           \
    template cudaError_t launch_lincomb<T>(cudaStream_t, int64_t, T, const T*, T, const T*, T, const T*, T*);
RS_INST_KR(double)
RS_INST_KR(cplx<double>)

}  // namespace rs
