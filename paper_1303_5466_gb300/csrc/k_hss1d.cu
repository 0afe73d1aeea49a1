// k_hss1d.cu -- kernels of the extra compression of Sec. 3 (HSS1D and low-rank forms of the
// large blocks), built from the explicit dense blocks:
//   zgather   : the ID input of every node of a batch -- for an HSS1D node the block column
//               and the transposed block row against every index outside the node, stacked;
//               for a low-rank block the block itself (Sec. 3.2, Eq. 2.9);
//   subgather : dense sub-blocks M(rows, cols) into the compressed store (sibling blocks,
//               leaf blocks, the skeleton columns of a low-rank block);
//   copy_rows : the row moves between the inverse apply's vectors and the apply scratch.
// The IDs themselves run in the column-pivoted QR and T kernels of the factorization.
#include <algorithm>

#include "k_common.cuh"

namespace rs {

template <class T>
__global__ void __launch_bounds__(256) zgather_kernel(const ZProb* __restrict__ probs, const int32_t* __restrict__ lists,
                                                      T* __restrict__ Y)
{
    const ZProb P = probs[blockIdx.y];
    const T* __restrict__ M = (const T*)P.M;
    const int r = P.mode == 0 ? 2 * P.nout : P.nout;
    const int64_t total = (int64_t)r * P.a;
    const int32_t* __restrict__ act = lists + P.act_off;
    const int32_t* __restrict__ out = lists + P.out_off;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / r), i = (int)(e - (int64_t)j * r);
        T v;
        if (P.mode == 1) v = M[(int64_t)i + (int64_t)act[j] * P.ld];
        else if (i < P.nout) v = M[(int64_t)out[i] + (int64_t)act[j] * P.ld];
        else v = M[(int64_t)act[j] + (int64_t)out[i - P.nout] * P.ld];
        Y[P.y_off + e] = v;
    }
}

template <class T>
__global__ void __launch_bounds__(256) subgather_kernel(const SubProb* __restrict__ probs,
                                                        const int32_t* __restrict__ lists, T* __restrict__ dst)
{
    const SubProb P = probs[blockIdx.y];
    const T* __restrict__ M = (const T*)P.M;
    const int64_t total = (int64_t)P.rows * P.cols;
    const int32_t* __restrict__ ri = P.row_off >= 0 ? lists + P.row_off : nullptr;
    const int32_t* __restrict__ ci = lists + P.col_off;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / P.rows), i = (int)(e - (int64_t)j * P.rows);
        const int64_t row = ri ? ri[i] : i;
        dst[P.dst_off + e] = M[row + (int64_t)ci[j] * P.ld];
    }
}

// out[dst[p] * nrhs + c] = in[src[p] * nrhs + c]  (add: +=); the dst rows of one launch are
// distinct.
template <class T>
__global__ void copy_rows_kernel(int64_t count, const int64_t* __restrict__ src, const int64_t* __restrict__ dst,
                                 const T* __restrict__ in, T* __restrict__ out, int nrhs, int add)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count * nrhs) return;
    const int64_t p = e / nrhs;
    const int c = (int)(e - p * nrhs);
    const T v = in[src[p] * nrhs + c];
    T* o = out + dst[p] * nrhs + c;
    *o = add ? *o + v : v;
}

static unsigned grid_x(int64_t maxel)
{
    const int64_t b = (maxel + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 1024));
}

template <class T>
cudaError_t launch_zgather(cudaStream_t st, const ZProb* probs, int np, const int32_t* lists, T* Y, int64_t max_el)
{
    if (np <= 0 || max_el <= 0) return cudaSuccess;
    count_launches(1);
    zgather_kernel<T><<<dim3(grid_x(max_el), (unsigned)np), 256, 0, st>>>(probs, lists, Y);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_subgather(cudaStream_t st, const SubProb* probs, int np, const int32_t* lists, T* dst,
                             int64_t max_el)
{
    if (np <= 0 || max_el <= 0) return cudaSuccess;
    count_launches(1);
    subgather_kernel<T><<<dim3(grid_x(max_el), (unsigned)np), 256, 0, st>>>(probs, lists, dst);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_copy_rows(cudaStream_t st, int64_t count, const int64_t* src, const int64_t* dst, const T* in, T* out,
                             int nrhs, int add)
{
    if (count <= 0) return cudaSuccess;
    count_launches(1);
    copy_rows_kernel<T><<<(unsigned)((count * nrhs + 255) / 256), 256, 0, st>>>(count, src, dst, in, out, nrhs, add);
    return cudaGetLastError();
}

#define RS_INST_HSS(T)                                                                                             \
    template cudaError_t launch_zgather<T>(cudaStream_t, const ZProb*, int, const int32_t*, T*, int64_t);        \
    template cudaError_t launch_subgather<T>(cudaStream_t, const SubProb*, int, const int32_t*, T*, int64_t);    \
    template cudaError_t launch_copy_rows<T>(cudaStream_t, int64_t, const int64_t*, const int64_t*, const T*, T*, \
                                             int, int);
RS_INST_HSS(double)
RS_INST_HSS(float)
RS_INST_HSS(cplx<double>)
RS_INST_HSS(cplx<float>)

}  // namespace rs
