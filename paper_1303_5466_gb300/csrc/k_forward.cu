// k_forward.cu -- the block products of the forward apply y = A x through the HSS form the
// factorization's IDs define: y(rows) += A(rows, cols) x(cols) for many (rows, cols) point
// lists at once, the entries generated on the fly (offset table or kernel formula, the
// diagonal where a row and a column are the same grid point).  Used for the leaves' diagonal
// blocks A(I_i, I_i) and, at every level, the two children's mutual blocks A(sk_c1, sk_c2)
// and A(sk_c2, sk_c1); nothing of A is stored.
#include "k_entry.cuh"

namespace rs {

// One block: KB_RB rows of one problem, 256 / KB_RB column phases, right-hand sides in chunks
// of KB_NC; the phases' partial sums are added in a fixed order.
constexpr int KB_RB = 64;
constexpr int KB_NC = 4;

template <class T>
__global__ void __launch_bounds__(256) kblock_mv_kernel(const KbProb* __restrict__ probs,
        const int64_t* __restrict__ blk0, int np, const int32_t* __restrict__ pts,
        const T* __restrict__ x, T* __restrict__ y, int nrhs, KernelK K, const double* __restrict__ a)
{
    constexpr int PH = 256 / KB_RB;
    __shared__ T part[256 * KB_NC];
    int lo = 0, hi = np - 1;
    const int64_t bid = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (blk0[mid] <= bid) lo = mid; else hi = mid - 1;
    }
    const KbProb P = probs[lo];
    const int orow0 = (int)(bid - blk0[lo]) * KB_RB;
    const int ri = threadIdx.x % KB_RB, cj = threadIdx.x / KB_RB;
    const int i = orow0 + ri;
    const int g = i < P.rows ? pts[P.r_off + i] : 0;
    for (int c0 = 0; c0 < nrhs; c0 += KB_NC) {
        const int nc = min(KB_NC, nrhs - c0);
        T acc[KB_NC];
#pragma unroll
        for (int c = 0; c < KB_NC; ++c) acc[c] = 0;
        if (i < P.rows) {
            for (int j = cj; j < P.cols; j += PH) {
                const int gp = pts[P.c_off + j];
                const T e = (g == gp) ? kdiag<T>(K, a, g) : kentry<T>(K, g, gp);
                const T* xp = x + (P.x_off + j) * nrhs + c0;
#pragma unroll
                for (int c = 0; c < KB_NC; ++c)
                    if (c < nc) acc[c] = fma_(e, xp[c], acc[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < KB_NC; ++c) part[(cj * KB_RB + ri) * KB_NC + c] = acc[c];
        __syncthreads();
        for (int e = threadIdx.x; e < KB_RB * KB_NC; e += 256) {
            const int r2 = e / KB_NC, c = e % KB_NC;
            const int i2 = orow0 + r2;
            if (i2 < P.rows && c < nc) {
                T s = part[r2 * KB_NC + c];
#pragma unroll
                for (int q = 1; q < PH; ++q) s += part[(q * KB_RB + r2) * KB_NC + c];
                T* yy = y + (P.y_off + i2) * nrhs + c0 + c;
                *yy = *yy + s;
            }
        }
        __syncthreads();
    }
}

template <class T>
cudaError_t launch_kblock_mv(cudaStream_t st, const KbProb* probs, const int64_t* blk0, int np, int64_t nblk,
                             const int32_t* pts, const T* x, T* y, int nrhs, const KernelK& K, const double* a)
{
    if (np <= 0 || nblk <= 0 || nrhs <= 0) return cudaSuccess;
    count_launches(1);
    kblock_mv_kernel<T><<<(unsigned)nblk, 256, 0, st>>>(probs, blk0, np, pts, x, y, nrhs, K, a);
    return cudaGetLastError();
}

int kblock_rows_per_block() { return KB_RB; }

#define RS_INST_KB(T)                                                                                                 \
    template cudaError_t launch_kblock_mv<T>(cudaStream_t, const KbProb*, const int64_t*, int, int64_t,             \
                                             const int32_t*, const T*, T*, int, const KernelK&, const double*);
RS_INST_KB(double)
RS_INST_KB(float)
RS_INST_KB(cplx<double>)
RS_INST_KB(cplx<float>)

}  // namespace rs
