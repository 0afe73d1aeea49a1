// k_matvec.cuh -- the block body of the batched matvec(s), shared by the per-level solve
// launch (k_linalg.cu) and the serving job kernel (k_serve.cu).
#pragma once
#include "k_common.cuh"

namespace rs {

// 64 output rows of one problem for all nrhs columns (chunks of 8), shared by the per-level
// launch below and the serving job kernel (k_serve.cu), so that a request's arithmetic does
// not depend on how it was batched.
template <class T>
__device__ __forceinline__ void matvec_block(const MatvecProb& P, int orow0, const T* __restrict__ A,
                                             const T* __restrict__ x, T* __restrict__ y, int nrhs,
                                             T (*part)[64][8])
{
    constexpr int RB = 64, CH = 8;
    const int out_n = P.trans ? P.cols : P.rows;
    const int in_n = P.trans ? P.rows : P.cols;
    for (int c0 = 0; c0 < nrhs; c0 += CH) {
        const int nc = min(CH, nrhs - c0);
        T acc[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) acc[c] = 0;
        if (!P.trans) {
            const int ri = threadIdx.x & 63, cj = threadIdx.x >> 6;   // 64 rows x 4 column phases
            const int i = orow0 + ri;
            if (i < out_n) {
                for (int j = cj; j < in_n; j += 4) {
                    const T a = A[(int64_t)j * P.ld + i];
#pragma unroll
                    for (int c = 0; c < CH; ++c)
                        if (c < nc) acc[c] = fma_(a, x[(int64_t)j * nrhs + c0 + c], acc[c]);
                }
            }
#pragma unroll
            for (int c = 0; c < CH; ++c) part[cj][ri][c] = acc[c];
            __syncthreads();
            if (threadIdx.x < RB) {
                const int i2 = orow0 + threadIdx.x;
                if (i2 < out_n)
                    for (int c = 0; c < nc; ++c) {
                        const T s = part[0][threadIdx.x][c] + part[1][threadIdx.x][c] + part[2][threadIdx.x][c] +
                                    part[3][threadIdx.x][c];
                        T* yy = y + (int64_t)i2 * nrhs + c0 + c;
                        *yy = (P.beta == 0.0) ? (T)P.alpha * s : (T)P.alpha * s + (T)P.beta * (*yy);
                    }
            }
            __syncthreads();
        } else {
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            for (int q = warp; q < RB; q += 8) {
                const int j = orow0 + q;
                if (j >= out_n) break;
                T a2[CH];
#pragma unroll
                for (int c = 0; c < CH; ++c) a2[c] = 0;
                const T* colj = A + (int64_t)j * P.ld;
                for (int i = lane; i < in_n; i += 32) {
                    const T a = colj[i];
#pragma unroll
                    for (int c = 0; c < CH; ++c)
                        if (c < nc) a2[c] = fma_(a, x[(int64_t)i * nrhs + c0 + c], a2[c]);
                }
#pragma unroll
                for (int c = 0; c < CH; ++c) a2[c] = warp_sum(a2[c]);
                if (lane == 0)
                    for (int c = 0; c < nc; ++c) {
                        T* yy = y + (int64_t)j * nrhs + c0 + c;
                        *yy = (P.beta == 0.0) ? (T)P.alpha * a2[c] : (T)P.alpha * a2[c] + (T)P.beta * (*yy);
                    }
            }
        }
    }
}

// Problem p of a descriptor set whose first block is blk0[p].
__device__ __forceinline__ int find_block(const int64_t* __restrict__ blk0, int np, int64_t t)
{
    int lo = 0, hi = np - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (blk0[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace rs
