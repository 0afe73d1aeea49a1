// k_matvec.cuh -- the block body of the batched matvec(s), shared by the per-level solve
// launch (k_linalg.cu) and the serving job kernel (k_serve.cu).
#pragma once
#include "k_common.cuh"

namespace rs {

// One chunk of NC right-hand sides (columns c0 .. c0 + NC) of RB output entries of one problem.
//   y = A x: RB rows x (256 / RB) column phases; the phases' partial sums meet in `part` and
//            are added in a fixed order, so the result does not depend on the launch;
//   y = A^T x: warp w takes outputs w, w + 8, ... of the RB, each a warp-wide dot product.
// NC is a compile-time count, so no FMA is spent on absent columns.
template <class T, int RB, int NC>
__device__ __forceinline__ void mv_chunk(const MatvecProb& P, int orow0, const T* __restrict__ A,
                                         const T* __restrict__ x, T* __restrict__ y, int nrhs, int c0,
                                         T* __restrict__ part)
{
    constexpr int PH = 256 / RB;
    const int out_n = P.trans ? P.cols : P.rows;
    const int in_n = P.trans ? P.rows : P.cols;
    T acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0;
    if (!P.trans) {
        const int ri = threadIdx.x % RB, cj = threadIdx.x / RB;
        const int i = orow0 + ri;
        if (i < out_n) {
            const T* __restrict__ ap = A + (int64_t)cj * P.ld + i;
            const T* __restrict__ xp = x + (int64_t)cj * nrhs + c0;
            const int64_t astep = (int64_t)PH * P.ld, xstep = (int64_t)PH * nrhs;
            for (int j = cj; j < in_n; j += PH, ap += astep, xp += xstep) {
                const T a = *ap;
#pragma unroll
                for (int c = 0; c < NC; ++c) acc[c] = fma_(a, xp[c], acc[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) part[(cj * RB + ri) * NC + c] = acc[c];
        __syncthreads();
        for (int e = threadIdx.x; e < RB * NC; e += 256) {
            const int r2 = e / NC, c = e - (e / NC) * NC;
            const int i2 = orow0 + r2;
            if (i2 < out_n) {
                T s = part[r2 * NC + c];
#pragma unroll 4
                for (int q = 1; q < PH; ++q) s += part[(q * RB + r2) * NC + c];
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
            T a2[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) a2[c] = 0;
            const T* colj = A + (int64_t)j * P.ld;
            for (int i = lane; i < in_n; i += 32) {
                const T a = colj[i];
#pragma unroll
                for (int c = 0; c < NC; ++c) a2[c] = fma_(a, x[(int64_t)i * nrhs + c0 + c], a2[c]);
            }
#pragma unroll
            for (int c = 0; c < NC; ++c) a2[c] = warp_sum(a2[c]);
            if (lane == 0)
                for (int c = 0; c < NC; ++c) {
                    T* yy = y + (int64_t)j * nrhs + c0 + c;
                    *yy = (P.beta == 0.0) ? (T)P.alpha * a2[c] : (T)P.alpha * a2[c] + (T)P.beta * (*yy);
                }
        }
    }
}

// RB output entries of one problem (orow0 .. orow0 + RB) for all nrhs columns, in chunks of
// 8; `part` holds 256 x 8 scalars.  Shared by the per-level launch (k_linalg.cu) and the
// serving job kernel (k_serve.cu), so that a request's arithmetic does not depend on how it
// was batched.
template <class T, int RB>
__device__ __forceinline__ void matvec_block(const MatvecProb& P, int orow0, const T* __restrict__ A,
                                             const T* __restrict__ x, T* __restrict__ y, int nrhs, T* part)
{
    for (int c0 = 0; c0 < nrhs; c0 += 8) {
        switch (min(8, nrhs - c0)) {
            case 1: mv_chunk<T, RB, 1>(P, orow0, A, x, y, nrhs, c0, part); break;
            case 2: mv_chunk<T, RB, 2>(P, orow0, A, x, y, nrhs, c0, part); break;
            case 3: mv_chunk<T, RB, 3>(P, orow0, A, x, y, nrhs, c0, part); break;
            case 4: mv_chunk<T, RB, 4>(P, orow0, A, x, y, nrhs, c0, part); break;
            case 5: mv_chunk<T, RB, 5>(P, orow0, A, x, y, nrhs, c0, part); break;
            case 6: mv_chunk<T, RB, 6>(P, orow0, A, x, y, nrhs, c0, part); break;
            case 7: mv_chunk<T, RB, 7>(P, orow0, A, x, y, nrhs, c0, part); break;
            default: mv_chunk<T, RB, 8>(P, orow0, A, x, y, nrhs, c0, part); break;
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
