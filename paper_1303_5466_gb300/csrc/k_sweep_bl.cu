// k_sweep_bl.cu -- the symmetric sweep of k_sweep.cu (S <- -S^{-1} for SPD S, lower triangle) in
// panels of 64, with the rank-64 updates on the digit-slice GEMM of k_gemm_oz.cu.
//
// The sweep of a symmetric S on an index block K (D = S_KK) is
//     S_KK <- -D^{-1},  S_OK <- S_OK D^{-1},  S_KO <- D^{-1} S_KO,  S_OO <- S_OO - S_OK D^{-1} S_KO,
// so with Q = S[:, K] (the old panel, both triangles) and X = Q D^{-1}, one step is
//   1. (copy kernel) Q, row-major, in 64 x 64 tiles; (one CTA per matrix) D^{-1} by the sweep of
//      the lower triangle of the 64 x 64 block D in pivot blocks of 8, in shared memory, FP64,
//      with the pivot test of k_sweep.cu (a pivot not above 1e3 unit roundoff times the largest
//      earlier one sets DEV_NOT_SPD);
//   2. X = Q D^{-1} and S <- S - X Q^T on the tiles touching the lower triangle (both on the
//      digit-slice GEMM: the m^3 flops of the inverse as 64-deep products);
//   3. (write kernel) the rows and columns of K, which step 2 left meaningless: S[i, K] = X[i, :]
//      below K, S[K, j] = X[j, :]^T left of K, S_KK = -D^{-1}.
// After the last panel S holds -S^{-1} in its lower triangle; launch_sweep_finish negates and
// mirrors it.  FP64 only.
#include <float.h>

#include <algorithm>
#include <vector>

#include "k_common.cuh"

namespace rs {

namespace {

constexpr int BS = 64;

// Q (row-major m x 64: Q[i 64 + t] = S(i, k0 + t), both triangles from the lower one) in tiles of
// 64 rows, each read where S is contiguous (down a column of storage below the panel, along a
// column of storage -- the panel's rows -- left of it) and transposed through shared memory.
__global__ void __launch_bounds__(256) sweep_bl_copy_kernel(int k0, const int32_t* __restrict__ msz,
        const int64_t* __restrict__ off, const double* __restrict__ Aall, const int64_t* __restrict__ qoff,
        double* __restrict__ Qall)
{
    __shared__ double tile[BS][BS + 1];
    const int b = blockIdx.y;
    const int m = msz[b];
    const int i0 = blockIdx.x * BS;
    if (k0 >= m || i0 >= m) return;
    const int w = min(BS, m - k0);
    const double* A = Aall + off[b];
    double* Q = Qall + qoff[b];
    const int rows = min(BS, m - i0);
    if (i0 + BS <= k0) {
        // rows left of the panel: S(i, k0 + t) = A[i m + k0 + t], contiguous in t
        for (int e = threadIdx.x; e < BS * BS; e += 256) {
            const int ii = e / BS, t = e - ii * BS;
            tile[ii][t] = (ii < rows && t < w) ? A[(int64_t)(i0 + ii) * m + k0 + t] : 0.0;
        }
    } else {
        // rows at or below the panel: S(i, c) = A[c m + i] for i >= c, contiguous in i
        for (int e = threadIdx.x; e < BS * BS; e += 256) {
            const int t = e / BS, ii = e - t * BS;
            const int i = i0 + ii, c = k0 + t;
            double v = 0.0;
            if (ii < rows && t < w) v = i >= c ? A[(int64_t)c * m + i] : A[(int64_t)i * m + c];
            tile[ii][t] = v;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rows * BS; e += 256) {
        const int ii = e / BS, t = e - ii * BS;
        Q[(int64_t)(i0 + ii) * BS + t] = tile[ii][t];
    }
}

// D^{-1} of the panel's diagonal block D = Q[k0 .. k0 + w) by the sweep of its lower triangle in
// pivot blocks of 8, in shared memory, FP64, with the pivot test of k_sweep.cu (the element sweep
// of each 8 x 8 pivot block by one warp); one CTA per matrix.  Block J: C = D(:, J) (old), the
// warp sweeps P = D(J, J) into P^{-1}, U = C P^{-1}, then every lower entry (r, s) off J becomes
// D(r, s) - U(r, :) C(s, :)^T, the entries of J's rows and columns U, and D(J, J) = -P^{-1}:
// three block barriers per 8 pivots instead of two per pivot.
__global__ void __launch_bounds__(256) sweep_bl_dinv_kernel(int k0, const int32_t* __restrict__ msz,
        const int64_t* __restrict__ qoff, const double* __restrict__ Qall, double* __restrict__ Dall,
        double* __restrict__ maxp, int* __restrict__ status)
{
    constexpr int PB = 8;
    __shared__ double sM[BS][BS + 1];
    __shared__ double s_col[BS][PB + 1], s_U[BS][PB + 1], s_P[PB][PB + 1];
    __shared__ int s_fail;
    __shared__ double s_mp;
    const int b = blockIdx.x;
    const int m = msz[b];
    if (k0 >= m) return;
    const int w = min(BS, m - k0);
    const double* Q = Qall + qoff[b] + (int64_t)k0 * BS;
    for (int e = threadIdx.x; e < BS * BS; e += 256) {
        const int r = e / BS, c = e - r * BS;
        sM[r][c] = (r < w && c < w) ? Q[e] : (r == c ? 1.0 : 0.0);
    }
    if (threadIdx.x == 0) {
        s_fail = 0;
        s_mp = maxp[b];
    }
    // the lower entries of this thread: e = tid + 256 u over the 2080 of the 64 x 64 triangle
    constexpr int NL = BS * (BS + 1) / 2, PER = (NL + 255) / 256;
    int er[PER], ec[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + 256 * u;
        int r = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
        while (r * (r + 1) / 2 > e) --r;
        while ((r + 1) * (r + 2) / 2 <= e) ++r;
        er[u] = e < NL ? r : -1;
        ec[u] = e - r * (r + 1) / 2;
    }
    __syncthreads();
    const int nblk = (w + PB - 1) / PB;
    for (int J = 0; J < nblk; ++J) {
        const int j0 = J * PB;
        // 1. C = D(:, J), from the lower triangle
        for (int e = threadIdx.x; e < BS * PB; e += 256) {
            const int r = e / PB, t = e - r * PB, c = j0 + t;
            s_col[r][t] = r >= c ? sM[r][c] : sM[c][r];
        }
        __syncthreads();
        // 2. warp 0: the element sweep of P = C(J, :) in s_P into -P^{-1}, the pivot test
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            double mp = s_mp;
            int fail = 0;
            int rr[2], cc[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                rr[u] = (lane + 32 * u) / PB;
                cc[u] = (lane + 32 * u) % PB;
                s_P[rr[u]][cc[u]] = s_col[j0 + rr[u]][cc[u]];
            }
            __syncwarp();
            for (int t = 0; t < PB; ++t) {
                const double p = s_P[t][t];
                if (!(p > 1e3 * 0.5 * DBL_EPSILON * mp) || !isfinite(p)) fail = 1;
                mp = fmax(mp, p);
                const double pinv = 1.0 / p;
                double nv[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int r = rr[u], c = cc[u];
                    if (r == t && c == t) nv[u] = -pinv;
                    else if (r == t) nv[u] = s_P[t][c] * pinv;
                    else if (c == t) nv[u] = s_P[r][t] * pinv;
                    else nv[u] = fma(-s_P[r][t] * pinv, s_P[t][c], s_P[r][c]);
                }
                __syncwarp();
#pragma unroll
                for (int u = 0; u < 2; ++u) s_P[rr[u]][cc[u]] = nv[u];
                __syncwarp();
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) s_P[rr[u]][cc[u]] = -s_P[rr[u]][cc[u]];     // P^{-1}
            if (lane == 0) {
                s_mp = mp;
                if (fail) s_fail = 1;
            }
        }
        __syncthreads();
        // 3. U = C P^{-1}
        for (int e = threadIdx.x; e < BS * PB; e += 256) {
            const int r = e / PB, t = e - r * PB;
            double a = 0.0;
#pragma unroll
            for (int q = 0; q < PB; ++q) a = fma(s_col[r][q], s_P[q][t], a);
            s_U[r][t] = a;
        }
        __syncthreads();
        // 4. the lower entries
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int r = er[u], c = ec[u];
            if (r < 0) continue;
            const bool rin = r >= j0 && r < j0 + PB, cin = c >= j0 && c < j0 + PB;
            double x;
            if (rin && cin) x = -s_P[r - j0][c - j0];
            else if (cin) x = s_U[r][c - j0];
            else if (rin) x = s_U[c][r - j0];
            else {
                x = sM[r][c];
#pragma unroll
                for (int t = 0; t < PB; ++t) x = fma(-s_U[r][t], s_col[c][t], x);
            }
            sM[r][c] = x;
        }
        __syncthreads();
    }
    double* Dinv = Dall + (int64_t)b * BS * BS;          // D^{-1}, column-major 64 x 64, both triangles
    for (int e = threadIdx.x; e < BS * BS; e += 256) {
        const int c = e / BS, r = e - c * BS;
        Dinv[e] = (r < w && c < w) ? -(r >= c ? sM[r][c] : sM[c][r]) : 0.0;
    }
    if (threadIdx.x == 0) {
        maxp[b] = s_mp;
        if (s_fail) atomicOr(status, DEV_NOT_SPD);
    }
}

__global__ void __launch_bounds__(256) sweep_bl_write_kernel(int k0, const int32_t* __restrict__ msz,
        const int64_t* __restrict__ off, double* __restrict__ Aall, const int64_t* __restrict__ qoff,
        const double* __restrict__ Xall, const double* __restrict__ Dall)
{
    const int b = blockIdx.y;
    const int m = msz[b];
    if (k0 >= m) return;
    const int w = min(BS, m - k0);
    double* A = Aall + off[b];
    const double* X = Xall + qoff[b];
    const double* Dinv = Dall + (int64_t)b * BS * BS;
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < (int64_t)m * w; e += (int64_t)gridDim.x * 256) {
        const int t = (int)(e / m), i = (int)(e - (int64_t)t * m);
        const int c = k0 + t;
        if (i >= k0 + w) A[(int64_t)c * m + i] = X[(int64_t)t * m + i];          // S[i, K] below K
        else if (i < k0) A[(int64_t)i * m + c] = X[(int64_t)t * m + i];          // S[K, i] left of K
        else if (i - k0 >= t) A[(int64_t)c * m + i] = -Dinv[t * BS + (i - k0)];  // S_KK = -D^{-1}
    }
}

}  // namespace

size_t sweep_bl_plan(int nb, const std::vector<int64_t>& sizes, int max_m, std::vector<int64_t>& qoff,
                     std::vector<std::vector<GemmProb>>& gx, std::vector<std::vector<GemmProb>>& gu,
                     const std::vector<int64_t>& off)
{
    qoff.assign(nb + 1, 0);
    for (int b = 0; b < nb; ++b) qoff[b + 1] = qoff[b] + (int64_t)BS * sizes[b];
    const int steps = (max_m + BS - 1) / BS;
    gx.assign(steps, {});
    gu.assign(steps, {});
    for (int q = 0; q < steps; ++q) {
        const int k0 = q * BS;
        for (int b = 0; b < nb; ++b) {
            const int m = (int)sizes[b];
            if (k0 >= m) continue;
            const int w = std::min(BS, m - k0);
            GemmProb g{};                                  // X = Q D^{-1}
            g.M = m; g.N = w; g.K = w; g.ta = 1; g.tb = 0;
            g.lda = BS; g.ldb = BS; g.ldc = m; g.ldc0 = m;
            g.a_off = qoff[b]; g.b_off = (int64_t)b * BS * BS; g.c_off = qoff[b]; g.c0_off = 0;
            g.alpha = 1.0; g.beta = 0.0;
            gx[q].push_back(g);
            GemmProb h{};                                  // S <- S - X Q^T, lower tiles
            h.M = m; h.N = m; h.K = w; h.ta = 0; h.tb = 0;
            h.lda = m; h.ldb = BS; h.ldc = m; h.ldc0 = m;
            h.a_off = qoff[b]; h.b_off = qoff[b]; h.c_off = off[b]; h.c0_off = off[b];
            h.alpha = -1.0; h.beta = 1.0; h.lower = 1;
            gu[q].push_back(h);
        }
    }
    return (size_t)qoff[nb];
}

cudaError_t launch_sweep_bl_panel(cudaStream_t st, int nb, int k0, int max_m, const int32_t* m, const int64_t* off,
                                  const double* A, const int64_t* qoff, double* Q, double* D, double* maxp, int* status)
{
    if (nb <= 0 || max_m <= k0) return cudaSuccess;
    count_launches(2);
    sweep_bl_copy_kernel<<<dim3((unsigned)((max_m + BS - 1) / BS), (unsigned)nb), 256, 0, st>>>(k0, m, off, A, qoff, Q);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sweep_bl_dinv_kernel<<<nb, 256, 0, st>>>(k0, m, qoff, Q, D, maxp, status);
    return cudaGetLastError();
}

cudaError_t launch_sweep_bl_write(cudaStream_t st, int nb, int k0, int max_m, const int32_t* m, const int64_t* off,
                                  double* A, const int64_t* qoff, const double* X, const double* D)
{
    if (nb <= 0 || max_m <= k0) return cudaSuccess;
    const int64_t work = (int64_t)(max_m - k0 < BS ? max_m - k0 : BS) * max_m;
    const unsigned gx = (unsigned)std::min<int64_t>((work + 255) / 256, 4096);
    count_launches(1);
    sweep_bl_write_kernel<<<dim3(gx, (unsigned)nb), 256, 0, st>>>(k0, m, off, A, qoff, X, D);
    return cudaGetLastError();
}

}  // namespace rs
