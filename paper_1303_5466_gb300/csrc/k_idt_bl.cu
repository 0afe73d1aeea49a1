// k_idt_bl.cu -- T = R11^{-1} R12 (Eq. 2.1) by blocks of 64 rows of R11, with the updates of the
// rows above each block on the digit-slice GEMM of k_gemm_oz.cu (FP64 operators).
//
//   1. (gather) R = [R11 | R12] of every box into a k x m column-major block (R11 from the pivot
//      columns of Y, its diagonal from diag; R12 from the residual columns);
//   2. for the blocks J of 64 rows from the bottom of R11: (solve) X_J = R_JJ^{-1} B_J in place,
//      one thread per right-hand side with the block's rows in registers, the reciprocals of
//      R_JJ's diagonal taken once per block; (digit-slice GEMM) B_I <- B_I - R_IJ X_J for the rows
//      I above J;
//   3. (scatter) T in the layout of id_T_kernel: rows by sorted skeleton position, columns by
//      residual rank.
#include <algorithm>
#include <vector>

#include "k_common.cuh"

namespace rs {

namespace {

constexpr int IB = 64;

__global__ void __launch_bounds__(256) idt_gather_kernel(const int64_t* __restrict__ act_off,
        const int32_t* __restrict__ kk, const int32_t* __restrict__ nnear, int P, const int64_t* __restrict__ y_off,
        const double* __restrict__ Yall, const int32_t* __restrict__ piv, const double* __restrict__ diag,
        const int32_t* __restrict__ rscol, const int64_t* __restrict__ rg_off, double* __restrict__ Rg)
{
    const int b = blockIdx.y;
    const int64_t a0 = act_off[b];
    const int m = (int)(act_off[b + 1] - a0), k = kk[b];
    if (k <= 0) return;
    const int r = nnear[b] + P;
    const double* Y = Yall + y_off[b];
    double* R = Rg + rg_off[b];
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < (int64_t)k * m; e += (int64_t)gridDim.x * 256) {
        const int c = (int)(e / k), i = (int)(e - (int64_t)c * k);
        double v;
        if (c < k) v = i < c ? Y[(int64_t)piv[a0 + c] * r + i] : (i == c ? diag[a0 + c] : 0.0);
        else v = Y[(int64_t)rscol[a0 + c - k] * r + i];
        R[e] = v;
    }
}

// Step q: the block J = [j0, j1), j1 = k - 64 q, of every box with j1 > 0; one right-hand side per
// thread, 64 per CTA, its 64 rows in registers (the block padded with the identity beyond w, so
// every loop has compile-time bounds), R_JJ and the reciprocals of its diagonal in shared memory
// (read by all threads at once): every FMA of the substitution does useful work.
__global__ void __launch_bounds__(IB) idt_solve_kernel(int q, const int64_t* __restrict__ act_off,
        const int32_t* __restrict__ kk, const int64_t* __restrict__ rg_off, double* __restrict__ Rg)
{
    __shared__ double sR[IB][IB + 1];
    __shared__ double sInv[IB];
    const int b = blockIdx.y;
    const int m = (int)(act_off[b + 1] - act_off[b]), k = kk[b];
    const int j1 = k - IB * q;
    if (j1 <= 0) return;
    const int j0 = max(0, j1 - IB), w = j1 - j0, nres = m - k;
    const int cb = blockIdx.x * IB;
    if (cb >= nres) return;
    const double* R = Rg + rg_off[b];
    for (int e = threadIdx.x; e < IB * IB; e += IB) {
        const int l = e / IB, i = e - l * IB;              // column l, row i of R_JJ
        double v = 0.0;
        if (i < w && l < w) v = i <= l ? R[(int64_t)(j0 + l) * k + j0 + i] : 0.0;
        else if (i == l) v = 1.0;
        sR[i][l] = v;
    }
    __syncthreads();
    sInv[threadIdx.x] = 1.0 / sR[threadIdx.x][threadIdx.x];
    __syncthreads();
    const int c = cb + threadIdx.x;
    if (c >= nres) return;
    double* col = Rg + rg_off[b] + (int64_t)k * k + (int64_t)c * k + j0;   // column c of R12, rows J
    double x[IB];
#pragma unroll
    for (int i = 0; i < IB; ++i) x[i] = i < w ? col[i] : 0.0;
#pragma unroll
    for (int i = IB - 1; i >= 0; --i) {
        x[i] *= sInv[i];
#pragma unroll
        for (int l = 0; l < i; ++l) x[l] = fma(-sR[l][i], x[i], x[l]);
    }
#pragma unroll
    for (int i = 0; i < IB; ++i)
        if (i < w) col[i] = x[i];
}

__global__ void __launch_bounds__(256) idt_scatter_kernel(const int64_t* __restrict__ act_off,
        const int32_t* __restrict__ kk, const int32_t* __restrict__ skpos, const int64_t* __restrict__ rg_off,
        const double* __restrict__ Rg, const int64_t* __restrict__ t_off, double* __restrict__ Tout)
{
    const int b = blockIdx.y;
    const int64_t a0 = act_off[b];
    const int m = (int)(act_off[b + 1] - a0), k = kk[b], nres = m - k;
    if (k <= 0 || nres <= 0) return;
    const double* B = Rg + rg_off[b] + (int64_t)k * k;
    double* Tb = Tout + t_off[b];
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < (int64_t)k * nres; e += (int64_t)gridDim.x * 256) {
        const int c = (int)(e / k), a = (int)(e - (int64_t)c * k);
        Tb[(int64_t)c * k + skpos[a0 + a]] = B[e];
    }
}

}  // namespace

size_t idt_bl_plan(int nb, const std::vector<int64_t>& m, const std::vector<int64_t>& k, int max_k,
                   std::vector<int64_t>& rg_off, std::vector<std::vector<GemmProb>>& gs)
{
    rg_off.assign(nb + 1, 0);
    for (int b = 0; b < nb; ++b) rg_off[b + 1] = rg_off[b] + k[b] * m[b];
    const int steps = (max_k + IB - 1) / IB;
    gs.assign(steps, {});
    for (int q = 0; q < steps; ++q)
        for (int b = 0; b < nb; ++b) {
            const int kb = (int)k[b], nres = (int)(m[b] - k[b]);
            const int j1 = kb - IB * q, j0 = std::max(0, j1 - IB);
            if (j1 <= 0 || j0 == 0 || nres <= 0) continue;
            GemmProb g{};                                  // B_I <- B_I - R_IJ X_J, I = rows above J
            g.M = j0; g.N = nres; g.K = j1 - j0; g.ta = 0; g.tb = 0;
            g.lda = kb; g.ldb = kb; g.ldc = kb; g.ldc0 = kb;
            g.a_off = rg_off[b] + (int64_t)j0 * kb;
            g.b_off = rg_off[b] + (int64_t)kb * kb + j0;
            g.c_off = rg_off[b] + (int64_t)kb * kb;
            g.c0_off = g.c_off;
            g.alpha = -1.0; g.beta = 1.0;
            gs[q].push_back(g);
        }
    return (size_t)rg_off[nb];
}

cudaError_t launch_idt_gather(cudaStream_t st, int nb, int64_t max_km, const int64_t* act_off, const int32_t* kk,
                              const int32_t* nnear, int P, const int64_t* y_off, const double* Y, const int32_t* piv,
                              const double* diag, const int32_t* rscol, const int64_t* rg_off, double* Rg)
{
    if (nb <= 0 || max_km <= 0) return cudaSuccess;
    count_launches(1);
    const unsigned gx = (unsigned)std::min<int64_t>((max_km + 255) / 256, 2048);
    idt_gather_kernel<<<dim3(gx, (unsigned)nb), 256, 0, st>>>(act_off, kk, nnear, P, y_off, Y, piv, diag, rscol,
                                                              rg_off, Rg);
    return cudaGetLastError();
}

cudaError_t launch_idt_solve(cudaStream_t st, int nb, int q, int max_res, const int64_t* act_off, const int32_t* kk,
                             const int64_t* rg_off, double* Rg)
{
    if (nb <= 0 || max_res <= 0) return cudaSuccess;
    count_launches(1);
    idt_solve_kernel<<<dim3((unsigned)((max_res + IB - 1) / IB), (unsigned)nb), IB, 0, st>>>(q, act_off, kk, rg_off,
                                                                                              Rg);
    return cudaGetLastError();
}

cudaError_t launch_idt_scatter(cudaStream_t st, int nb, int64_t max_kres, const int64_t* act_off, const int32_t* kk,
                               const int32_t* skpos, const int64_t* rg_off, const double* Rg, const int64_t* t_off,
                               double* Tout)
{
    if (nb <= 0 || max_kres <= 0) return cudaSuccess;
    count_launches(1);
    const unsigned gx = (unsigned)std::min<int64_t>((max_kres + 255) / 256, 2048);
    idt_scatter_kernel<<<dim3(gx, (unsigned)nb), 256, 0, st>>>(act_off, kk, skpos, rg_off, Rg, t_off, Tout);
    return cudaGetLastError();
}

}  // namespace rs
