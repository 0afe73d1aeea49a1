// k_residual.cu -- FP64 direct-sum residual r = f - A x of the Nystrom matrix (Laplace, or
// Helmholtz in its original form A = a + kappa^2 b K with complex128 arithmetic), used by the
// iterative refinement of the low-precision factorizations and by rs_residual, and the update
// r <- r - A dx of a residual by a small correction dx, whose product runs in FP32 (complex64).
//
// The off-diagonal entries depend only on the integer offset (d1, d2) between two grid points,
// so they are tabulated once for the (2n-1)^2 offsets; the sum over all N^2 pairs is then one
// FP64 FMA per pair with the table and the sources staged in shared memory, 16 x 16 targets
// against 16 x 16 sources per step.
#include "k_common.cuh"

namespace rs {

// Kt[(d1 + n - 1) + (2n - 1)(d2 + n - 1)] = c0 log((d1 h)^2 + (d2 h)^2), 0 at d1 = d2 = 0.
__global__ void laplace_table_kernel(int n, double h, double c0, double* __restrict__ Kt)
{
    const int W = 2 * n - 1;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)W * W) return;
    const int d1 = (int)(e % W) - (n - 1), d2 = (int)(e / W) - (n - 1);
    const double dx = (double)d1 * h, dy = (double)d2 * h;
    Kt[e] = (d1 == 0 && d2 == 0) ? 0.0 : c0 * log(dx * dx + dy * dy);
}

// Kt[...] = (i/4) H0^(1)(kappa |d| h) h^2 = (h^2/4)(-Y0 + i J0), 0 at d1 = d2 = 0.
__global__ void helmholtz_table_kernel(int n, double h, double kappa, cplx<double>* __restrict__ Kt)
{
    const int W = 2 * n - 1;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)W * W) return;
    const int d1 = (int)(e % W) - (n - 1), d2 = (int)(e / W) - (n - 1);
    if (d1 == 0 && d2 == 0) { Kt[e] = cplx<double>(0.0, 0.0); return; }
    const double z = kappa * h * sqrt((double)d1 * d1 + (double)d2 * d2);
    const double q = 0.25 * h * h;
    Kt[e] = cplx<double>(-q * y0(z), q * j0(z));
}

constexpr int DS = 16;          // tile side of targets and sources
constexpr int DS_RHS = 4;       // right-hand sides per pass

// yg = A xg in grid order: yg[c N + g] = dg[g] xg[c N + g] + rs[g] sum_{g' != g} K(g - g') xg[c N + g']
// (rs = NULL means 1).  Products and the sum over one 16 x 16 source tile run in S; the tile
// sums are added in A (A = S for the FP64 residual; A = FP64 for an FP32 product, so that the
// FP32 rounding stays that of 256-term sums however large the grid).  Each pass takes NC
// right-hand sides, NC fixed at compile time, so no FMA is issued for absent columns.
template <class S, class A, int NC>
__device__ __forceinline__ void direct_sum_pass(int n, const S* __restrict__ Kt, const S* __restrict__ dg,
        const double* __restrict__ rs, const S* __restrict__ xg, A* __restrict__ yg, int c0,
        S (*Kw)[2 * DS], S (*xs)[DS * DS])
{
    const int64_t N = (int64_t)n * n;
    const int W = 2 * n - 1;
    const int tx0 = blockIdx.x * DS, ty0 = blockIdx.y * DS;
    const int lx = threadIdx.x % DS, ly = threadIdx.x / DS;
    const int ti1 = tx0 + lx, ti2 = ty0 + ly;
    const bool tin = ti1 < n && ti2 < n;
    A acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = A(0.0);
    for (int sy0 = 0; sy0 < n; sy0 += DS) {
        for (int sx0 = 0; sx0 < n; sx0 += DS) {
            __syncthreads();
            for (int e = threadIdx.x; e < (2 * DS - 1) * (2 * DS - 1); e += blockDim.x) {
                const int e1 = e % (2 * DS - 1), e2 = e / (2 * DS - 1);
                const int d1 = tx0 - sx0 - (DS - 1) + e1, d2 = ty0 - sy0 - (DS - 1) + e2;
                Kw[e2][e1] = (d1 > -n && d1 < n && d2 > -n && d2 < n)
                                 ? Kt[(int64_t)(d1 + n - 1) + (int64_t)W * (d2 + n - 1)]
                                 : S(0.0);
            }
            for (int e = threadIdx.x; e < NC * DS * DS; e += blockDim.x) {
                const int c = e / (DS * DS), j = e - c * (DS * DS);
                const int s1 = sx0 + j % DS, s2 = sy0 + j / DS;
                xs[c][j] = (s1 < n && s2 < n) ? xg[(int64_t)(c0 + c) * N + s1 + (int64_t)n * s2] : S(0.0);
            }
            __syncthreads();
            if (tin) {
                S t[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) t[c] = S(0.0);
#pragma unroll 4
                for (int j2 = 0; j2 < DS; ++j2) {
#pragma unroll
                    for (int j1 = 0; j1 < DS; ++j1) {
                        const S k = Kw[ly - j2 + DS - 1][lx - j1 + DS - 1];
#pragma unroll
                        for (int c = 0; c < NC; ++c) t[c] = fma_(k, xs[c][j2 * DS + j1], t[c]);
                    }
                }
#pragma unroll
                for (int c = 0; c < NC; ++c) acc[c] += cast_<A>(t[c]);
            }
        }
    }
    if (tin) {
        const int64_t g = ti1 + (int64_t)n * ti2;
        const A sum_scale = rs ? A(rs[g]) : A(1.0);
#pragma unroll
        for (int c = 0; c < NC; ++c)
            yg[(int64_t)(c0 + c) * N + g] =
                fma_(cast_<A>(dg[g]), cast_<A>(xg[(int64_t)(c0 + c) * N + g]), sum_scale * acc[c]);
    }
}

template <class S, class A>
__global__ void __launch_bounds__(256) direct_sum_kernel(int n, const S* __restrict__ Kt, const S* __restrict__ dg,
        const double* __restrict__ rs, const S* __restrict__ xg, A* __restrict__ yg, int nrhs)
{
    __shared__ S Kw[2 * DS - 1][2 * DS];
    __shared__ S xs[DS_RHS][DS * DS];
    for (int c0 = 0; c0 < nrhs; c0 += DS_RHS) {
        switch (min(DS_RHS, nrhs - c0)) {
            case 1: direct_sum_pass<S, A, 1>(n, Kt, dg, rs, xg, yg, c0, Kw, xs); break;
            case 2: direct_sum_pass<S, A, 2>(n, Kt, dg, rs, xg, yg, c0, Kw, xs); break;
            case 3: direct_sum_pass<S, A, 3>(n, Kt, dg, rs, xg, yg, c0, Kw, xs); break;
            default: direct_sum_pass<S, A, 4>(n, Kt, dg, rs, xg, yg, c0, Kw, xs); break;
        }
    }
}

// The same sum with 32 x 32 target tiles, four targets per thread (column lx, rows ly + 8q),
// against 32 x 32 source tiles: the 63 x 63 table window and the sources are staged once per
// source tile for four times the products of the 16 x 16 form, so the staging and the two
// CTA barriers per tile stay small beside the FMAs even at one right-hand side.  The products
// of each 8-row band of a source tile (256 terms) are summed in S and the band sums added in
// A, the rounding structure of the 16 x 16 form.  Taken when the grid has at least three
// 32 x 32 target tiles per SM (1024 x 1024 and up on 152 SMs; fewer tiles would leave SMs
// with uneven shares) and for scalars of at most 8 bytes (its static shared memory holds
// 63 x 64 + 2 x 1024 scalars, within the 48 KB static limit).
constexpr int DT = 32;          // tile side of the large form
constexpr int DT_RHS = 2;       // right-hand sides per pass of the large form

// One pass of the large form over NC (compile-time, so no FMA is issued for absent columns)
// right-hand sides c0 .. c0 + NC.
template <class S, class A, int NC>
__device__ __forceinline__ void direct_sum32_pass(int n, const S* __restrict__ Kt, const S* __restrict__ dg,
        const double* __restrict__ rs, const S* __restrict__ xg, A* __restrict__ yg, int c0,
        S (*Kw)[2 * DT], S (*xs)[DT * DT])
{
    const int64_t N = (int64_t)n * n;
    const int W = 2 * n - 1;
    const int tx0 = blockIdx.x * DT, ty0 = blockIdx.y * DT;
    const int lx = threadIdx.x % DT, ly = threadIdx.x / DT;          // ly in 0..7
    const int ti1 = tx0 + lx;
    A acc[4][NC];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[q][c] = A(0.0);
    for (int sy0 = 0; sy0 < n; sy0 += DT) {
        for (int sx0 = 0; sx0 < n; sx0 += DT) {
            __syncthreads();
            for (int e = threadIdx.x; e < (2 * DT - 1) * (2 * DT - 1); e += blockDim.x) {
                const int e1 = e % (2 * DT - 1), e2 = e / (2 * DT - 1);
                const int d1 = tx0 - sx0 - (DT - 1) + e1, d2 = ty0 - sy0 - (DT - 1) + e2;
                Kw[e2][e1] = (d1 > -n && d1 < n && d2 > -n && d2 < n)
                                 ? Kt[(int64_t)(d1 + n - 1) + (int64_t)W * (d2 + n - 1)]
                                 : S(0.0);
            }
            for (int e = threadIdx.x; e < NC * DT * DT; e += blockDim.x) {
                const int c = e / (DT * DT), j = e - c * (DT * DT);
                const int s1 = sx0 + j % DT, s2 = sy0 + j / DT;
                xs[c][j] = (s1 < n && s2 < n) ? xg[(int64_t)(c0 + c) * N + s1 + (int64_t)n * s2] : S(0.0);
            }
            __syncthreads();
            for (int jb = 0; jb < DT; jb += 8) {                 // bands of 8 source rows
                S t[4][NC];
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int c = 0; c < NC; ++c) t[q][c] = S(0.0);
#pragma unroll 2
                for (int j2 = jb; j2 < jb + 8; ++j2) {
#pragma unroll 8
                    for (int j1 = 0; j1 < DT; ++j1) {
                        S xv[NC];
#pragma unroll
                        for (int c = 0; c < NC; ++c) xv[c] = xs[c][j2 * DT + j1];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const S k = Kw[ly + 8 * q - j2 + DT - 1][lx - j1 + DT - 1];
#pragma unroll
                            for (int c = 0; c < NC; ++c) t[q][c] = fma_(k, xv[c], t[q][c]);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int c = 0; c < NC; ++c) acc[q][c] += cast_<A>(t[q][c]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int ti2 = ty0 + ly + 8 * q;
        if (ti1 < n && ti2 < n) {
            const int64_t g = ti1 + (int64_t)n * ti2;
            const A sum_scale = rs ? A(rs[g]) : A(1.0);
#pragma unroll
            for (int c = 0; c < NC; ++c)
                yg[(int64_t)(c0 + c) * N + g] =
                    fma_(cast_<A>(dg[g]), cast_<A>(xg[(int64_t)(c0 + c) * N + g]), sum_scale * acc[q][c]);
        }
    }
}

template <class S, class A>
__global__ void __launch_bounds__(256) direct_sum32_kernel(int n, const S* __restrict__ Kt, const S* __restrict__ dg,
        const double* __restrict__ rs, const S* __restrict__ xg, A* __restrict__ yg, int nrhs)
{
    __shared__ S Kw[2 * DT - 1][2 * DT];
    __shared__ S xs[DT_RHS][DT * DT];
    for (int c0 = 0; c0 < nrhs; c0 += DT_RHS) {
        if (nrhs - c0 >= 2) direct_sum32_pass<S, A, 2>(n, Kt, dg, rs, xg, yg, c0, Kw, xs);
        else direct_sum32_pass<S, A, 1>(n, Kt, dg, rs, xg, yg, c0, Kw, xs);
    }
}

// One direct sum, by the form that suits the grid.
template <class S, class A>
static void launch_direct_sum(cudaStream_t st, int n, const S* Kt, const S* dg, const double* rs, const S* xg, A* yg,
                              int nrhs)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    const int64_t tiles32 = (int64_t)((n + DT - 1) / DT) * ((n + DT - 1) / DT);
    if constexpr (sizeof(S) <= 8) {
        if (tiles32 >= 3 * (int64_t)sms) {
            dim3 grid((unsigned)((n + DT - 1) / DT), (unsigned)((n + DT - 1) / DT));
            direct_sum32_kernel<S, A><<<grid, 256, 0, st>>>(n, Kt, dg, rs, xg, yg, nrhs);
            return;
        }
    }
    {
        dim3 grid((unsigned)((n + DS - 1) / DS), (unsigned)((n + DS - 1) / DS));
        direct_sum_kernel<S, A><<<grid, 256, 0, st>>>(n, Kt, dg, rs, xg, yg, nrhs);
    }
}

// xg[c N + g] = x[c N + ing[g]]
template <class S>
__global__ void to_grid_kernel(int64_t N, int nrhs, const int64_t* __restrict__ ing, const S* __restrict__ x,
                               S* __restrict__ xg)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * nrhs) return;
    const int64_t c = e / N, g = e - c * N;
    xg[e] = x[c * N + ing[g]];
}

// r[c N + ing[g]] = f[c N + ing[g]] - yg[c N + g]
template <class S>
__global__ void residual_finish_kernel(int64_t N, int nrhs, const int64_t* __restrict__ ing,
                                       const S* __restrict__ f, const S* __restrict__ yg, S* __restrict__ r)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * nrhs) return;
    const int64_t c = e / N, g = e - c * N;
    const int64_t i = c * N + ing[g];
    r[i] = f[i] - yg[e];
}

// out[2c] += sum_i |r[c N + i]|^2, out[2c + 1] += sum_i |f[c N + i]|^2
template <class S>
__global__ void __launch_bounds__(256) colnorm2_kernel(int64_t N, int nrhs, const S* __restrict__ r,
                                                       const S* __restrict__ f, double* __restrict__ out)
{
    __shared__ double sr[8], sf[8];
    const int c = blockIdx.y;
    double a = 0.0, b = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        a += abs2d(r[(int64_t)c * N + i]);
        b += abs2d(f[(int64_t)c * N + i]);
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if ((threadIdx.x & 31) == 0) { sr[threadIdx.x >> 5] = a; sf[threadIdx.x >> 5] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < 8; ++w) { ta += sr[w]; tb += sf[w]; }
        atomicAdd(out + 2 * c, ta);
        atomicAdd(out + 2 * c + 1, tb);
    }
}

static unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

cudaError_t launch_laplace_table(cudaStream_t st, int n, double h, double c0, double* Kt)
{
    const int64_t W = 2 * (int64_t)n - 1;
    count_launches(1);
    laplace_table_kernel<<<nblk(W * W), 256, 0, st>>>(n, h, c0, Kt);
    return cudaGetLastError();
}

cudaError_t launch_helmholtz_table(cudaStream_t st, int n, double h, double kappa, cplx<double>* Kt)
{
    const int64_t W = 2 * (int64_t)n - 1;
    count_launches(1);
    helmholtz_table_kernel<<<nblk(W * W), 256, 0, st>>>(n, h, kappa, Kt);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_residual(cudaStream_t st, int n, int nrhs, const S* Kt, const S* dg, const double* rs,
                            const int64_t* ing, const S* x, const S* f, S* xg, S* yg, S* r, double* norms)
{
    const int64_t N = (int64_t)n * n;
    count_launches(4);
    to_grid_kernel<S><<<nblk(N * nrhs), 256, 0, st>>>(N, nrhs, ing, x, xg);
    launch_direct_sum<S, S>(st, n, Kt, dg, rs, xg, yg, nrhs);
    residual_finish_kernel<S><<<nblk(N * nrhs), 256, 0, st>>>(N, nrhs, ing, f, yg, r);
    cudaError_t e = cudaMemsetAsync(norms, 0, sizeof(double) * 2 * nrhs, st);
    if (e != cudaSuccess) return e;
    dim3 g2((unsigned)std::min<int64_t>(nblk(N), 1024), (unsigned)nrhs);
    colnorm2_kernel<S><<<g2, 256, 0, st>>>(N, nrhs, r, f, norms);
    return cudaGetLastError();
}
// Low-precision copy of a table or diagonal: out[i] = (L) in[i].
template <class S, class L>
__global__ void narrow_kernel(int64_t n, const S* __restrict__ in, L* __restrict__ out)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] = cast_<L>(in[e]);
}

// xg[c N + g] = (L) dx[c N + ing[g]]
template <class S, class L>
__global__ void to_grid_narrow_kernel(int64_t N, int nrhs, const int64_t* __restrict__ ing, const S* __restrict__ x,
                                      L* __restrict__ xg)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * nrhs) return;
    const int64_t c = e / N, g = e - c * N;
    xg[e] = cast_<L>(x[c * N + ing[g]]);
}

// r[c N + ing[g]] -= yg[c N + g]
template <class S>
__global__ void residual_sub_kernel(int64_t N, int nrhs, const int64_t* __restrict__ ing, const S* __restrict__ yg,
                                    S* __restrict__ r)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * nrhs) return;
    const int64_t c = e / N, g = e - c * N;
    const int64_t i = c * N + ing[g];
    r[i] = r[i] - yg[e];
}

template <class S, class L>
cudaError_t launch_narrow(cudaStream_t st, int64_t n, const S* in, L* out)
{
    if (n <= 0) return cudaSuccess;
    count_launches(1);
    narrow_kernel<S, L><<<nblk(n), 256, 0, st>>>(n, in, out);
    return cudaGetLastError();
}

template <class S, class L>
cudaError_t launch_residual_update(cudaStream_t st, int n, int nrhs, const L* Kt, const L* dg, const double* rs,
                                   const int64_t* ing, const S* dx, S* r, L* xg, S* yg, double* norms)
{
    const int64_t N = (int64_t)n * n;
    count_launches(4);
    to_grid_narrow_kernel<S, L><<<nblk(N * nrhs), 256, 0, st>>>(N, nrhs, ing, dx, xg);
    launch_direct_sum<L, S>(st, n, Kt, dg, rs, xg, yg, nrhs);
    residual_sub_kernel<S><<<nblk(N * nrhs), 256, 0, st>>>(N, nrhs, ing, yg, r);
    cudaError_t e = cudaMemsetAsync(norms, 0, sizeof(double) * 2 * nrhs, st);
    if (e != cudaSuccess) return e;
    dim3 g2((unsigned)std::min<int64_t>(nblk(N), 1024), (unsigned)nrhs);
    colnorm2_kernel<S><<<g2, 256, 0, st>>>(N, nrhs, r, r, norms);
    return cudaGetLastError();
}
template cudaError_t launch_narrow<double, float>(cudaStream_t, int64_t, const double*, float*);
template cudaError_t launch_narrow<cplx<double>, cplx<float>>(cudaStream_t, int64_t, const cplx<double>*,
                                                              cplx<float>*);
template cudaError_t launch_residual_update<double, float>(cudaStream_t, int, int, const float*, const float*,
                                                           const double*, const int64_t*, const double*, double*,
                                                           float*, double*, double*);
template cudaError_t launch_residual_update<cplx<double>, cplx<float>>(cudaStream_t, int, int, const cplx<float>*,
                                                                       const cplx<float>*, const double*,
                                                                       const int64_t*, const cplx<double>*,
                                                                       cplx<double>*, cplx<float>*, cplx<double>*,
                                                                       double*);
template cudaError_t launch_residual<double>(cudaStream_t, int, int, const double*, const double*, const double*,
                                             const int64_t*, const double*, const double*, double*, double*, double*,
                                             double*);
template cudaError_t launch_residual<cplx<double>>(cudaStream_t, int, int, const cplx<double>*, const cplx<double>*,
                                                   const double*, const int64_t*, const cplx<double>*,
                                                   const cplx<double>*, cplx<double>*, cplx<double>*, cplx<double>*,
                                                   double*);

}  // namespace rs
