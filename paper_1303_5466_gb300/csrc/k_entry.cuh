// k_entry.cuh -- matrix entries of the discretized operator, evaluated on the device in the
// storage type S of the kernel that reads them (shared by the factor's assembly kernels and the
// forward apply).
#pragma once
#include "k_common.cuh"

namespace rs {

__device__ __forceinline__ void grid_xy(const KernelK& K, int g, double& x, double& y)
{
    const int i1 = g % K.n, i2 = g / K.n;
    x = ((double)i1 + 0.5) * K.h;
    y = ((double)i2 + 0.5) * K.h;
}

// Matrix entries in the storage type S (the arithmetic of the factor's precision).
//   Laplace (real S): off-diagonal -(1/2pi) h^2 log|x - y| = c0 log(|x - y|^2);
//   Helmholtz (complex S): s_g (i/4) H0^(1)(kappa r) h^2 s_g' with H0^(1) = J0 + i Y0.
template <class S>
__device__ __forceinline__ S hank_row(const KernelK& K, double r)
{
    // (i/4) H0^(1)(kappa r) h^2 = (h^2/4) (-Y0 + i J0)
    using R = typename sc_traits<S>::real;
    if constexpr (sizeof(R) == sizeof(float)) {
        const float z = (float)(K.kappa * r);
        const float q = (float)(0.25 * K.h * K.h);
        return S(-q * y0f(z), q * j0f(z));
    } else {
        const double z = K.kappa * r;
        const double q = 0.25 * K.h * K.h;
        return S(-q * y0(z), q * j0(z));
    }
}

// Helmholtz scaling s_g of the symmetric form (per grid point, or the constant s0)
__device__ __forceinline__ double kscale(const KernelK& K, int g) { return K.s ? K.s[g] : K.s0; }

template <class S>
__device__ __forceinline__ S kentry(const KernelK& K, int g, int gp)
{
    if (K.tab) {
        const int d1 = g % K.n - gp % K.n, d2 = g / K.n - gp / K.n;
        const S t = ((const S*)K.tab)[(d1 + K.n - 1) + (int64_t)(2 * K.n - 1) * (d2 + K.n - 1)];
        if constexpr (is_cplx<S>::value) return rscale<S>(kscale(K, g) * kscale(K, gp), t);
        else return t;
    }
    if constexpr (is_cplx<S>::value) {
        double x, y, xp, yp;
        grid_xy(K, g, x, y);
        grid_xy(K, gp, xp, yp);
        const double dx = x - xp, dy = y - yp;
        return rscale<S>(kscale(K, g) * kscale(K, gp), hank_row<S>(K, sqrt(dx * dx + dy * dy)));
    } else if constexpr (sizeof(S) == sizeof(float)) {
        const int d1 = g % K.n - gp % K.n, d2 = g / K.n - gp / K.n;
        const float hf = (float)K.h;
        const float dx = (float)d1 * hf, dy = (float)d2 * hf;
        return (float)K.c0 * logf(dx * dx + dy * dy);
    } else {
        double x, y, xp, yp;
        grid_xy(K, g, x, y);
        grid_xy(K, gp, xp, yp);
        const double dx = x - xp, dy = y - yp;
        return K.c0 * log(dx * dx + dy * dy);
    }
}

template <class S>
__device__ __forceinline__ S kdiag(const KernelK& K, const double* a, int g)
{
    if constexpr (is_cplx<S>::value) {
        const double s2 = kscale(K, g) * kscale(K, g);
        return S(a[g] + s2 * K.hs_re, s2 * K.hs_im);
    } else {
        return S(a[g] + K.self);
    }
}

template <class S>
__device__ __forceinline__ S kproxy(const KernelK& K, double zx, double zy, int g)
{
    double x, y;
    grid_xy(K, g, x, y);
    if constexpr (is_cplx<S>::value) {
        const double dx = zx - x, dy = zy - y;
        return rscale<S>(kscale(K, g), hank_row<S>(K, sqrt(dx * dx + dy * dy)));
    } else if constexpr (sizeof(S) == sizeof(float)) {
        const float dx = (float)(zx - x), dy = (float)(zy - y);
        return (float)K.c0 * logf(dx * dx + dy * dy);
    } else {
        const double dx = zx - x, dy = zy - y;
        return K.c0 * log(dx * dx + dy * dy);
    }
}

}  // namespace rs
