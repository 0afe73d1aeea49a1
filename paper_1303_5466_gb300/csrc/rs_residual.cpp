// rs_residual.cpp -- FP64 direct-sum residual and the iterative refinement of low-precision
// solves (the paper's round of refinement, Sec. 5.3-5.4, repeated to a tolerance), plus the
// Helmholtz cell integral used on the diagonal.
#include <math.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "rs_host.h"

namespace rs {

// Integral of H0^(1)(kappa |y - x|) over the h x h cell centred at x.  In polar coordinates
// over the eight triangles of the square, with rho(th) = (h/2)/cos th,
//   int_0^rho r H0(kappa r) dr = (kappa rho H1(kappa rho) + 2i/pi) / kappa^2,
// and the remaining integral over th in [0, pi/4] is smooth: 48-point Gauss-Legendre.
void helmholtz_cell_integral(double h, double kappa, double* re, double* im)
{
    const int n = 48;
    std::vector<double> x(n), w(n);
    for (int i = 0; i < n; ++i) {                 // Legendre roots by Newton's method
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-15) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    double ar = 0.0, ai = 0.0;
    for (int i = 0; i < n; ++i) {
        const double th = 0.125 * M_PI * (1.0 + x[i]);
        const double z = kappa * 0.5 * h / std::cos(th);
        const double wt = 0.125 * M_PI * w[i] / (kappa * kappa);
        ar += wt * z * j1(z);                      // Re: kappa rho J1
        ai += wt * (z * y1(z) + 2.0 / M_PI);       // Im: kappa rho Y1 + 2/pi
    }
    *re = 8.0 * ar;
    *im = 8.0 * ai;
}

namespace {

// Offset table, FP64 diagonal, row scale and the grid -> input permutation, built once.
int residual_setup(rs_op* op, cudaStream_t st)
{
    if (op->d_ktab.p) return RS_OK;
    const int n = (int)op->n;
    const int64_t W = 2 * (int64_t)n - 1;
    const size_t N = (size_t)op->N;
    std::vector<double> a((size_t)N);
    RS_CUDA(cudaMemcpy(a.data(), op->d_a.p, sizeof(double) * N, cudaMemcpyDeviceToHost));
    if (op->kind == RS_HELMHOLTZ) {
        using Z = cplx<double>;
        RS_CUDA(op->d_ktab.alloc(sizeof(Z) * (size_t)(W * W)));
        RS_CUDA(launch_helmholtz_table(st, n, op->K.h, op->kappa, op->d_ktab.as<Z>()));
        std::vector<double> s(N);
        RS_CUDA(cudaMemcpy(s.data(), op->d_s.p, sizeof(double) * N, cudaMemcpyDeviceToHost));
        std::vector<Z> dg(N);
        std::vector<double> rsv(N);
        for (size_t g = 0; g < N; ++g) {            // original form: a + kappa^2 b (i/4) int_cell H0
            const double s2 = s[g] * s[g];
            dg[g] = Z(a[g] + s2 * op->K.hs_re, s2 * op->K.hs_im);
            rsv[g] = s2;
        }
        RS_CUDA(op->d_diag.alloc(sizeof(Z) * N));
        RS_CUDA(cudaMemcpy(op->d_diag.p, dg.data(), sizeof(Z) * N, cudaMemcpyHostToDevice));
        RS_CUDA(op->d_rs.alloc(sizeof(double) * N));
        RS_CUDA(cudaMemcpy(op->d_rs.p, rsv.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
    } else {
        RS_CUDA(op->d_ktab.alloc(sizeof(double) * (size_t)(W * W)));
        RS_CUDA(launch_laplace_table(st, n, op->K.h, op->K.c0, op->d_ktab.as<double>()));
        for (size_t g = 0; g < N; ++g) a[g] += op->K.self;
        RS_CUDA(op->d_diag.alloc(sizeof(double) * N));
        RS_CUDA(cudaMemcpy(op->d_diag.p, a.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
    }
    RS_CUDA(op->d_ing.alloc(sizeof(int64_t) * N));
    RS_CUDA(cudaMemcpyAsync(op->d_ing.p, op->input_of_g.data(), sizeof(int64_t) * N, cudaMemcpyHostToDevice, st));
    RS_CUDA(cudaStreamSynchronize(st));
    return RS_OK;
}

template <class Z>
int residual_t(rs_op* op, const Z* x, const Z* f, int64_t nrhs, Z* r, double* rel, cudaStream_t st)
{
    int rc = residual_setup(op, st);
    if (rc) return rc;
    const size_t bytes = sizeof(Z) * (size_t)(op->N * nrhs);
    RS_CUDA(op->r_xg.alloc(bytes));
    RS_CUDA(op->r_yg.alloc(bytes));
    RS_CUDA(op->r_norm.alloc(sizeof(double) * 2 * (size_t)nrhs));
    RS_CUDA(launch_residual<Z>(st, (int)op->n, (int)nrhs, op->d_ktab.as<Z>(), op->d_diag.as<Z>(),
                               op->kind == RS_HELMHOLTZ ? op->d_rs.as<double>() : nullptr, op->d_ing.as<int64_t>(), x,
                               f, op->r_xg.as<Z>(), op->r_yg.as<Z>(), r, op->r_norm.as<double>()));
    std::vector<double> nm(2 * (size_t)nrhs);
    RS_CUDA(cudaMemcpyAsync(nm.data(), op->r_norm.p, sizeof(double) * nm.size(), cudaMemcpyDeviceToHost, st));
    RS_CUDA(cudaStreamSynchronize(st));
    for (int64_t c = 0; c < nrhs; ++c)
        rel[c] = nm[2 * c + 1] > 0.0 ? std::sqrt(nm[2 * c] / nm[2 * c + 1]) : std::sqrt(nm[2 * c]);
    return RS_OK;
}

// FP32 (complex64) copies of the residual's table and diagonal, built once.
template <class Z, class L>
int residual_setup_lo(rs_op* op, cudaStream_t st)
{
    int rc = residual_setup(op, st);
    if (rc) return rc;
    if (op->d_ktab_lo.p) return RS_OK;
    const int64_t W = 2 * op->n - 1;
    RS_CUDA(op->d_ktab_lo.alloc(sizeof(L) * (size_t)(W * W)));
    RS_CUDA(op->d_diag_lo.alloc(sizeof(L) * (size_t)op->N));
    RS_CUDA(launch_narrow<Z, L>(st, W * W, op->d_ktab.as<Z>(), op->d_ktab_lo.as<L>()));
    RS_CUDA(launch_narrow<Z, L>(st, op->N, op->d_diag.as<Z>(), op->d_diag_lo.as<L>()));
    return RS_OK;
}

// Iterative refinement (Z: FP64 or complex128 solution and residual; L: FP32 or complex64):
//   x = A_eps^{-1} f;  r = f - A x by the FP64 direct sum;
//   repeat: dx = A_eps^{-1} r;  x += dx;  r -= A dx
// until max_c |r_c| / |f_c| <= refine_tol.  r - A dx equals f - A x in exact arithmetic; the
// corrections are small, so their products run in L with FP64 sums of 256-term tiles, which
// costs a fraction of the FP64 direct sum.  The tolerance is only ever declared met on an FP64
// direct-sum residual: when the updated r reaches it, r = f - A x is recomputed in FP64 and the
// loop goes on from that value if it falls short.
template <class Z, class L>
int refine_t(rs_op* op, const Z* fd, Z* xd, int64_t nrhs, cudaStream_t st)
{
    const size_t bytes = sizeof(Z) * (size_t)(op->N * nrhs);
    RS_CUDA(op->r_res.alloc(bytes));
    RS_CUDA(op->r_dx.alloc(bytes));
    std::vector<double> rel((size_t)nrhs, 1.0), fn((size_t)nrhs, 0.0);
    double worst = 1.0;
    int fp64_sums = 0;
    // r = f - A x by the FP64 direct sum; |f_c| from the same pass
    auto exact_residual = [&]() -> int {
        int rc = residual_t<Z>(op, xd, fd, nrhs, op->r_res.as<Z>(), rel.data(), st);
        if (rc) return rc;
        std::vector<double> nm(2 * (size_t)nrhs);
        RS_CUDA(cudaMemcpy(nm.data(), op->r_norm.p, sizeof(double) * nm.size(), cudaMemcpyDeviceToHost));
        for (int64_t c = 0; c < nrhs; ++c) fn[c] = std::sqrt(nm[2 * c + 1]);
        ++fp64_sums;
        return RS_OK;
    };
    for (int it = 1; it <= op->opts.refine_max_iter; ++it) {
        int rc;
        bool exact = true;
        if (it == 1) {
            if ((rc = apply_once(op, (const double*)fd, (double*)xd, nrhs, st))) return rc;
            if ((rc = exact_residual())) return rc;
        } else {
            if ((rc = apply_once(op, op->r_res.as<double>(), op->r_dx.as<double>(), nrhs, st))) return rc;
            RS_CUDA(launch_axpby<Z>(st, op->N * nrhs, Z(1.0), op->r_dx.as<Z>(), Z(1.0), xd));
            if ((rc = residual_setup_lo<Z, L>(op, st))) return rc;
            RS_CUDA(op->r_xg_lo.alloc(sizeof(L) * (size_t)(op->N * nrhs)));
            RS_CUDA(op->r_yg.alloc(bytes));
            RS_CUDA(op->r_norm.alloc(sizeof(double) * 2 * (size_t)nrhs));
            RS_CUDA(launch_residual_update<Z, L>(st, (int)op->n, (int)nrhs, op->d_ktab_lo.as<L>(),
                                                 op->d_diag_lo.as<L>(),
                                                 op->kind == RS_HELMHOLTZ ? op->d_rs.as<double>() : nullptr,
                                                 op->d_ing.as<int64_t>(), op->r_dx.as<Z>(), op->r_res.as<Z>(),
                                                 op->r_xg_lo.as<L>(), op->r_yg.as<Z>(), op->r_norm.as<double>()));
            std::vector<double> nm(2 * (size_t)nrhs);
            RS_CUDA(cudaMemcpyAsync(nm.data(), op->r_norm.p, sizeof(double) * nm.size(), cudaMemcpyDeviceToHost, st));
            RS_CUDA(cudaStreamSynchronize(st));
            for (int64_t c = 0; c < nrhs; ++c)
                rel[c] = fn[c] > 0.0 ? std::sqrt(nm[2 * c]) / fn[c] : std::sqrt(nm[2 * c]);
            exact = false;
        }
        worst = *std::max_element(rel.begin(), rel.end());
        if (!exact && worst <= op->opts.refine_tol) {      // confirm on the FP64 residual
            if ((rc = exact_residual())) return rc;
            worst = *std::max_element(rel.begin(), rel.end());
        }
        op->stats.refine_iters = it;
        op->stats.refine_residual = worst;
        op->stats.refine_fp64_sums = fp64_sums;
        if (worst <= op->opts.refine_tol) return RS_OK;
    }
    return fail(RS_E_NOT_CONVERGED, "refinement stopped at relative residual " + std::to_string(worst) + " after " +
                                        std::to_string(op->opts.refine_max_iter) + " solves");
}

}  // namespace

// Offset tables of the kernel for the factorization's entries (and the residual): FP64 or
// complex128, plus the FP32 / complex64 copy for the reduced precisions; sets op->K.tab.
int kernel_tables(rs_op* op, cudaStream_t st)
{
    RS_CUDA(cudaStreamSynchronize(st));          // a(x) and the scaling were uploaded on st
    int rc;
    if (op->kind == RS_HELMHOLTZ) {
        if (op->opts.precision == RS_C64_REFINED) {
            if ((rc = residual_setup_lo<cplx<double>, cplx<float>>(op, st))) return rc;
            op->K.tab = op->d_ktab_lo.p;
        } else {
            if ((rc = residual_setup(op, st))) return rc;
            op->K.tab = op->d_ktab.p;
        }
    } else if (op->opts.precision == RS_MIXED_FP32) {
        if ((rc = residual_setup_lo<double, float>(op, st))) return rc;
        op->K.tab = op->d_ktab_lo.p;
    } else {
        if ((rc = residual_setup(op, st))) return rc;
        op->K.tab = op->d_ktab.p;
    }
    RS_CUDA(cudaStreamSynchronize(st));
    return RS_OK;
}

// r = f - A x (device, N x nrhs column-major in input order, FP64 or complex128 by kernel);
// rel[c] = |r_c| / |f_c|.
int residual_apply(rs_op* op, const double* x, const double* f, int64_t nrhs, double* r, double* rel,
                   cudaStream_t st)
{
    if (op->kind == RS_HELMHOLTZ)
        return residual_t<cplx<double>>(op, (const cplx<double>*)x, (const cplx<double>*)f, nrhs, (cplx<double>*)r,
                                        rel, st);
    return residual_t<double>(op, x, f, nrhs, r, rel, st);
}

// x = A_eps^{-1} f (low-precision factors), r = f - A x (FP64 direct sum); repeat dx =
// A_eps^{-1} r, x += dx, r -= A dx (products in FP32 / complex64) until max_c |r_c| / |f_c| <=
// refine_tol on an FP64 direct-sum residual, or refine_max_iter solves were made.
int refine_solve(rs_op* op, const double* fd, double* xd, int64_t nrhs, cudaStream_t st)
{
    if (op->kind == RS_HELMHOLTZ)
        return refine_t<cplx<double>, cplx<float>>(op, (const cplx<double>*)fd, (cplx<double>*)xd, nrhs, st);
    return refine_t<double, float>(op, fd, xd, nrhs, st);
}

}  // namespace rs

using namespace rs;

extern "C" int rs_residual(rs_op* op, const void* x, const void* f, int64_t nrhs, double* rel_out, void* stream)
{
    if (!op || !x || !f || nrhs < 1 || !rel_out) return fail(RS_E_INVALID, "bad argument");
    int dev = 0;
    RS_CUDA(cudaGetDevice(&dev));
    if (dev != op->device) return fail(RS_E_INVALID, "the current device is not the one the operator was factored on");
    cudaStream_t st = (cudaStream_t)stream;
    if (on_other_device(x) || on_other_device(f))
        return fail(RS_E_INVALID, "x or f is device memory of another GPU than the operator's");
    const bool dx = is_device_ptr(x), df = is_device_ptr(f);
    if (dx != df) return fail(RS_E_INVALID, "x and f must both be device or both be host pointers");
    const size_t io = op->kind == RS_HELMHOLTZ ? 2 * sizeof(double) : sizeof(double);
    const size_t bytes = io * (size_t)(op->N * nrhs);
    DevMem hx, hf, r;
    const double* xd = (const double*)x;
    const double* fd = (const double*)f;
    if (!dx) {
        RS_CUDA(hx.alloc(bytes));
        RS_CUDA(hf.alloc(bytes));
        RS_CUDA(cudaMemcpyAsync(hx.p, x, bytes, cudaMemcpyHostToDevice, st));
        RS_CUDA(cudaMemcpyAsync(hf.p, f, bytes, cudaMemcpyHostToDevice, st));
        xd = hx.as<double>();
        fd = hf.as<double>();
    }
    RS_CUDA(r.alloc(bytes));
    return residual_apply(op, xd, fd, nrhs, r.as<double>(), rel_out, st);
}
