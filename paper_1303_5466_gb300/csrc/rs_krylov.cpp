// rs_krylov.cpp -- the preconditioned iterative solver of Sec. 5.4: BiCGstab on A x = f with a
// right preconditioner M^{-1} (A M^{-1} y = f, x = M^{-1} y).  A is applied through its HSS
// form (rs_fwd_apply: the tree build of a forward-only operator, or any factored operator),
// M^{-1} through a factorization (rs_solve), e.g. the translation-invariant Helmholtz inverse
// (b = 1) for the Lippmann-Schwinger operator (b varying).  Every vector operation is a device
// kernel (k_krylov.cu); the scalars of the recurrence come back to the host once per dot
// product.
#include <math.h>

#include <cmath>

#include "rs.h"
#include "rs_host.h"
#include "rs_internal.h"

namespace rs {
namespace {

inline double mag(double v) { return std::fabs(v); }
inline double mag(const cplx<double>& v) { return std::hypot(v.re, v.im); }
inline double real_of(double v) { return v; }
inline double real_of(const cplx<double>& v) { return v.re; }
inline cplx<double> div_(const cplx<double>& a, const cplx<double>& b)
{
    const double d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
inline double div_(double a, double b) { return a / b; }

template <class T>
int bicgstab_t(rs_op* A, rs_op* M, const T* f, T* x, double tol, int max_iter, int* iters_out, double* rel_out,
               cudaStream_t st)
{
    const int64_t n = A->N;
    DevMem buf, part, sc;
    RS_CUDA(buf.alloc(sizeof(T) * (size_t)(8 * n)));
    RS_CUDA(part.alloc(sizeof(T) * (size_t)dot_partials()));
    RS_CUDA(sc.alloc(sizeof(T)));
    T* r = buf.as<T>();
    T* rh = r + n;
    T* p = rh + n;
    T* v = p + n;
    T* s = v + n;
    T* t = s + n;
    T* ph = t + n;
    T* sh = ph + n;
    auto dot = [&](const T* a, const T* b, T* out) -> int {
        RS_CUDA(launch_dot<T>(st, n, a, b, part.as<T>(), sc.as<T>()));
        RS_CUDA(cudaMemcpyAsync(out, sc.p, sizeof(T), cudaMemcpyDeviceToHost, st));
        RS_CUDA(cudaStreamSynchronize(st));
        return RS_OK;
    };
    const T one = T(1.0), zero = T(0.0);
    int rc;
    // x = 0, r = r^ = f
    RS_CUDA(launch_lincomb<T>(st, n, zero, f, zero, nullptr, zero, nullptr, x));
    RS_CUDA(launch_lincomb<T>(st, n, one, f, zero, nullptr, zero, nullptr, r));
    RS_CUDA(launch_lincomb<T>(st, n, one, f, zero, nullptr, zero, nullptr, rh));
    T ff;
    if ((rc = dot(f, f, &ff))) return rc;
    const double fnorm = std::sqrt(real_of(ff));
    *iters_out = 0;
    *rel_out = 1.0;
    if (!(fnorm > 0.0)) { *rel_out = 0.0; return RS_OK; }
    T rho_prev = one, alpha = one, omega = one;
    for (int it = 1; it <= max_iter; ++it) {
        T rho;
        if ((rc = dot(rh, r, &rho))) return rc;
        if (!(mag(rho) > 0.0)) return fail(RS_E_NOT_CONVERGED, "BiCGstab breakdown (rho = 0)");
        if (it == 1) {
            RS_CUDA(launch_lincomb<T>(st, n, one, r, zero, nullptr, zero, nullptr, p));
        } else {
            const T beta = div_(rho, rho_prev) * div_(alpha, omega);
            RS_CUDA(launch_lincomb<T>(st, n, one, r, beta, p, zero - beta * omega, v, p));
        }
        if ((rc = rs_solve(M, p, 1, ph, st))) return rc;              // p^ = M^{-1} p
        if ((rc = rs_fwd_apply(A, ph, 1, v, st))) return rc;          // v = A p^
        T rv;
        if ((rc = dot(rh, v, &rv))) return rc;
        if (!(mag(rv) > 0.0)) return fail(RS_E_NOT_CONVERGED, "BiCGstab breakdown (r^ . v = 0)");
        alpha = div_(rho, rv);
        RS_CUDA(launch_lincomb<T>(st, n, one, r, zero - alpha, v, zero, nullptr, s));
        T ss;
        if ((rc = dot(s, s, &ss))) return rc;
        double rel = std::sqrt(real_of(ss)) / fnorm;
        if (rel <= tol) {
            RS_CUDA(launch_lincomb<T>(st, n, one, x, alpha, ph, zero, nullptr, x));
            RS_CUDA(cudaStreamSynchronize(st));
            *iters_out = it;
            *rel_out = rel;
            return RS_OK;
        }
        if ((rc = rs_solve(M, s, 1, sh, st))) return rc;              // s^ = M^{-1} s
        if ((rc = rs_fwd_apply(A, sh, 1, t, st))) return rc;          // t = A s^
        T ts, tt;
        if ((rc = dot(t, s, &ts))) return rc;
        if ((rc = dot(t, t, &tt))) return rc;
        if (!(mag(tt) > 0.0)) return fail(RS_E_NOT_CONVERGED, "BiCGstab breakdown (t = 0)");
        omega = div_(ts, tt);
        RS_CUDA(launch_lincomb<T>(st, n, one, x, alpha, ph, omega, sh, x));
        RS_CUDA(launch_lincomb<T>(st, n, one, s, zero - omega, t, zero, nullptr, r));
        T rr;
        if ((rc = dot(r, r, &rr))) return rc;
        rel = std::sqrt(real_of(rr)) / fnorm;
        *iters_out = it;
        *rel_out = rel;
        if (rel <= tol) return RS_OK;
        if (!(mag(omega) > 0.0)) return fail(RS_E_NOT_CONVERGED, "BiCGstab breakdown (omega = 0)");
        rho_prev = rho;
    }
    return fail(RS_E_NOT_CONVERGED, "BiCGstab did not reach the tolerance in max_iter iterations");
}

}  // namespace
}  // namespace rs

using namespace rs;

int rs_bicgstab(rs_op* A, rs_op* M, const void* f, void* x, double tol, int max_iter, int* iters, double* rel_res,
                void* stream)
{
    if (!A || !M || !f || !x || !iters || !rel_res || f == x) return fail(RS_E_INVALID, "bad argument");
    if (!(tol > 0.0) || max_iter < 1) return fail(RS_E_INVALID, "need tol > 0 and max_iter >= 1");
    if (A->N != M->N || A->kind != M->kind) return fail(RS_E_INVALID, "A and M differ in size or kernel kind");
    if (M->opts.forward_only) return fail(RS_E_INVALID, "the preconditioner must be a factored operator");
    if (!is_device_ptr(f) || !is_device_ptr(x)) return fail(RS_E_INVALID, "f and x must be device pointers");
    {
        int dev = 0;
        RS_CUDA(cudaGetDevice(&dev));
        if (dev != A->device || dev != M->device)
            return fail(RS_E_INVALID, "the current device is not the one the operators were factored on");
        if (on_other_device(f) || on_other_device(x))
            return fail(RS_E_INVALID, "f or x is device memory of another GPU than the operators'");
    }
    const cudaStream_t st = (cudaStream_t)stream;
    if (A->kind == RS_HELMHOLTZ)
        return bicgstab_t<cplx<double>>(A, M, (const cplx<double>*)f, (cplx<double>*)x, tol, max_iter, iters, rel_res,
                                        st);
    return bicgstab_t<double>(A, M, (const double*)f, (double*)x, tol, max_iter, iters, rel_res, st);
}
