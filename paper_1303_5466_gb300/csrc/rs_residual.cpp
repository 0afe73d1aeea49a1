// rs_residual.cpp -- FP64 direct-sum residual and the iterative refinement of mixed-precision
// solves (the paper's one round of refinement, Sec. 5.3/5.4, repeated to a tolerance).
#include <math.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "rs_host.h"

namespace rs {

// Offset table, FP64 diagonal (a_g + self) and the grid -> input permutation, built once.
static int residual_setup(rs_op* op, cudaStream_t st)
{
    if (op->d_ktab.p) return RS_OK;
    const int n = (int)op->n;
    const int64_t W = 2 * (int64_t)n - 1;
    RS_CUDA(op->d_ktab.alloc(sizeof(double) * (size_t)(W * W)));
    RS_CUDA(launch_laplace_table(st, n, op->K.h, op->K.c0, op->d_ktab.as<double>()));
    RS_CUDA(op->d_diag.alloc(sizeof(double) * (size_t)op->N));
    // diagonal = a_g + self: a in grid order is already resident; add self on the device
    std::vector<double> selfv((size_t)op->N, op->K.self);
    DevMem tmp;
    RS_CUDA(tmp.alloc(sizeof(double) * (size_t)op->N));
    RS_CUDA(cudaMemcpyAsync(tmp.p, selfv.data(), sizeof(double) * selfv.size(), cudaMemcpyHostToDevice, st));
    RS_CUDA(cudaMemcpyAsync(op->d_diag.p, op->d_a.p, sizeof(double) * (size_t)op->N, cudaMemcpyDeviceToDevice, st));
    RS_CUDA(launch_axpby<double>(st, op->N, 1.0, tmp.as<double>(), 1.0, op->d_diag.as<double>()));
    RS_CUDA(op->d_ing.alloc(sizeof(int64_t) * (size_t)op->N));
    RS_CUDA(cudaMemcpyAsync(op->d_ing.p, op->input_of_g.data(), sizeof(int64_t) * (size_t)op->N,
                            cudaMemcpyHostToDevice, st));
    RS_CUDA(cudaStreamSynchronize(st));
    return RS_OK;
}

// r = f - A x (device, FP64, N x nrhs column-major in input order); rel[c] = |r_c| / |f_c|.
int residual_apply(rs_op* op, const double* x, const double* f, int64_t nrhs, double* r, double* rel,
                   cudaStream_t st)
{
    int rc = residual_setup(op, st);
    if (rc) return rc;
    const size_t bytes = sizeof(double) * (size_t)(op->N * nrhs);
    RS_CUDA(op->r_xg.alloc(bytes));
    RS_CUDA(op->r_yg.alloc(bytes));
    RS_CUDA(op->r_norm.alloc(sizeof(double) * 2 * (size_t)nrhs));
    RS_CUDA(launch_residual(st, (int)op->n, (int)nrhs, op->d_ktab.as<double>(), op->d_diag.as<double>(),
                            op->d_ing.as<int64_t>(), x, f, op->r_xg.as<double>(), op->r_yg.as<double>(), r,
                            op->r_norm.as<double>()));
    std::vector<double> nm(2 * (size_t)nrhs);
    RS_CUDA(cudaMemcpyAsync(nm.data(), op->r_norm.p, sizeof(double) * nm.size(), cudaMemcpyDeviceToHost, st));
    RS_CUDA(cudaStreamSynchronize(st));
    for (int64_t c = 0; c < nrhs; ++c)
        rel[c] = nm[2 * c + 1] > 0.0 ? std::sqrt(nm[2 * c] / nm[2 * c + 1]) : std::sqrt(nm[2 * c]);
    return RS_OK;
}

// x = 0; repeat: dx = A_eps^{-1} r (the low-precision factors), x += dx, r = f - A x (FP64),
// until max_c |r_c| / |f_c| <= refine_tol or refine_max_iter solves were made.
int refine_solve(rs_op* op, const double* fd, double* xd, int64_t nrhs, cudaStream_t st)
{
    const size_t bytes = sizeof(double) * (size_t)(op->N * nrhs);
    RS_CUDA(op->r_res.alloc(bytes));
    RS_CUDA(op->r_dx.alloc(bytes));
    RS_CUDA(cudaMemsetAsync(xd, 0, bytes, st));
    RS_CUDA(cudaMemcpyAsync(op->r_res.p, fd, bytes, cudaMemcpyDeviceToDevice, st));
    std::vector<double> rel((size_t)nrhs, 1.0);
    double worst = 1.0;
    for (int it = 1; it <= op->opts.refine_max_iter; ++it) {
        int rc = apply_once(op, op->r_res.as<double>(), op->r_dx.as<double>(), nrhs, st);
        if (rc) return rc;
        RS_CUDA(launch_axpby<double>(st, op->N * nrhs, 1.0, op->r_dx.as<double>(), 1.0, xd));
        rc = residual_apply(op, xd, fd, nrhs, op->r_res.as<double>(), rel.data(), st);
        if (rc) return rc;
        worst = *std::max_element(rel.begin(), rel.end());
        op->stats.refine_iters = it;
        op->stats.refine_residual = worst;
        if (worst <= op->opts.refine_tol) return RS_OK;
    }
    return fail(RS_E_NOT_CONVERGED, "refinement stopped at relative residual " + std::to_string(worst) + " after " +
                                        std::to_string(op->opts.refine_max_iter) + " solves");
}

}  // namespace rs

using namespace rs;

extern "C" int rs_residual(rs_op* op, const void* x, const void* f, int64_t nrhs, double* rel_out, void* stream)
{
    if (!op || !x || !f || nrhs < 1 || !rel_out) return fail(RS_E_INVALID, "bad argument");
    if (op->kind != RS_LAPLACE) return fail(RS_E_INVALID, "the direct-sum residual covers the Laplace kernel");
    int dev = 0;
    RS_CUDA(cudaGetDevice(&dev));
    if (dev != op->device) return fail(RS_E_INVALID, "the current device is not the one the operator was factored on");
    cudaStream_t st = (cudaStream_t)stream;
    const bool dx = is_device_ptr(x), df = is_device_ptr(f);
    if (dx != df) return fail(RS_E_INVALID, "x and f must both be device or both be host pointers");
    const size_t bytes = sizeof(double) * (size_t)(op->N * nrhs);
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
