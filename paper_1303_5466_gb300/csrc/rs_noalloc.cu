// rs_noalloc.cu -- rs_solve_noalloc: the inverse apply with its workspace in a fixed device
// array, for callers that must not allocate device memory during a solve.
//
// Such callers include serving processes whose device memory is owned entirely by another
// allocator (a framework's caching allocator, or a fixed budget split ahead of time), where a
// cudaMalloc may fail or break the budget, and latency-bound request paths, where a
// cudaMalloc/cudaFree pair would synchronise the device.  rs_solve grows its workspace with
// cudaMalloc on first use; this entry point instead takes its workspace from the static array
// below and calls no allocating routine at all.
#include <mutex>

#include "rs_host.h"

namespace rs {

// Workspace of rs_solve_noalloc: RS_NOALLOC_SCRATCH_DOUBLES doubles (32 MiB) in device
// memory, reserved on every GPU that loads the library until the process exits.  In host
// code the symbol is only a stand-in: kernels receive the device address taken below.
static __device__ __align__(256) double g_noalloc_scratch[RS_NOALLOC_SCRATCH_DOUBLES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[MAX_DEVICES] = {};

// Device address of the scratch array on `dev` (which must be current), looked up once per
// device.
int scratch_address(int dev, double** out)
{
    if (dev < 0 || dev >= MAX_DEVICES) return fail(RS_E_INVALID, "device index out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_ptr[dev] = (double*)p;
    }
    *out = g_scratch_ptr[dev];
    return RS_OK;
}

}  // namespace
}  // namespace rs

using namespace rs;

extern "C" int rs_solve_noalloc(rs_op* op, const void* f, int64_t nrhs, void* x, void* stream)
{
    if (!op || !f || !x || nrhs < 1) return fail(RS_E_INVALID, "bad argument");
    // Bound nrhs before any size arithmetic: the workspace needs at least N doubles per
    // column, so a larger nrhs cannot fit (and would overflow the layout's products).
    if (op->N < 1 || nrhs > (int64_t)RS_NOALLOC_SCRATCH_DOUBLES / op->N)
        return fail(RS_E_INVALID, "rs_solve_noalloc: nrhs=" + std::to_string(nrhs) +
                                      " needs more workspace than its fixed scratch of " +
                                      std::to_string((int64_t)RS_NOALLOC_SCRATCH_DOUBLES) + " doubles (use rs_solve)");
    if (f == x) return fail(RS_E_INVALID, "x may not alias f");
    if (op->kind != RS_LAPLACE || op->opts.precision != RS_FP64 || op->opts.forward_only)
        return fail(RS_E_INVALID, "rs_solve_noalloc covers real FP64 (RS_FP64 Laplace) factored operators");
    int dev = 0;
    RS_CUDA(cudaGetDevice(&dev));
    if (dev != op->device) return fail(RS_E_INVALID, "the current device is not the one the operator was factored on");
    if (on_other_device(f) || on_other_device(x))
        return fail(RS_E_INVALID, "f or x is device memory of another GPU than the operator's");
    if (!is_device_ptr(f) || !is_device_ptr(x))
        return fail(RS_E_INVALID, "rs_solve_noalloc takes device pointers only (host buffers would need staging)");
    const SolveLayout Ls = solve_layout(op, nrhs);
    const int64_t need = Ls.total();
    if (need > (int64_t)RS_NOALLOC_SCRATCH_DOUBLES)
        return fail(RS_E_INVALID, "rs_solve_noalloc needs " + std::to_string(need) + " doubles of workspace for nrhs=" +
                                      std::to_string(nrhs) + "; its fixed scratch holds " +
                                      std::to_string((int64_t)RS_NOALLOC_SCRATCH_DOUBLES) + " (use fewer RHS or rs_solve)");
    double* base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc) return rc;
    // FP64 operator: workspace counts are in doubles
    double* w = base;
    double* g = w + Ls.n_w;
    double* phi = g + Ls.n_g;
    double* u = phi + Ls.n_g;
    double* out = u + Ls.n_u;
    double* t = out + Ls.n_u;
    double* z = t + Ls.n_t;
    SolveWork ws{w, g, phi, u, out, t, z};
    return solve_run(op, Ls, ws, (const double*)f, (double*)x, nrhs, (cudaStream_t)stream, false);
}
