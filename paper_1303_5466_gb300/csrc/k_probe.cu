// k_probe.cu -- throughput probes of the pipes this library's factorization runs on.
//
// The factor and the solve are FP64 dense linear algebra, so the roofline that bounds them is
// the chip's FP64 rate, which GB300 gives through two routes: the FP64 FMA of the CUDA cores
// (DFMA) and the FP64 matrix instruction (mma.sync m8n8k4 .f64, "DMMA").  Each probe keeps
// every warp busy with independent register-only chains of one instruction kind, long enough
// that launch cost is negligible, at 16, 32 and 64 warps per SM, and returns the best rate
// from CUDA-event timing.  The
// larger of the two is the FP64 peak the benchmark divides by; their ratio decides which pipe
// the FP64 contractions should use.  A third probe measures the bf16 mma.sync rate that the
// digit-slice GEMM (k_gemm_oz.cu) runs its FP64 products on.
#include <algorithm>

#include "k_common.cuh"
#include "rs.h"
#include "rs_host.h"

namespace rs {

namespace {

constexpr int PROBE_NT = 256;
constexpr int PROBE_CHAINS = 8;

// DFMA: 8 independent chains per thread, a = a * m + c (m, c kept near 1 so nothing overflows
// or underflows over the iterations).
__global__ void __launch_bounds__(PROBE_NT) dfma_probe_kernel(int iters, double m, double c, double* out)
{
    double a[PROBE_CHAINS];
#pragma unroll
    for (int q = 0; q < PROBE_CHAINS; ++q) a[q] = 1.0 + 1e-3 * (threadIdx.x + q);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < PROBE_CHAINS; ++q) a[q] = fma(a[q], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < PROBE_CHAINS; ++q) s += a[q];
    if (s == 12345.678) out[blockIdx.x] = s;      // never true: keeps the chains live
}

// DFMA with CH independent chains whose multiplier and addend are per-chain registers
// (a = a * b_q + c_q).
template <int CH>
__global__ void __launch_bounds__(PROBE_NT) dfma_probe2_kernel(int iters, double m, double c, double* out)
{
    double a[CH], bq[CH], cq[CH];
#pragma unroll
    for (int q = 0; q < CH; ++q) {
        a[q] = 1.0 + 1e-3 * (threadIdx.x + q);
        bq[q] = m * (1.0 - 1e-9 * q);
        cq[q] = c * (1.0 + 1e-3 * q);
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < CH; ++q) a[q] = fma(a[q], bq[q], cq[q]);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < CH; ++q) s += a[q];
    if (s == 12345.678) out[blockIdx.x] = s;
}

// DMMA: 4 independent m8n8k4 accumulations per warp, D = A B + D with A, B fixed fragments of
// small values (each step adds a bounded amount; no overflow over the iterations).
__global__ void __launch_bounds__(PROBE_NT) dmma_probe_kernel(int iters, double av, double bv, double* out)
{
    double d[4][2];
#pragma unroll
    for (int q = 0; q < 4; ++q) d[q][0] = d[q][1] = 0.0;
    const double a = av * (1.0 + 1e-3 * (threadIdx.x & 31));
    const double b = bv;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                         : "+d"(d[q][0]), "+d"(d[q][1])
                         : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) s += d[q][0] + d[q][1];
    if (s == 12345.678) out[blockIdx.x] = s;
}

// bf16 mma.sync m16n8k16 with FP32 accumulation (the pipe of the digit-slice GEMM): 4
// independent accumulations per warp, operands fixed fragments of small values.
__global__ void __launch_bounds__(PROBE_NT) bf16_mma_probe_kernel(int iters, double* out)
{
    float d[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) d[q][e] = 0.0f;
    const uint32_t a = 0x3f803f80u ^ (threadIdx.x & 1u), b = 0x3c003c00u;   // bf16 1.0 and 2^-7
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                         "{%8,%9}, {%0,%1,%2,%3};"
                         : "+f"(d[q][0]), "+f"(d[q][1]), "+f"(d[q][2]), "+f"(d[q][3])
                         : "r"(a), "r"(a), "r"(a), "r"(a), "r"(b), "r"(b));
    }
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) s += d[q][e];
    if (s == 12345.678f) out[blockIdx.x] = s;
}

}  // namespace

}  // namespace rs

using namespace rs;

extern "C" int rs_fp64_probe(int kind, double* tflops_out, void* stream)
{
    if (!tflops_out || (kind != RS_PROBE_DFMA && kind != RS_PROBE_DMMA && kind != RS_PROBE_BF16_MMA))
        return fail(RS_E_INVALID, "bad argument");
    const cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    RS_CUDA(cudaGetDevice(&dev));
    RS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DevMem out;
    RS_CUDA(out.alloc(sizeof(double) * (size_t)(8 * sms)));
    cudaEvent_t e0, e1;
    RS_CUDA(cudaEventCreate(&e0));
    RS_CUDA(cudaEventCreate(&e1));
    // 2, 4 and 8 CTAs of 256 threads per SM (16 to 64 warps); the best rate of three timed
    // launches of each, after one warm-up launch
    double best_rate = 0.0;
    // DFMA forms: 0 = eight chains sharing their multiplier and addend, 1 = four and 2 = two
    // chains with their own
    const int forms = kind == RS_PROBE_DFMA ? 3 : 1;
    for (int form = 0; form < forms; ++form)
    for (int per_sm = 2; per_sm <= 8; per_sm *= 2) {
        const int blocks = per_sm * sms;
        const int chains = kind != RS_PROBE_DFMA ? 1 : form == 0 ? PROBE_CHAINS : form == 1 ? 4 : 2;
        const int iters = kind == RS_PROBE_DFMA ? 32768 * PROBE_CHAINS / chains / per_sm
                          : kind == RS_PROBE_DMMA ? 8192 / per_sm : 65536 / per_sm;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, st);
            count_launches(1);
            if (kind == RS_PROBE_DFMA && form == 0)
                dfma_probe_kernel<<<blocks, PROBE_NT, 0, st>>>(iters, 0.9999999, 1e-7, out.as<double>());
            else if (kind == RS_PROBE_DFMA && form == 1)
                dfma_probe2_kernel<4><<<blocks, PROBE_NT, 0, st>>>(iters, 0.9999999, 1e-7, out.as<double>());
            else if (kind == RS_PROBE_DFMA)
                dfma_probe2_kernel<2><<<blocks, PROBE_NT, 0, st>>>(iters, 0.9999999, 1e-7, out.as<double>());
            else if (kind == RS_PROBE_DMMA)
                dmma_probe_kernel<<<blocks, PROBE_NT, 0, st>>>(iters, 1e-3, 1e-3, out.as<double>());
            else
                bf16_mma_probe_kernel<<<blocks, PROBE_NT, 0, st>>>(iters, out.as<double>());
            cudaEventRecord(e1, st);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return cuda_fail(e, "probe kernel");
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep == 0 || ms <= 0.0f) continue;
            const double threads = (double)blocks * PROBE_NT;
            // DFMA: 2 flops per FMA; DMMA: 8 x 8 x 4 FMAs = 512 flops per warp-instruction;
            // bf16: 16 x 8 x 16 FMAs = 4096 flops per warp-instruction
            const double flops = kind == RS_PROBE_DFMA ? threads * iters * chains * 2.0
                                 : kind == RS_PROBE_DMMA ? threads / 32.0 * iters * 4 * 512.0
                                                         : threads / 32.0 * iters * 4 * 4096.0;
            best_rate = std::max(best_rate, flops / (ms * 1e-3) / 1e12);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    RS_CUDA(cudaGetLastError());
    *tflops_out = best_rate;
    return RS_OK;
}
