// k_common.cuh -- device helpers shared by the library's kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "k_scalar.cuh"
#include "rs_internal.h"

namespace rs {

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl_xor_(v, o);
    return v;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// Block-wide sum with a fixed reduction order (same result in every CTA for the same data);
// scratch holds NT / 32 + 1 doubles.  Warp 0 adds the warp sums, so the FP64 pipe sees one
// short butterfly rather than every thread adding them all.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* scratch)
{
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) scratch[w] = v;
    __syncthreads();
    if (w == 0) {
        double t = l < NT / 32 ? scratch[l] : 0.0;
#pragma unroll
        for (int o = NT / 64; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (l == 0) scratch[NT / 32] = t;
    }
    __syncthreads();
    return scratch[NT / 32];
}

template <int NT>
__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v, unsigned long long* scratch)
{
    v = warp_max_u64(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) scratch[w] = v;
    __syncthreads();
    unsigned long long t = 0;
#pragma unroll
    for (int q = 0; q < NT / 32; ++q) t = scratch[q] > t ? scratch[q] : t;
    return t;
}

// Barrier among the CTAs of one group (all co-resident: cooperative launch).  `ctr` grows
// monotonically; the caller passes target = (barrier index + 1) * group size.  Every wait is
// bounded: past `limit` polls the CTA sets DEV_TIMEOUT in *status and the barrier returns
// false, as it does when another CTA has already flagged a timeout.
__device__ __forceinline__ bool group_sync(unsigned int* ctr, unsigned int target, int* status, long long limit)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        __threadfence();
        atomicAdd(ctr, 1u);
        long long it = 0;
        while (ld_acquire_u32(ctr) < target) {
            if (*(volatile int*)status & DEV_TIMEOUT) { ok = 0; break; }
            if (++it > limit) { atomicOr(status, DEV_TIMEOUT); ok = 0; break; }
            __nanosleep(32);
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Squared norm -> pivot key (see KEY_BITS in rs_internal.h).
__device__ __forceinline__ unsigned long long pivot_key(double nrm2, int col)
{
    if (!(nrm2 > 0.0)) nrm2 = 0.0;
    unsigned long long u = (unsigned long long)__double_as_longlong(nrm2);
    return (u & ~KEY_MASK) | (KEY_MASK - (unsigned long long)col);
}

}  // namespace rs
