// k_linalg.cu -- batched dense kernels of the inversion and solve phases.
//
//   gj_inverse : in-place Gauss-Jordan inverse with partial pivoting (F_i^{-1}, E_i)
//   gemm       : grouped GEMM over the boxes of a level (E_i^{-1} = R_i F_i^{-1} L_i)
//   matvec     : batched y = alpha op(A) x + beta y for nrhs right-hand sides (Algorithm 6)
//   gathers    : index gathers/scatters between the tree levels of the solve
#include <float.h>

#include "k_common.cuh"
#include "k_matvec.cuh"

namespace rs {

// ------------------------------------------------------------------ Gauss-Jordan inverse
// Blocked in-place Gauss-Jordan inverse with partial pivoting, G CTAs per matrix.  Columns are
// cut into panels of NB; panel q belongs to CTA q % G.  Block step q:
//   1. the owner runs unblocked Gauss-Jordan on its panel alone (pivot = largest |A_ic|,
//      i >= c, lowest i on ties; the row swap only touches the panel), leaving in the panel
//      P = the panel of the partial inverse, and publishes the NB pivot rows;
//   2. after one barrier every CTA updates each of its other columns j: apply the NB row
//      swaps, then A[:, j] = D_K A[:, j] + P A[K, j] (D_K zeroes the panel's rows K), a rank-NB
//      update with NB FMAs per element loaded.
// This equals the unblocked algorithm step for step (same pivots, same operations per row).
// A pivot with |pivot| not above 1e3 * unit roundoff * (largest earlier pivot of the same CTA)
// sets DEV_SINGULAR; the loop still finishes.  The panel arithmetic (pivot values and the
// panel's own elimination) runs in FP64 for every storage type T; the rank-NB trailing update
// runs in T.
template <int NT, int NB, bool SP, class T>
__global__ void __launch_bounds__(NT) gj_kernel(int G, const int32_t* __restrict__ msz, const int64_t* __restrict__ off,
        T* __restrict__ Aall, int32_t* __restrict__ ipiv, const int64_t* __restrict__ ipiv_off,
        int* __restrict__ pivbuf, unsigned int* __restrict__ bar, int* __restrict__ status, long long spin)
{
    constexpr int CB = 32;                 // own columns updated per chunk
    using W = typename sc_traits<T>::wide;      // FP64 panel arithmetic
    extern __shared__ double sm[];
    __shared__ double dred[NT / 32];
    __shared__ int ired[NT / 32];
    __shared__ int s_piv[NB];
    __shared__ W s_row[NB];
    __shared__ T s_aK[NB][CB];
    __shared__ int s_col[CB];
    const int b = blockIdx.x / G, gi = blockIdx.x - (blockIdx.x / G) * G;
    const int m = msz[b];
    T* __restrict__ A = Aall + off[b];
    W* f = (W*)sm;                         // m: the current pivot column (panel step)
    // SP: the owner factors its panel in shared memory (NB columns of m after f), so the
    // column steps of the panel -- the serial part of a block step -- touch no global memory
    T* pan = (T*)(sm + (((size_t)sizeof(W) * m + 15) / 16) * 2);
    int32_t* ip = ipiv + ipiv_off[b];
    int* pb = pivbuf + (int64_t)b * 2 * NB;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int npan = (m + NB - 1) / NB;
    double maxpiv = 0.0;
    for (int q = 0; q < npan; ++q) {
        const int k0 = q * NB, kw = min(NB, m - k0);
        if (q % G == gi) {
            T* pbase = SP ? pan : A + (int64_t)k0 * m;      // panel column jj at pbase + jj m
            if (SP) {
                for (int e = threadIdx.x; e < m * kw; e += NT) pan[e] = A[(int64_t)k0 * m + e];
                __syncthreads();
            }
            for (int t = 0; t < kw; ++t) {
                const int c = k0 + t;
                const T* col = pbase + (int64_t)t * m;
                double best = -1.0;
                int bi = m;
                for (int i = c + threadIdx.x; i < m; i += NT) {
                    const double a = absd(col[i]);
                    if (a > best) { best = a; bi = i; }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
                }
                if (lane == 0) { dred[warp] = best; ired[warp] = bi; }
                __syncthreads();
                if (threadIdx.x == 0) {
                    double bb = dred[0];
                    int ii = ired[0];
                    for (int w = 1; w < NT / 32; ++w)
                        if (dred[w] > bb || (dred[w] == bb && ired[w] < ii)) { bb = dred[w]; ii = ired[w]; }
                    s_piv[t] = ii < m ? ii : c;
                    ip[c] = s_piv[t];
                }
                __syncthreads();
                const int p = s_piv[t];
                if (threadIdx.x < kw && p != c) {           // swap rows c, p inside the panel
                    T* cj = pbase + (int64_t)threadIdx.x * m;
                    const T u = cj[c];
                    cj[c] = cj[p];
                    cj[p] = u;
                }
                __syncthreads();
                for (int i = threadIdx.x; i < m; i += NT) f[i] = cast_<W>(col[i]);
                if (threadIdx.x < kw) s_row[threadIdx.x] = cast_<W>(pbase[(int64_t)threadIdx.x * m + c]);
                __syncthreads();
                const W pv = f[c];
                const double apv = absd(pv);
                if (threadIdx.x == 0 && (!(apv > 1e3 * 0.5 * DBL_EPSILON * maxpiv) || !finite_(pv)))
                    atomicOr(status, DEV_SINGULAR);
                maxpiv = fmax(maxpiv, apv);
                const W pinv = (apv > 0.0) ? W(1.0) / pv : W(0.0);
                for (int e = threadIdx.x; e < m * kw; e += NT) {
                    const int jj = e / m, i = e - jj * m;
                    T* cj = pbase + (int64_t)jj * m;
                    if (k0 + jj == c) {
                        cj[i] = cast_<T>((i == c) ? pinv : -f[i] * pinv);
                    } else {
                        const W aj = s_row[jj] * pinv;
                        cj[i] = cast_<T>((i == c) ? aj : fma_(-f[i], aj, cast_<W>(cj[i])));
                    }
                }
                __syncthreads();
            }
            if (SP) {
                for (int e = threadIdx.x; e < m * kw; e += NT) A[(int64_t)k0 * m + e] = pan[e];
            }
            if (threadIdx.x < kw) pb[(q & 1) * NB + threadIdx.x] = s_piv[threadIdx.x];
        }
        if (G > 1) {
            if (!group_sync(bar + b, (unsigned)(q + 1) * (unsigned)G, status, spin)) return;
        } else {
            __syncthreads();
        }
        if (threadIdx.x < kw) s_piv[threadIdx.x] = (G > 1) ? __ldcg(pb + (q & 1) * NB + threadIdx.x) : pb[(q & 1) * NB + threadIdx.x];
        __syncthreads();
        // trailing update of this CTA's other columns, CB at a time
        int qq = gi, jin = 0;
        while (qq < npan) {
            int nc = 0;
            while (nc < CB && qq < npan) {
                if (qq == q) { qq += G; jin = 0; continue; }
                const int w = min(NB, m - qq * NB);
                if (threadIdx.x == 0) s_col[nc] = qq * NB + jin;
                ++nc;
                if (++jin == w) { qq += G; jin = 0; }
            }
            __syncthreads();
            if (nc == 0) break;
            // row swaps of block q, then the pivot rows a_K of each column
            if (threadIdx.x < nc) {
                T* cj = A + (int64_t)s_col[threadIdx.x] * m;
                for (int t = 0; t < kw; ++t) {
                    const int p = s_piv[t];
                    if (p != k0 + t) {
                        const T u = cj[k0 + t];
                        cj[k0 + t] = cj[p];
                        cj[p] = u;
                    }
                }
                for (int t = 0; t < kw; ++t) s_aK[t][threadIdx.x] = cj[k0 + t];
            }
            __syncthreads();
            for (int i = threadIdx.x; i < m; i += NT) {
                T P[NB];
#pragma unroll
                for (int t = 0; t < NB; ++t) P[t] = (t < kw) ? ldcg_(A + (int64_t)(k0 + t) * m + i) : (T)0;
                const bool inK = (i >= k0) && (i < k0 + kw);
                for (int jj = 0; jj < nc; ++jj) {
                    T* cj = A + (int64_t)s_col[jj] * m;
                    T v = inK ? (T)0 : cj[i];
#pragma unroll
                    for (int t = 0; t < NB; ++t) v = fma_(P[t], s_aK[t][jj], v);
                    cj[i] = v;
                }
            }
            __syncthreads();
        }
    }
}

// Undo the row exchanges: swap columns (c, ipiv[c]) for c = m-1 .. 0.  One CTA per matrix.
template <class T>
__global__ void __launch_bounds__(256) gj_unpivot_kernel(const int32_t* __restrict__ msz, const int64_t* __restrict__ off,
        T* __restrict__ Aall, const int32_t* __restrict__ ipiv, const int64_t* __restrict__ ipiv_off)
{
    const int b = blockIdx.x;
    const int m = msz[b];
    T* A = Aall + off[b];
    const int32_t* ip = ipiv + ipiv_off[b];
    for (int c = m - 1; c >= 0; --c) {
        const int p = ip[c];
        if (p == c) continue;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const T t = A[(int64_t)c * m + i];
            A[(int64_t)c * m + i] = A[(int64_t)p * m + i];
            A[(int64_t)p * m + i] = t;
        }
        __syncthreads();
    }
}

constexpr int GJ_NT = 256, GJ_NB = 8;

// Dynamic shared memory of the GJ kernel: the pivot column f, and with sp the owner's panel.
template <class T>
static size_t gj_shm(int max_m, bool sp)
{
    const size_t fb = ((sizeof(typename sc_traits<T>::wide) * (size_t)max_m + 15) / 16) * 16;
    return fb + (sp ? sizeof(T) * (size_t)GJ_NB * (size_t)max_m : 0) + 64;
}
// Panels go to shared memory for a launch of a single matrix (the root, where the panel steps
// are the serial part and every SM shares the one matrix) when the CTA stays within 160 KB;
// with more matrices the smaller CTA keeps more CTAs, and so more panels, resident (measured
// at 512^2: the root 61 -> 55 ms, the 2- and 4-matrix levels slower with the larger CTA).
template <class T>
static bool gj_sp(int max_m, int nb) { return nb == 1 && gj_shm<T>(max_m, true) <= 160 * 1024; }

template <bool SP, class T>
static int gj_capacity(size_t shm)
{
    if (cudaFuncSetAttribute(gj_kernel<GJ_NT, GJ_NB, SP, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) !=
        cudaSuccess)
        return 0;
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gj_kernel<GJ_NT, GJ_NB, SP, T>, GJ_NT, shm) != cudaSuccess)
        return 0;
    return per_sm * sms;
}

template <class T>
int gj_max_ctas(int max_m, int nb)
{
    const bool sp = gj_sp<T>(max_m, nb);
    const size_t shm = gj_shm<T>(max_m, sp);
    return sp ? gj_capacity<true, T>(shm) : gj_capacity<false, T>(shm);
}

int gj_panel_width() { return GJ_NB; }

template <bool SP, class T>
static cudaError_t launch_gj_t(cudaStream_t st, int nb, int G, const int32_t* m, const int64_t* off, T* A,
                               int32_t* ipiv, const int64_t* ipiv_off, int* pivbuf, unsigned int* bar, int* status,
                               long long spin_limit, size_t shm)
{
    cudaError_t e = cudaFuncSetAttribute(gj_kernel<GJ_NT, GJ_NB, SP, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)shm);
    if (e != cudaSuccess) return e;
    count_launches(1);
    if (G == 1) {
        gj_kernel<GJ_NT, GJ_NB, SP, T><<<nb, GJ_NT, shm, st>>>(G, m, off, A, ipiv, ipiv_off, pivbuf, bar, status,
                                                               spin_limit);
        return cudaGetLastError();
    }
    void* args[] = {(void*)&G, (void*)&m, (void*)&off, (void*)&A, (void*)&ipiv, (void*)&ipiv_off, (void*)&pivbuf,
                    (void*)&bar, (void*)&status, (void*)&spin_limit};
    return cudaLaunchCooperativeKernel((void*)gj_kernel<GJ_NT, GJ_NB, SP, T>, dim3((unsigned)(nb * G)), dim3(GJ_NT),
                                       args, shm, st);
}

template <class T>
cudaError_t launch_gj_inverse(cudaStream_t st, int nb, int G, const int32_t* m, const int64_t* off, T* A,
                              int32_t* ipiv, const int64_t* ipiv_off, int* pivbuf, unsigned int* bar, int* status,
                              long long spin_limit, int max_m)
{
    if (nb <= 0 || max_m <= 0) return cudaSuccess;
    const bool sp = gj_sp<T>(max_m, nb);
    const size_t shm = gj_shm<T>(max_m, sp);
    cudaError_t e = sp ? launch_gj_t<true, T>(st, nb, G, m, off, A, ipiv, ipiv_off, pivbuf, bar, status, spin_limit, shm)
                       : launch_gj_t<false, T>(st, nb, G, m, off, A, ipiv, ipiv_off, pivbuf, bar, status, spin_limit,
                                               shm);
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    count_launches(1);
    gj_unpivot_kernel<T><<<nb, 256, 0, st>>>(m, off, A, ipiv, ipiv_off);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ grouped GEMM
// 64 x 64 tile per CTA, 256 threads with a 4 x 4 register block each, K in steps of 16.
template <class T>
__global__ void __launch_bounds__(256) gemm_kernel(const GemmProb* __restrict__ probs, int np,
        const T* __restrict__ Ab, const T* __restrict__ Bb, T* Cb, const T* C0b)
{
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const int64_t t = blockIdx.x;
    int lo = 0, hi = np - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (probs[mid].tile0 <= t) lo = mid; else hi = mid - 1;
    }
    const GemmProb P = probs[lo];
    const int64_t lt = t - P.tile0;
    int tm, tn;
    if (P.lower) {           // row-by-row enumeration of the lower triangle of tiles
        tm = (int)((sqrt(8.0 * (double)lt + 1.0) - 1.0) * 0.5);
        while ((int64_t)tm * (tm + 1) / 2 > lt) --tm;
        while ((int64_t)(tm + 1) * (tm + 2) / 2 <= lt) ++tm;
        tn = (int)(lt - (int64_t)tm * (tm + 1) / 2);
    } else {
        tm = (int)(lt % P.tiles_m);
        tn = (int)(lt / P.tiles_m);
    }
    const int row0 = tm * BM, col0 = tn * BN;
    const T* A = Ab + P.a_off;
    const T* B = Bb + P.b_off;
    T* C = Cb + P.c_off;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[u][w] = 0;
    for (int k0 = 0; k0 < P.K; k0 += BK) {
        for (int e = threadIdx.x; e < BM * BK; e += 256) {
            const int i = e % BM, kk = e / BM;
            const int gi = row0 + i, gk = k0 + kk;
            T v = 0;
            if (gi < P.M && gk < P.K) v = P.ta ? A[(int64_t)gi * P.lda + gk] : A[(int64_t)gk * P.lda + gi];
            As[kk][i] = v;
        }
        for (int e = threadIdx.x; e < BN * BK; e += 256) {
            const int kk = e % BK, j = e / BK;
            const int gj = col0 + j, gk = k0 + kk;
            T v = 0;
            if (gj < P.N && gk < P.K) v = P.tb ? B[(int64_t)gk * P.ldb + gj] : B[(int64_t)gj * P.ldb + gk];
            Bs[kk][j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = As[kk][tx + 16 * u];
#pragma unroll
            for (int w = 0; w < 4; ++w) bv[w] = Bs[kk][ty + 16 * w];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[u][w] = fma_(a[u], bv[w], acc[u][w]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int gi = row0 + tx + 16 * u, gj = col0 + ty + 16 * w;
            if (gi < P.M && gj < P.N) {
                T* c = C + (int64_t)gj * P.ldc + gi;
                const T c0 = (P.beta == 0.0) ? (T)0 : C0b[P.c0_off + (int64_t)gj * P.ldc0 + gi];
                *c = (T)P.alpha * acc[u][w] + (T)P.beta * c0;
            }
        }
}

template <class T>
cudaError_t launch_gemm(cudaStream_t st, const GemmProb* probs, int np, int64_t tiles, const T* A, const T* B, T* C,
                        const T* C0)
{
    if (np <= 0 || tiles <= 0) return cudaSuccess;
    count_launches(1);
    gemm_kernel<T><<<(unsigned)tiles, 256, 0, st>>>(probs, np, A, B, C, C0);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ batched matvec(s)
template <class T, int RB>
__global__ void __launch_bounds__(256) matvec_kernel(const MatvecProb* __restrict__ probs,
        const int64_t* __restrict__ blk0, int np, const T* __restrict__ Ab, const T* __restrict__ xb,
        T* __restrict__ yb, int nrhs)
{
    __shared__ T part[256 * 8];
    const int64_t t = blockIdx.x;
    const int pi = find_block(blk0, np, t);
    const MatvecProb P = probs[pi];
    matvec_block<T, RB>(P, (int)(t - blk0[pi]) * RB, Ab + P.a_off, xb + P.x_off * nrhs, yb + P.y_off * nrhs, nrhs,
                        part);
}

int matvec_rows_per_block(int64_t blocks64)
{
    // enough blocks for four CTAs per SM, else smaller blocks (more column phases per row)
    if (blocks64 >= 608) return 64;
    if (2 * blocks64 >= 608) return 32;
    return 16;
}

template <class T>
cudaError_t launch_matvec(cudaStream_t st, const MatvecProb* probs, const int64_t* blk0, int np, int64_t blocks,
                          const T* A, const T* x, T* y, int nrhs, int rb)
{
    if (np <= 0 || blocks <= 0) return cudaSuccess;
    count_launches(1);
    if (rb == 16) matvec_kernel<T, 16><<<(unsigned)blocks, 256, 0, st>>>(probs, blk0, np, A, x, y, nrhs);
    else if (rb == 32) matvec_kernel<T, 32><<<(unsigned)blocks, 256, 0, st>>>(probs, blk0, np, A, x, y, nrhs);
    else matvec_kernel<T, 64><<<(unsigned)blocks, 256, 0, st>>>(probs, blk0, np, A, x, y, nrhs);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ gathers
template <class T>
__global__ void gather_rows_kernel(int64_t count, const int64_t* __restrict__ idx, const T* __restrict__ in,
                                   T* __restrict__ out, int nrhs)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count * nrhs) return;
    const int64_t p = e / nrhs;
    const int c = (int)(e - p * nrhs);
    out[e] = in[idx[p] * nrhs + c];
}

template <class T>
__global__ void scatter_rows_kernel(int64_t count, const int64_t* __restrict__ idx, const T* __restrict__ in,
                                    T* __restrict__ out, int nrhs)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count * nrhs) return;
    const int64_t p = e / nrhs;
    const int c = (int)(e - p * nrhs);
    out[idx[p] * nrhs + c] = in[e];
}

template <class Ti, class To>
__global__ void gather_cm_kernel(int64_t count, const int64_t* __restrict__ idx, const Ti* __restrict__ in,
                                 int64_t N, To* __restrict__ out, int nrhs)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count * nrhs) return;
    const int64_t p = e / nrhs;
    const int c = (int)(e - p * nrhs);
    out[e] = cast_<To>(in[(int64_t)c * N + idx[p]]);
}

template <class Ti, class To>
__global__ void scatter_cm_kernel(int64_t count, const int64_t* __restrict__ idx, const Ti* __restrict__ in,
                                  int64_t N, To* __restrict__ out, int nrhs)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count * nrhs) return;
    const int64_t p = e / nrhs;
    const int c = (int)(e - p * nrhs);
    out[(int64_t)c * N + idx[p]] = cast_<To>(in[e]);
}

template <class T>
__global__ void axpby_kernel(int64_t n, T a, const T* __restrict__ x, T b, T* __restrict__ y)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) y[e] = fma_(a, x[e], b * y[e]);
}

static unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

template <class T>
cudaError_t launch_gather_rows(cudaStream_t st, int64_t count, const int64_t* idx, const T* in, T* out, int nrhs)
{
    if (count <= 0) return cudaSuccess;
    count_launches(1);
    gather_rows_kernel<T><<<nblk(count * nrhs), 256, 0, st>>>(count, idx, in, out, nrhs);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_scatter_rows(cudaStream_t st, int64_t count, const int64_t* idx, const T* in, T* out, int nrhs)
{
    if (count <= 0) return cudaSuccess;
    count_launches(1);
    scatter_rows_kernel<T><<<nblk(count * nrhs), 256, 0, st>>>(count, idx, in, out, nrhs);
    return cudaGetLastError();
}

template <class Ti, class To>
cudaError_t launch_gather_cm(cudaStream_t st, int64_t count, const int64_t* idx, const Ti* in, int64_t N, To* out,
                             int nrhs)
{
    if (count <= 0) return cudaSuccess;
    count_launches(1);
    gather_cm_kernel<Ti, To><<<nblk(count * nrhs), 256, 0, st>>>(count, idx, in, N, out, nrhs);
    return cudaGetLastError();
}

template <class Ti, class To>
cudaError_t launch_scatter_cm(cudaStream_t st, int64_t count, const int64_t* idx, const Ti* in, int64_t N, To* out,
                              int nrhs)
{
    if (count <= 0) return cudaSuccess;
    count_launches(1);
    scatter_cm_kernel<Ti, To><<<nblk(count * nrhs), 256, 0, st>>>(count, idx, in, N, out, nrhs);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_axpby(cudaStream_t st, int64_t n, T a, const T* x, T b, T* y)
{
    if (n <= 0) return cudaSuccess;
    count_launches(1);
    axpby_kernel<T><<<nblk(n), 256, 0, st>>>(n, a, x, b, y);
    return cudaGetLastError();
}

// y[c N + i] = s[i]^pw x[c N + i] (pw = +1 or -1), real s, T real or complex
template <class T>
__global__ void scale_cm_kernel(int64_t N, int nrhs, const double* __restrict__ sc, int pw, const T* __restrict__ x,
                                T* __restrict__ y)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * nrhs) return;
    const int64_t i = e % N;
    const double f = pw > 0 ? sc[i] : 1.0 / sc[i];
    y[e] = rscale<T>(f, x[e]);
}

template <class T>
cudaError_t launch_scale_cm(cudaStream_t st, int64_t N, int nrhs, const double* sc, int pw, const T* x, T* y)
{
    if (N <= 0 || nrhs <= 0) return cudaSuccess;
    count_launches(1);
    scale_cm_kernel<T><<<nblk(N * nrhs), 256, 0, st>>>(N, nrhs, sc, pw, x, y);
    return cudaGetLastError();
}
template cudaError_t launch_scale_cm<cplx<double>>(cudaStream_t, int64_t, int, const double*, int, const cplx<double>*,
                                                   cplx<double>*);

#define RS_INST_LINALG(T)                                                                                             \
    template int gj_max_ctas<T>(int, int);                                                                          \
    template cudaError_t launch_gj_inverse<T>(cudaStream_t, int, int, const int32_t*, const int64_t*, T*, int32_t*, \
                                              const int64_t*, int*, unsigned int*, int*, long long, int);           \
    template cudaError_t launch_gemm<T>(cudaStream_t, const GemmProb*, int, int64_t, const T*, const T*, T*,        \
                                        const T*);                                                                  \
    template cudaError_t launch_matvec<T>(cudaStream_t, const MatvecProb*, const int64_t*, int, int64_t, const T*,  \
                                          const T*, T*, int, int);                                                  \
    template cudaError_t launch_gather_rows<T>(cudaStream_t, int64_t, const int64_t*, const T*, T*, int);           \
    template cudaError_t launch_scatter_rows<T>(cudaStream_t, int64_t, const int64_t*, const T*, T*, int);          \
    template cudaError_t launch_gather_cm<typename sc_traits<T>::io, T>(cudaStream_t, int64_t, const int64_t*,      \
                                                                      const typename sc_traits<T>::io*, int64_t,  \
                                                                      T*, int);                                   \
    template cudaError_t launch_scatter_cm<T, typename sc_traits<T>::io>(cudaStream_t, int64_t, const int64_t*,     \
                                                                       const T*, int64_t,                         \
                                                                       typename sc_traits<T>::io*, int);          \
    template cudaError_t launch_axpby<T>(cudaStream_t, int64_t, T, const T*, T, T*);
RS_INST_LINALG(double)
RS_INST_LINALG(float)
RS_INST_LINALG(cplx<double>)
RS_INST_LINALG(cplx<float>)

}  // namespace rs
