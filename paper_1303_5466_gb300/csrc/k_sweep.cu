// k_sweep.cu -- in-place inverse of symmetric positive definite matrices (F_i, E_i and the
// root of a real symmetric kernel) by the symmetric sweep, lower triangle only.
//
// The sweep of a symmetric S on an index block K (D = S_KK) is
//     S_KK <- -D^{-1},  S_OK <- S_OK D^{-1},  S_KO <- D^{-1} S_KO,  S_OO <- S_OO - S_OK D^{-1} S_KO.
// It keeps S symmetric, sweeps of disjoint blocks compose, and sweeping every index of an SPD
// matrix leaves -S^{-1}; the pivots are the diagonals of successive Schur complements, so an
// SPD matrix needs no pivoting.  Updating only the lower triangle costs m^3 flops, half of
// Gauss-Jordan with partial pivoting.
#include <float.h>

#include "k_common.cuh"

namespace rs {

// Owner CTA of panel p in a group of G: panels are dealt back and forth (0, 1, .., G-1,
// G-1, .., 1, 0, 0, 1, ..), so every CTA holds panels from both ends of the matrix and the
// lower-triangle work stays even across the group.
__device__ __forceinline__ int sweep_owner(int p, int G)
{
    const int c = p % (2 * G);
    return c < G ? c : 2 * G - 1 - c;
}

// Row i of a panel buffer: NB values, 16-byte aligned (NB * sizeof(T) is a multiple of 16).
template <int NB, class T>
__device__ __forceinline__ void load_row(const T* p, T (&v)[NB])
{
    if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int t = 0; t < NB; t += 2) {
            const double2 q = __ldcg((const double2*)(p + t));
            v[t] = q.x;
            v[t + 1] = q.y;
        }
    } else {
#pragma unroll
        for (int t = 0; t < NB; t += 4) {
            const float4 q = __ldcg((const float4*)(p + t));
            v[t] = q.x;
            v[t + 1] = q.y;
            v[t + 2] = q.z;
            v[t + 3] = q.w;
        }
    }
}

// Panel buffer rows i >= k0 for the panel K = [k0, k0 + kw): row i holds S[i, K], the
// rows inside K the full symmetric diagonal block (from its lower triangle).
template <int NT, int NB, class T>
__device__ __forceinline__ void write_panel_rows(const T* __restrict__ A, int m, int k0, int kw, T* __restrict__ pb)
{
    const int rows = m - k0;
    for (int e = threadIdx.x; e < rows * NB; e += NT) {
        const int t = e / rows, ii = e - t * rows;       // consecutive threads: consecutive rows
        const int i = k0 + ii;
        T v = T(0);
        if (t < kw) {
            if (ii >= kw) v = ldcg_(A + (int64_t)(k0 + t) * m + i);
            else v = (ii >= t) ? ldcg_(A + (int64_t)(k0 + t) * m + i) : ldcg_(A + (int64_t)i * m + k0 + t);
        }
        pb[(int64_t)i * NB + t] = v;
    }
}

// G CTAs per matrix (cooperative when G > 1); panel q (columns [q NB, q NB + NB)) belongs to
// CTA sweep_owner(q, G).  Every CTA reads panel values only from the double buffer Pb (2 x m x
// NB per matrix; buffer q & 1 holds S[:, K_q] before step q), so no CTA reads another CTA's
// columns.  The rows of a panel's own columns are rewritten by the whole group (step 3), so
// every load of the matrix or of Pb bypasses L1 (ld.cg).  Step q:
//   1. one group barrier; every CTA sweeps the NB x NB block D (FP64) into D^{-1}; a pivot not
//      above 1e3 unit roundoff times the largest earlier pivot (a matrix that is not SPD to
//      working accuracy) makes every CTA of the group return, with DEV_NOT_SPD in *status;
//   2. each CTA updates the lower triangle of its own columns j outside K, CB at a time:
//      c_j = D^{-1} S[K, j]; S[i, j] -= S[i, K] c_j (rows i >= j outside K); rows K of
//      columns left of K become c_j; then it copies rows K_{q+1} of its columns left of
//      K_{q+1} into the other buffer;
//   3. the rows of panel K below K are split over the group: S[i, K] <- S[i, K] D^{-1} (the
//      ones inside K_{q+1} also go to the other buffer), and the owner writes S_KK = -D^{-1};
//   4. the owner of panel q + 1 copies its panel's rows into the other buffer.
// The result is -S^{-1} in the lower triangle; sweep_finish_kernel negates and mirrors it.
template <int NT, int NB, class T>
__global__ void __launch_bounds__(NT) sweep_kernel(int G0, const int32_t* __restrict__ cta_off,
        const int32_t* __restrict__ msz,
        const int64_t* __restrict__ off, T* __restrict__ Aall, T* __restrict__ Pball,
        const int64_t* __restrict__ pb_off, unsigned int* __restrict__ bar, int* __restrict__ status, long long spin)
{
    constexpr int CB = 32;                 // own columns updated per chunk
    constexpr int NE = (NB * NB + 31) / 32;
    __shared__ double s_M[NB][NB + 1];     // D, swept in place
    __shared__ double s_Di[NB][NB];        // D^{-1}
    __shared__ T s_c[NB][CB];              // -c_j of the chunk's columns
    __shared__ int s_col[CB];
    __shared__ int s_fail;

    // matrix and rank in its group: G0 CTAs per matrix, or (cta_off given) G0 matrices, matrix b
    // owning CTAs cta_off[b] .. cta_off[b+1]
    int b, gi, G;
    if (cta_off) {
        int lo = 0, hi = G0 - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (cta_off[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
        }
        b = lo;
        gi = (int)blockIdx.x - cta_off[b];
        G = cta_off[b + 1] - cta_off[b];
    } else {
        G = G0;
        b = blockIdx.x / G;
        gi = blockIdx.x - b * G;
    }
    const int m = msz[b];
    if (m <= 0) return;                    // the whole group returns
    T* __restrict__ A = Aall + off[b];
    T* __restrict__ Pb = Pball + pb_off[b];
    const int npan = (m + NB - 1) / NB;
    const int tid = threadIdx.x;
    double maxpiv = 0.0;                   // warp 0: largest pivot so far (same in every CTA)

    if (gi == sweep_owner(0, G)) write_panel_rows<NT, NB>(A, m, 0, min(NB, m), Pb);
    for (int q = 0; q < npan; ++q) {
        const int k0 = q * NB, kw = min(NB, m - k0);
        const int k0n = k0 + NB, kwn = min(NB, m - k0n);     // next panel (kwn <= 0: none)
        const T* pb = Pb + (int64_t)(q & 1) * m * NB;
        T* pbn = Pb + (int64_t)((q + 1) & 1) * m * NB;
        if (G > 1) {
            if (!group_sync(bar + b, (unsigned)(q + 1) * (unsigned)G, status, spin)) return;
        } else {
            __syncthreads();
        }
        // 1. D^{-1} by the sweep of D (warp 0, FP64)
        if (tid < 32) {
            for (int e = tid; e < NB * NB; e += 32) {
                const int r = e / NB, c = e - (e / NB) * NB;
                s_M[r][c] = (r < kw && c < kw) ? (double)ldcg_(pb + (int64_t)(k0 + r) * NB + c) : 0.0;
            }
            __syncwarp();
            int fail = 0;
            for (int t = 0; t < kw; ++t) {
                const double p = s_M[t][t];
                if (!(p > 1e3 * 0.5 * DBL_EPSILON * maxpiv) || !isfinite(p)) fail = 1;
                maxpiv = fmax(maxpiv, p);
                const double pinv = 1.0 / p;
                double nv[NE];
#pragma unroll
                for (int u = 0; u < NE; ++u) {
                    const int e = tid + 32 * u;
                    nv[u] = 0.0;
                    if (e < NB * NB) {
                        const int r = e / NB, c = e - (e / NB) * NB;
                        if (r == t && c == t) nv[u] = -pinv;
                        else if (r == t) nv[u] = s_M[t][c] * pinv;
                        else if (c == t) nv[u] = s_M[r][t] * pinv;
                        else nv[u] = fma(-s_M[r][t] * pinv, s_M[t][c], s_M[r][c]);
                    }
                }
                __syncwarp();
#pragma unroll
                for (int u = 0; u < NE; ++u) {
                    const int e = tid + 32 * u;
                    if (e < NB * NB) s_M[e / NB][e - (e / NB) * NB] = nv[u];
                }
                __syncwarp();
            }
            for (int e = tid; e < NB * NB; e += 32) {
                const int r = e / NB, c = e - (e / NB) * NB;
                s_Di[r][c] = (r < kw && c < kw) ? -s_M[r][c] : 0.0;
            }
            if (tid == 0) s_fail = fail;
        }
        __syncthreads();
        if (s_fail) {
            if (tid == 0 && gi == 0) atomicOr(status, DEV_NOT_SPD);
            return;
        }
        // 2. own columns outside K
        int s = 0, jin = 0;
        while (true) {
            int nc = 0;
            while (nc < CB) {
                const int p = (s >> 1) * 2 * G + ((s & 1) ? 2 * G - 1 - gi : gi);
                if (p >= npan) break;
                if (p == q) { ++s; jin = 0; continue; }
                const int w = min(NB, m - p * NB);
                if (tid == 0) s_col[nc] = p * NB + jin;
                ++nc;
                if (++jin == w) { ++s; jin = 0; }
            }
            if (nc == 0) break;
            __syncthreads();
            for (int e = tid; e < nc * NB; e += NT) {
                const int jj = e / NB, t = e - (e / NB) * NB;
                const int j = s_col[jj];
                double c = 0.0;
                if (t < kw) {
                    T a[NB];
                    load_row<NB>(pb + (int64_t)j * NB, a);
#pragma unroll
                    for (int u = 0; u < NB; ++u) c = fma(s_Di[t][u], (double)a[u], c);
                    if (j < k0) A[(int64_t)j * m + k0 + t] = (T)c;
                }
                s_c[t][jj] = (T)(-c);
            }
            __syncthreads();
            for (int i = s_col[0] + tid; i < m; i += NT) {
                if (i >= k0 && i < k0 + kw) continue;
                T P[NB];
                load_row<NB>(pb + (int64_t)i * NB, P);
                // the chunk's columns with j <= i (lower triangle): a prefix, the columns ascend
                int nv = 0;
                for (int step = CB / 2; step > 0; step >>= 1)
                    if (nv + step <= nc && s_col[nv + step - 1] <= i) nv += step;
                if (nv < nc && s_col[nv] <= i) ++nv;
                int jj = 0;
                for (; jj + 3 < nv; jj += 4) {           // four independent FMA chains
                    T* c0 = A + (int64_t)s_col[jj] * m + i;
                    T* c1 = A + (int64_t)s_col[jj + 1] * m + i;
                    T* c2 = A + (int64_t)s_col[jj + 2] * m + i;
                    T* c3 = A + (int64_t)s_col[jj + 3] * m + i;
                    T v0 = ldcg_(c0), v1 = ldcg_(c1), v2 = ldcg_(c2), v3 = ldcg_(c3);
#pragma unroll
                    for (int t = 0; t < NB; ++t) {
                        v0 = fma_(P[t], s_c[t][jj], v0);
                        v1 = fma_(P[t], s_c[t][jj + 1], v1);
                        v2 = fma_(P[t], s_c[t][jj + 2], v2);
                        v3 = fma_(P[t], s_c[t][jj + 3], v3);
                    }
                    *c0 = v0;
                    *c1 = v1;
                    *c2 = v2;
                    *c3 = v3;
                }
                for (; jj < nv; ++jj) {
                    T* cp = A + (int64_t)s_col[jj] * m + i;
                    T v = ldcg_(cp);
#pragma unroll
                    for (int t = 0; t < NB; ++t) v = fma_(P[t], s_c[t][jj], v);
                    *cp = v;
                }
            }
            __syncthreads();
            if (kwn > 0) {
                for (int e = tid; e < nc * NB; e += NT) {
                    const int jj = e / NB, t = e - (e / NB) * NB;
                    const int j = s_col[jj];
                    if (j < k0n) pbn[(int64_t)j * NB + t] = (t < kwn) ? ldcg_(A + (int64_t)j * m + k0n + t) : T(0);
                }
            }
            __syncthreads();
        }
        // 3. panel K: rows below K shared by the group, the diagonal block by its owner
        for (int i = k0 + kw + gi * NT + tid; i < m; i += G * NT) {
            T P[NB];
            load_row<NB>(pb + (int64_t)i * NB, P);
#pragma unroll
            for (int t = 0; t < NB; ++t) {
                if (t >= kw) break;
                double c = 0.0;
#pragma unroll
                for (int u = 0; u < NB; ++u) c = fma(s_Di[t][u], (double)P[u], c);
                A[(int64_t)(k0 + t) * m + i] = (T)c;
                if (kwn > 0 && i < k0n + kwn) pbn[(int64_t)(k0 + t) * NB + (i - k0n)] = (T)c;
            }
        }
        if (gi == sweep_owner(q, G)) {
            for (int e = tid; e < kw * kw; e += NT) {
                const int r = e / kw, c = e - (e / kw) * kw;
                if (r >= c) A[(int64_t)(k0 + c) * m + k0 + r] = (T)(-s_Di[r][c]);
            }
        }
        // 4. the next panel's rows
        if (kwn > 0 && gi == sweep_owner(q + 1, G)) write_panel_rows<NT, NB>(A, m, k0n, kwn, pbn);
    }
}

// A <- -S with S's lower triangle mirrored into the upper: one 32 x 32 tile of the lower
// triangle per CTA (tile t of matrix blockIdx.y, t = I(I+1)/2 + J, I >= J).
template <class T>
__global__ void __launch_bounds__(256) sweep_finish_kernel(const int32_t* __restrict__ msz,
        const int64_t* __restrict__ off, T* __restrict__ Aall)
{
    __shared__ T tile[32][33];
    const int b = blockIdx.y;
    const int m = msz[b];
    const int nt = (m + 31) / 32;
    const int64_t t = blockIdx.x;
    if (t >= (int64_t)nt * (nt + 1) / 2) return;
    int I = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((int64_t)(I + 1) * (I + 2) / 2 <= t) ++I;
    while ((int64_t)I * (I + 1) / 2 > t) --I;
    const int J = (int)(t - (int64_t)I * (I + 1) / 2);
    T* __restrict__ A = Aall + off[b];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int c = ty; c < 32; c += 8) {
        const int i = I * 32 + tx, j = J * 32 + c;
        if (i < m && j < m && (I > J || tx >= c)) tile[tx][c] = A[(int64_t)j * m + i];
    }
    __syncthreads();
    for (int c = ty; c < 32; c += 8) {
        const int i = I * 32 + tx, j = J * 32 + c;
        if (i < m && j < m) A[(int64_t)j * m + i] = -((I > J || tx >= c) ? tile[tx][c] : tile[c][tx]);
    }
    if (I > J) {
        for (int c = ty; c < 32; c += 8) {
            const int i = J * 32 + tx, j = I * 32 + c;
            if (i < m && j < m) A[(int64_t)j * m + i] = -tile[c][tx];
        }
    }
}

constexpr int SW_NT = 256, SW_NB = 8;

int sweep_panel_width() { return SW_NB; }

// The kernel for panel width nbw (8 or 16: twice the FMAs per element loaded, half the steps).
template <class T>
static const void* sweep_fn(int nbw)
{
    return nbw == 16 ? (const void*)sweep_kernel<SW_NT, 16, T> : (const void*)sweep_kernel<SW_NT, SW_NB, T>;
}

template <class T>
int sweep_max_ctas(int nbw)
{
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_fn<T>(nbw), SW_NT, 0) != cudaSuccess)
        return 0;
    return per_sm * sms;
}

template <class T>
cudaError_t launch_sweep_inverse(cudaStream_t st, int nb, int G, const int32_t* cta_off, int ctas, const int32_t* m,
                                 const int64_t* off, T* A, T* Pb, const int64_t* pb_off, unsigned int* bar,
                                 int* status, long long spin_limit, int max_m, int nbw)
{
    if (nb <= 0 || max_m <= 0) return cudaSuccess;
    if (nbw != SW_NB && nbw != 16) return cudaErrorInvalidValue;
    count_launches(1);
    if (!cta_off && G == 1) {
        if (nbw == 16)
            sweep_kernel<SW_NT, 16, T><<<nb, SW_NT, 0, st>>>(1, nullptr, m, off, A, Pb, pb_off, bar, status, spin_limit);
        else
            sweep_kernel<SW_NT, SW_NB, T><<<nb, SW_NT, 0, st>>>(1, nullptr, m, off, A, Pb, pb_off, bar, status,
                                                                spin_limit);
    } else {
        int g0 = cta_off ? nb : G;
        void* args[] = {(void*)&g0, (void*)&cta_off, (void*)&m, (void*)&off, (void*)&A, (void*)&Pb, (void*)&pb_off,
                        (void*)&bar, (void*)&status, (void*)&spin_limit};
        cudaError_t e = cudaLaunchCooperativeKernel(sweep_fn<T>(nbw), dim3((unsigned)(cta_off ? ctas : nb * G)),
                                                    dim3(SW_NT), args, 0, st);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t nt = (max_m + 31) / 32;
    count_launches(1);
    sweep_finish_kernel<T><<<dim3((unsigned)(nt * (nt + 1) / 2), (unsigned)nb), 256, 0, st>>>(m, off, A);
    return cudaGetLastError();
}

// The negation and mirroring of the sweep's result alone (for the blocked sweep of k_sweep_bl.cu).
template <class T>
cudaError_t launch_sweep_finish(cudaStream_t st, int nb, const int32_t* m, const int64_t* off, T* A, int max_m)
{
    if (nb <= 0 || max_m <= 0) return cudaSuccess;
    const int64_t nt = (max_m + 31) / 32;
    count_launches(1);
    sweep_finish_kernel<T><<<dim3((unsigned)(nt * (nt + 1) / 2), (unsigned)nb), 256, 0, st>>>(m, off, A);
    return cudaGetLastError();
}

#define RS_INST_SWEEP(T)                                                                                              \
    template cudaError_t launch_sweep_finish<T>(cudaStream_t, int, const int32_t*, const int64_t*, T*, int);      \
    template int sweep_max_ctas<T>(int);                                                                            \
    template cudaError_t launch_sweep_inverse<T>(cudaStream_t, int, int, const int32_t*, int, const int32_t*,       \
                                                 const int64_t*, T*, T*, const int64_t*, unsigned int*, int*,       \
                                                 long long, int, int);
RS_INST_SWEEP(double)
RS_INST_SWEEP(float)

}  // namespace rs
