// k_cpqr_bl.cu -- column-pivoted Householder QR of Y (Sec. 2.1, Eq. 2.1) with the trailing
// updates deferred over panels of NB steps (variant 7: NB = 16; variant 8: NB = 8).
//
// Same decomposition, pivot rule and rank rule as cpqr_kernel; only the order in which the
// reflectors reach the open columns differs.  Within a panel that started at step s0, after
// the reflectors H_i = I - tau_i v_i v_i^T of steps s0 .. s-1 the matrix is A - V F^T, where A is
// the matrix at the panel start (what Y still holds for the open columns), V = [v_s0 .. v_s-1]
// and F(j, i) = tau_i (v_i^T A_j - F(j, 0:i) V(:, 0:i)^T v_i).  Each step:
//   1. (group barrier) the pivot p: the largest of the keys the CTAs wrote at the end of the
//      previous step, as in cpqr_kernel;
//   2. every CTA corrects its slice of rows s0 .. r-1 of column p in place, A_p - V F(p, :)^T,
//      and writes the slice's partial |c|^2 (rows >= s) and V^T c;
//   3. (group barrier) every CTA adds the G partials in one fixed order -- the same alpha, the
//      same rank test and the same reflector in every CTA -- reads the corrected column and
//      forms v_s and w = V^T v_s = V^T c - beta V(s, :);
//   4. every CTA takes, for its share of the open columns, the dot product v_s^T A_j (4 to 32
//      lanes per column, by the size of the share), F(j, k) = tau (v_s^T A_j - F(j, 0:k) w),
//      row s of R, R(s, j) = A(s, j) - V(s, 0:k+1) F(j, 0:k+1)^T, the downdate of the squared
//      norm (recomputed from the corrected column once below 1e-4 of the value it was last
//      computed from) and the column's key for the next step.
// At the end of a panel, and when the rank test stops the factorization, one more group
// barrier, then every CTA applies A_j -= V F(j, :)^T to its share of the open columns (rows
// s0 .. r-1, or only the rows of R at the stop).  An open column is thus read once per step and
// read and written once per panel (cpqr_kernel: read twice and written once per step), and the
// update FMAs need no cross-lane sums.  Outputs as cpqr_kernel: kout, piv, diag, and rows
// 0..k-1 of every column of Y hold R.  Real scalars only (double, float).
#include <algorithm>
#include <type_traits>

#include "k_common.cuh"

namespace rs {

namespace {

constexpr int BL_NT = 256;
constexpr int BL_U = 8;          // rows per lane in flight in the dot products
constexpr int BL_PC = 4;         // columns per warp in the panel update

template <class T>
size_t bl_shm(int max_r, int max_m)
{
    return sizeof(int) * (size_t)(2 * max_m + 2) + sizeof(T) * (size_t)max_r + 64;
}

template <int NT, int NB, class T>
__global__ void __launch_bounds__(NT, 4) cpqr_bl_kernel(int G0, const int32_t* __restrict__ cta_off,
        const int64_t* __restrict__ act_off, const int32_t* __restrict__ nnear, int P,
        const int64_t* __restrict__ y_off, T* __restrict__ Yall, double eps, int32_t* __restrict__ kout,
        int32_t* __restrict__ piv, T* __restrict__ diag, unsigned int* __restrict__ bar,
        unsigned long long* __restrict__ keys, int* __restrict__ status, long long spin,
        double* __restrict__ nrm_all, double* __restrict__ ref_all, T* __restrict__ Vall, int vld,
        T* __restrict__ Fall, double* __restrict__ part)
{
    static_assert(!is_cplx<T>::value, "real scalars only");
    extern __shared__ double smem[];
    __shared__ T Vd[NB][NB];         // Vd[a][i] = V(s0 + a, i)
    __shared__ T wsh[NB];            // w = V^T v_s
    __shared__ T Fp[NB];             // F(p, 0:k) of the step's pivot
    __shared__ double red[NB + 1];   // |c|^2 and V^T c, summed over the group
    __shared__ unsigned long long kred[NT / 32];
    __shared__ unsigned long long s_key;

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
    const int64_t a0 = act_off[b];
    const int m = (int)(act_off[b + 1] - a0);
    const int r = nnear[b] + P;
    T* __restrict__ Y = Yall + y_off[b];
    T* __restrict__ V = Vall + (int64_t)b * NB * vld;       // V(row, i) at V[i vld + row]
    T* __restrict__ F = Fall + a0 * NB;                    // F(j, i) at F[j NB + i]
    const int64_t cta0 = cta_off ? (int64_t)cta_off[b] : (int64_t)b * G;
    double* __restrict__ pb = part + cta0 * (NB + 1);      // CTA q of the group at pb[q (NB + 1)]
    double* __restrict__ nrm = nrm_all + a0;
    double* __restrict__ ref = ref_all + a0;
    int* alist = (int*)smem;
    int* apos = alist + m;
    T* v = (T*)(alist + 2 * m);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int NW = NT / 32;
    unsigned long long* kb = keys + 2 * cta0;               // [2][G], by step parity
    unsigned int nsync = 0;
    auto gsync = [&]() -> bool {
        if (G > 1) return group_sync(bar + b, ++nsync * (unsigned)G, status, spin);
        __syncthreads();
        return true;
    };

    for (int j = threadIdx.x; j < m; j += NT) { alist[j] = j; apos[j] = j; }
    {
        const int lo = (int)(((int64_t)gi * m) / G), hi = (int)(((int64_t)(gi + 1) * m) / G);
        unsigned long long best = 0;
        for (int j = lo + warp; j < hi; j += NW) {
            const T* col = Y + (int64_t)j * r;
            double q = 0.0;
            for (int i = lane; i < r; i += 32) q += abs2d(col[i]);
            q = warp_sum(q);
            if (lane == 0) { nrm[j] = q; ref[j] = q; }
            const unsigned long long kq = pivot_key(q, j);
            best = kq > best ? kq : best;
        }
        best = block_max_u64<NT>(best, kred);
        if (threadIdx.x == 0) kb[gi] = best;
    }

    // A_j -= V(:, 0:kk) F(j, 0:kk)^T on this CTA's share of the open columns, rows s0 .. rend-1:
    // BL_PC columns per warp, the lanes over the rows, each V entry loaded once for the BL_PC;
    // with fewer column groups than warps, the rows are split into segments as well
    auto panel_update = [&](int nopen, int s0, int rend, int kk) {
        if (kk <= 0 || rend <= s0) return;
        const int lo = (int)(((int64_t)gi * nopen) / G), hi = (int)(((int64_t)(gi + 1) * nopen) / G);
        const int ncg = (hi - lo + BL_PC - 1) / BL_PC;
        const int nseg = max(1, min(NW / max(ncg, 1), (rend - s0 + 63) / 64));
        const int seg_len = ((rend - s0 + nseg - 1) / nseg + 31) & ~31;
        T* Fs = v + warp * BL_PC * NB;   // the warp's rows of F (v is free here)
        for (int item = warp; item < ncg * nseg; item += NW) {
            const int cg = item / nseg, sg = item - cg * nseg;
            const int t0 = lo + BL_PC * cg;
            const int nc = min(BL_PC, hi - t0);
            __syncwarp();
            for (int e = lane; e < BL_PC * NB; e += 32) {
                const int c = e / NB, q = e - c * NB;
                Fs[e] = (c < nc && q < kk) ? ldcg_(F + (int64_t)alist[t0 + c] * NB + q) : T(0);
            }
            T* cp[BL_PC];
#pragma unroll
            for (int c = 0; c < BL_PC; ++c) cp[c] = Y + (int64_t)alist[t0 + (c < nc ? c : 0)] * r;
            __syncwarp();
            const int i1 = min(rend, s0 + (sg + 1) * seg_len);
            for (int i = s0 + sg * seg_len + lane; i < i1; i += 32) {
                T x[BL_PC];
#pragma unroll
                for (int c = 0; c < BL_PC; ++c)
                    if (c < nc) x[c] = ldcg_(cp[c] + i);
                for (int q = 0; q < kk; ++q) {
                    const T vq = ldcg_(V + (int64_t)q * vld + i);
#pragma unroll
                    for (int c = 0; c < BL_PC; ++c)
                        if (c < nc) x[c] = fma_(-vq, Fs[c * NB + q], x[c]);
                }
#pragma unroll
                for (int c = 0; c < BL_PC; ++c)
                    if (c < nc) cp[c][i] = x[c];
            }
        }
    };

    int nopen = m, k = 0, s0 = 0;
    const int kmax = min(r, m);
    double alpha0 = 0.0;
    bool stopped = false;
    for (int s = 0; s < kmax; ++s) {
        const int kp = s - s0;           // the step's index in its panel
        // 1. the group's pivot
        if (!gsync()) return;
        if (warp == 0) {
            unsigned long long t = 0;
            for (int q = lane; q < G; q += 32) {
                const unsigned long long u = G > 1 ? __ldcg(kb + (s & 1) * G + q) : kb[(s & 1) * G + q];
                t = u > t ? u : t;
            }
            t = warp_max_u64(t);
            if (lane == 0) s_key = t;
        }
        __syncthreads();
        const int p = (int)(KEY_MASK - (s_key & KEY_MASK));
        if (p < 0 || p >= m) {
            if (threadIdx.x == 0) atomicOr(status, DEV_BADSIZE);
            return;                      // every CTA of the group reads the same key
        }
        if (threadIdx.x < kp) Fp[threadIdx.x] = ldcg_(F + (int64_t)p * NB + threadIdx.x);
        if (threadIdx.x == 0) {
            const int t = apos[p], last = alist[nopen - 1];
            alist[t] = last;
            apos[last] = t;
        }
        --nopen;
        __syncthreads();
        // 2. this CTA's slice of column p, corrected in place; its partial sums
        const int R0 = s0 + (int)(((int64_t)gi * (r - s0)) / G);
        const int R1 = s0 + (int)(((int64_t)(gi + 1) * (r - s0)) / G);
        T* colp = Y + (int64_t)p * r;
        for (int i = R0 + threadIdx.x; i < R1; i += NT) {
            T c = ldcg_(colp + i);
            for (int q = 0; q < kp; ++q) c = fma_(-ldcg_(V + (int64_t)q * vld + i), Fp[q], c);
            if (kp > 0) colp[i] = c;
            v[i] = c;
        }
        __syncthreads();
        const int Rs = max(R0, s);
        for (int t = warp; t <= kp; t += NW) {
            double acc = 0.0;
            if (t == 0) {
                for (int i = Rs + lane; i < R1; i += 32) acc += abs2d(v[i]);
            } else {
                const T* Vq = V + (int64_t)(t - 1) * vld;
                T a = T(0);
                for (int i = Rs + lane; i < R1; i += 32) a = fma_(ldcg_(Vq + i), v[i], a);
                acc = (double)a;
            }
            acc = warp_sum(acc);
            if (lane == 0) pb[gi * (NB + 1) + t] = acc;
        }
        // 3. the partials of the group, added in one fixed order
        if (!gsync()) return;
        for (int t = warp; t <= kp; t += NW) {
            double acc = 0.0;
            for (int q = lane; q < G; q += 32) acc += __ldcg(pb + q * (NB + 1) + t);
            acc = warp_sum(acc);
            if (lane == 0) red[t] = acc;
        }
        __syncthreads();
        const double alpha = sqrt(red[0]);
        if (s == 0) alpha0 = alpha;
        if (!(alpha > eps * alpha0)) { stopped = true; break; }
        for (int i = s + threadIdx.x; i < r; i += NT) v[i] = ldcg_(colp + i);
        __syncthreads();
        const T x0 = v[s];
        const T beta = (T)(((double)x0 < 0.0) ? alpha : -alpha);
        const T tau = (T)(1.0 / (alpha * (alpha + absd(x0))));
        __syncthreads();
        if (threadIdx.x == 0) {
            v[s] = x0 - beta;
            if (gi == 0) { piv[a0 + s] = p; diag[a0 + s] = beta; }
        }
        __syncthreads();
        if (threadIdx.x < kp) wsh[threadIdx.x] = (T)red[1 + threadIdx.x] - beta * Vd[kp][threadIdx.x];
        if (threadIdx.x < NB) {
            const int row = s0 + threadIdx.x;
            Vd[threadIdx.x][kp] = (row >= s && row < r) ? v[row] : T(0);
        }
        for (int i = R0 + threadIdx.x; i < R1; i += NT) V[(int64_t)kp * vld + i] = i >= s ? v[i] : T(0);
        __syncthreads();
        // 4. this CTA's share of the open columns: L lanes per column, L the smallest of 4, 8,
        // 16, 32 that still gives every warp a column (more lanes per column cost one more
        // butterfly add, fewer leave warps idle and each lane with a longer serial row loop)
        const int lo = (int)(((int64_t)gi * nopen) / G), hi = (int)(((int64_t)(gi + 1) * nopen) / G);
        const T vs = v[s];
        unsigned long long wbest = 0;
        auto gemv = [&](auto Lc) {
            constexpr int L = decltype(Lc)::value, CPW = 32 / L;
            const int ngr = (hi - lo + CPW - 1) / CPW;
            const int cme = lane / L, tl = lane % L;
            for (int g = warp; g < ngr; g += NW) {
                const int tt = lo + CPW * g + cme;
                const bool act = tt < hi;
                const int j = alist[act ? tt : lo + CPW * g];
                const T* col = Y + (int64_t)j * r;
                T d0 = T(0), d1 = T(0);
                int i = s + tl;
                for (; i + L * (BL_U - 1) < r; i += L * BL_U) {
                    T x[BL_U];
#pragma unroll
                    for (int u = 0; u < BL_U; ++u) x[u] = ldcg_(col + i + L * u);
#pragma unroll
                    for (int u = 0; u < BL_U; u += 2) {
                        d0 = fma_(v[i + L * u], x[u], d0);
                        d1 = fma_(v[i + L * u + L], x[u + 1], d1);
                    }
                }
                for (; i < r; i += L) d0 = fma_(v[i], ldcg_(col + i), d0);
                T acc = d0 + d1, cr = T(0);
                const T* Fj = F + (int64_t)j * NB;
                for (int q = tl; q < kp; q += L) {
                    const T f = ldcg_(Fj + q);
                    acc = fma_(-f, wsh[q], acc);
                    cr = fma_(Vd[kp][q], f, cr);
                }
#pragma unroll
                for (int o = 1; o < L; o <<= 1) {
                    acc += shfl_xor_(acc, o);
                    cr += shfl_xor_(cr, o);
                }
                const T f = tau * acc;
                double nv = 0.0;
                bool need = false;
                if (tl == 0 && act) {
                    F[(int64_t)j * NB + kp] = f;
                    const T rsj = ldcg_(col + s) - cr - vs * f;
                    nv = ldcg_(nrm + j) - abs2d(rsj);
                    need = nv < 1e-4 * ldcg_(ref + j);
                }
                // norms that fell below 1e-4 of their reference: recomputed from the corrected
                // column (rows s+1 ..), the whole warp on each such column in turn
                unsigned rec = __ballot_sync(0xffffffffu, need);
                while (rec) {
                    const int src = __ffs(rec) - 1;
                    rec &= rec - 1;
                    const int jq = __shfl_sync(0xffffffffu, j, src);
                    const T fq = shfl_(f, src);
                    const T* cq = Y + (int64_t)jq * r;
                    const T* Fq = F + (int64_t)jq * NB;
                    double q2 = 0.0;
                    for (int i2 = s + 1 + lane; i2 < r; i2 += 32) {
                        T c = fma_(-v[i2], fq, ldcg_(cq + i2));
                        for (int q = 0; q < kp; ++q) c = fma_(-ldcg_(V + (int64_t)q * vld + i2), ldcg_(Fq + q), c);
                        q2 += abs2d(c);
                    }
                    q2 = warp_sum(q2);
                    if (lane == src) {
                        nv = q2;
                        ref[jq] = q2;
                    }
                }
                if (tl == 0 && act) {
                    nrm[j] = nv;
                    const unsigned long long kq = pivot_key(nv, j);
                    wbest = kq > wbest ? kq : wbest;
                }
            }
        };
        const int C = hi - lo;
        if (C >= 8 * NW) gemv(std::integral_constant<int, 4>{});
        else if (C >= 4 * NW) gemv(std::integral_constant<int, 8>{});
        else if (C >= 2 * NW) gemv(std::integral_constant<int, 16>{});
        else gemv(std::integral_constant<int, 32>{});
        wbest = block_max_u64<NT>(wbest, kred);
        if (threadIdx.x == 0) kb[((s + 1) & 1) * G + gi] = wbest;
        k = s + 1;
        // the end of a panel: the deferred updates
        if (kp + 1 == NB || s + 1 == kmax) {
            if (!gsync()) return;
            panel_update(nopen, s0, r, kp + 1);
            s0 = s + 1;
        }
    }
    if (stopped && k > s0) {
        // the rank test ended the panel early: only the rows of R (s0 .. k-1) are still owed
        if (!gsync()) return;
        panel_update(nopen, s0, k, k - s0);
    }
    if (gi == 0 && threadIdx.x == 0) kout[b] = k;
}

template <int NB, class T>
const void* bl_fn()
{
    return (const void*)cpqr_bl_kernel<BL_NT, NB, T>;
}

}  // namespace

template <class T>
bool cpqr_bl_fits(int max_r, int max_m)
{
    if constexpr (is_cplx<T>::value) {
        (void)max_r;
        (void)max_m;
        return false;
    } else {
        // the panel update borrows v for BL_PC rows of F per warp
        return bl_shm<T>(std::max(max_r, BL_PC * 16 * (BL_NT / 32)), max_m) <= 227 * 1024;
    }
}

template <class T>
int cpqr_bl_max_ctas(int max_r, int max_m, int nbp)
{
    if constexpr (is_cplx<T>::value) {
        (void)max_r;
        (void)max_m;
        (void)nbp;
        return 0;
    } else {
        if (!cpqr_bl_fits<T>(max_r, max_m)) return 0;
        const size_t shm = bl_shm<T>(std::max(max_r, BL_PC * nbp * (BL_NT / 32)), max_m);
        const void* fn = nbp == 16 ? bl_fn<16, T>() : bl_fn<8, T>();
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) != cudaSuccess) return 0;
        int per_sm = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, BL_NT, shm) != cudaSuccess) return 0;
        return per_sm * sms;
    }
}

template <class T>
size_t cpqr_bl_bytes(int nb, int max_r, int64_t sum_m, int ctas, int nbp)
{
    const size_t v = sizeof(T) * (size_t)nb * (size_t)nbp * (size_t)max_r;
    const size_t f = sizeof(T) * (size_t)(sum_m + 1) * (size_t)nbp;
    return ((v + f + 15) & ~(size_t)15) + sizeof(double) * (size_t)ctas * (size_t)(nbp + 1);
}

template <class T>
cudaError_t launch_cpqr_bl(cudaStream_t st, int nb, int G, const int32_t* cta_off, int ctas, int nbp,
                           const int64_t* act_off, const int32_t* nnear, int P, const int64_t* y_off, T* Y,
                           double eps, int32_t* kout, int32_t* piv, T* diag, unsigned int* bar,
                           unsigned long long* keys, int* status, long long spin_limit, int max_r, int max_m,
                           int64_t sum_m, double* nrm, double* ref, void* scratch)
{
    if (nb <= 0) return cudaSuccess;
    if constexpr (is_cplx<T>::value) {
        return cudaErrorInvalidValue;
    } else {
        if (!scratch || (nbp != 8 && nbp != 16) || !cpqr_bl_fits<T>(max_r, max_m)) return cudaErrorInvalidValue;
        const int vld = max_r;
        const size_t shm = bl_shm<T>(std::max(max_r, BL_PC * nbp * (BL_NT / 32)), max_m);
        T* Vall = (T*)scratch;
        T* Fall = Vall + (size_t)nb * (size_t)nbp * (size_t)max_r;
        const size_t vf = sizeof(T) * ((size_t)nb * (size_t)nbp * (size_t)max_r + (size_t)(sum_m + 1) * (size_t)nbp);
        double* part = (double*)((char*)scratch + ((vf + 15) & ~(size_t)15));
        const void* fn = nbp == 16 ? bl_fn<16, T>() : bl_fn<8, T>();
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        if (e != cudaSuccess) return e;
        int g0 = cta_off ? nb : G;
        void* args[] = {(void*)&g0, (void*)&cta_off, (void*)&act_off, (void*)&nnear, (void*)&P, (void*)&y_off,
                        (void*)&Y, (void*)&eps, (void*)&kout, (void*)&piv, (void*)&diag, (void*)&bar, (void*)&keys,
                        (void*)&status, (void*)&spin_limit, (void*)&nrm, (void*)&ref, (void*)&Vall, (void*)&vld,
                        (void*)&Fall, (void*)&part};
        const unsigned grid = (unsigned)(cta_off ? ctas : nb * G);
        count_launches(1);
        if (!cta_off && G == 1) return cudaLaunchKernel(fn, dim3(grid), dim3(BL_NT), args, shm, st);
        return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(BL_NT), args, shm, st);
    }
}

#define RS_INST_CPQR_BL(T)                                                                                           \
    template bool cpqr_bl_fits<T>(int, int);                                                                         \
    template int cpqr_bl_max_ctas<T>(int, int, int);                                                                 \
    template size_t cpqr_bl_bytes<T>(int, int, int64_t, int, int);                                                   \
    template cudaError_t launch_cpqr_bl<T>(cudaStream_t, int, int, const int32_t*, int, int, const int64_t*,        \
                                           const int32_t*, int, const int64_t*, T*, double, int32_t*, int32_t*, T*,  \
                                           unsigned int*, unsigned long long*, int*, long long, int, int, int64_t,  \
                                           double*, double*, void*);
RS_INST_CPQR_BL(double)
RS_INST_CPQR_BL(float)
RS_INST_CPQR_BL(cplx<double>)
RS_INST_CPQR_BL(cplx<float>)

}  // namespace rs
