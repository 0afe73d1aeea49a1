// k_factor.cu -- kernels of the ID ("tree build") phase and of F assembly.
//
//   assemble_Y : Y_i = [ K(near_i, I_i) ; K(proxy_i, I_i) ]  (Sec. 2.2, equivalent densities)
//   cpqr       : Householder QR with column pivoting of Y_i  (Sec. 2.1, Eq. 2.1)
//   id_T       : T_i = R11^{-1} R12                           (Eq. 2.1)
//   assemble_F : F_i = D_i (+ diag(E_c1, E_c2))                (Algorithm 1)
#include "k_entry.cuh"

namespace rs {

// ------------------------------------------------------------------ Y assembly
template <class T>
__global__ void __launch_bounds__(256) assemble_Y_kernel(const int32_t* __restrict__ act,
        const int64_t* __restrict__ act_off, const int32_t* __restrict__ near,
        const int64_t* __restrict__ near_off, const double* __restrict__ geo,
        const double* __restrict__ ucirc, int P, const int64_t* __restrict__ y_off,
        T* __restrict__ Y, KernelK K)
{
    const int b = blockIdx.y;
    const int64_t a0 = act_off[b];
    const int m = (int)(act_off[b + 1] - a0);
    const int64_t n0 = near_off[b];
    const int nn = (int)(near_off[b + 1] - n0);
    const int r = nn + P;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)r * m) return;
    const int j = (int)(e / r), i = (int)(e - (int64_t)j * r);
    const int g = act[a0 + j];
    T v;
    if (i < nn) {
        v = kentry<T>(K, near[n0 + i], g);
    } else {
        const int q = i - nn;
        const double cx = geo[3 * b], cy = geo[3 * b + 1], R = geo[3 * b + 2];
        v = kproxy<T>(K, cx + R * ucirc[q], cy + R * ucirc[P + q], g);
    }
    Y[y_off[b] + e] = v;
}

template <class T>
cudaError_t launch_assemble_Y(cudaStream_t st, int nb, const int32_t* act, const int64_t* act_off,
                              const int32_t* near, const int64_t* near_off, const double* geo,
                              const double* ucirc, int P, const int64_t* y_off, T* Y, KernelK K,
                              int max_entries)
{
    if (nb <= 0 || max_entries <= 0) return cudaSuccess;
    dim3 grid((unsigned)((max_entries + 255) / 256), (unsigned)nb);
    count_launches(1);
    assemble_Y_kernel<T><<<grid, 256, 0, st>>>(act, act_off, near, near_off, geo, ucirc, P, y_off, Y, K);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ column-pivoted QR
// One group of G CTAs per box (cooperative when G > 1); Y is column-major with ld = r.
// Columns never move: the pivot order is recorded in piv[], and R is read back from the
// physical columns (rows < k) with its diagonal in diag[].  The squared column norms live in
// global memory (nrm, ref: act_off-indexed), and every CTA keeps the same list of open
// (unselected) columns, updated identically from the same pivot each step; step s splits the
// list evenly over the group's CTAs, so the work stays balanced however the pivots fall.
// Each step:
//   1. the group's best pivot key (computed by every CTA for its share at the end of the
//      previous step) is read from `keys` after one group barrier and names the pivot p;
//   2. every CTA drops p from its list and builds the Householder vector of column p
//      (rows s..r-1) in shared memory;
//   3. every CTA applies the reflector to its share of the open columns (two per warp, four
//      rows in flight per lane), downdates their squared norms (recomputed from the data once
//      below 1e-4 of the value they were last computed from) and takes the best key of its
//      share for the next step.
// The rank test |R_ss| > eps |R_00| ends the loop in all CTAs at the same step (every CTA
// computes alpha from the same data in the same order).
template <int NT, int U, bool GL, class T, bool BT>
__device__ __forceinline__ void cpqr_body(int G0, const int32_t* __restrict__ cta_off,
        const int64_t* __restrict__ act_off,
        const int32_t* __restrict__ nnear, int P, const int64_t* __restrict__ y_off,
        T* __restrict__ Yall, double eps, int32_t* __restrict__ kout, int32_t* __restrict__ piv,
        T* __restrict__ diag, unsigned int* __restrict__ bar, unsigned long long* __restrict__ keys,
        int* __restrict__ status, long long spin, double* __restrict__ nrm_all, double* __restrict__ ref_all,
        int* __restrict__ gwork, int gstride)
{
    extern __shared__ double smem[];
    __shared__ double dred[NT / 32 + 1];
    __shared__ unsigned long long kred[NT / 32];
    __shared__ unsigned long long s_key;

    // box and rank in its group: G0 CTAs per box, or (cta_off given) G0 boxes, box b owning CTAs
    // cta_off[b] .. cta_off[b+1]
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
    double* __restrict__ nrm = nrm_all + a0;
    double* __restrict__ ref = ref_all + a0;
    // open-column list (m: same order in every CTA), positions in it (m), Householder vector (r):
    // all in shared memory, or (GL: boxes too large for that) the two lists in this CTA's slice of
    // global memory; the vector's address is formed from the shared base either way, so its
    // reads in the hot loops stay shared-memory loads
    int* alist = GL ? gwork + (int64_t)blockIdx.x * gstride : (int*)smem;
    int* apos = alist + m;
    T* v = (T*)((int*)smem + (GL ? 0 : 2 * m));    // (2m ints keep it 8-byte aligned)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int NW = NT / 32;
    unsigned long long* kb = keys + 2 * (cta_off ? (int64_t)cta_off[b] : (int64_t)b * G);   // [2][G], by parity

    for (int j = threadIdx.x; j < m; j += NT) { alist[j] = j; apos[j] = j; }
    {
        // initial norms of this CTA's share, and its best key for step 0
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
    int nopen = m;
    const int kmax = min(r, m);
    int k = 0;
    double alpha0 = 0.0;
    for (int s = 0; s < kmax; ++s) {
        // 1. the group's pivot
        if (G > 1) {
            if (!group_sync(bar + b, (unsigned)(s + 1) * (unsigned)G, status, spin)) return;
        } else {
            __syncthreads();
        }
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
        const unsigned long long best = s_key;
        const int p = (int)(KEY_MASK - (best & KEY_MASK));
        if (p < 0 || p >= m) { if (threadIdx.x == 0) atomicOr(status, DEV_BADSIZE); break; }
        // 2. drop p from the open list (every CTA the same way), Householder vector
        const T* colp = Y + (int64_t)p * r;
        double part = 0.0;
        for (int i = s + threadIdx.x; i < r; i += NT) {
            const T x = ldcg_(colp + i);
            v[i] = x;
            part += abs2d(x);
        }
        const double a2 = block_sum<NT>(part, dred);    // its barriers also order the loads above
        if (threadIdx.x == 0) {
            const int t = apos[p], last = alist[nopen - 1];
            alist[t] = last;
            apos[last] = t;
        }
        --nopen;
        const double alpha = sqrt(a2);
        if (s == 0) alpha0 = alpha;
        if (!(alpha > eps * alpha0)) break;
        using R = typename sc_traits<T>::real;
        const T x0 = v[s];
        const double ax0 = absd(x0);
        // beta = -(x0 / |x0|) alpha (the sign of x0 for real data), so that v_s = x0 - beta
        // does not cancel
        T beta;
        if constexpr (is_cplx<T>::value) beta = (ax0 > 0.0) ? rscale<T>(-alpha / ax0, x0) : T(R(-alpha));
        else beta = (T)(((double)x0 < 0.0) ? alpha : -alpha);
        const R tau = (R)(1.0 / (alpha * (alpha + ax0)));   // 2 / ||v||^2
        __syncthreads();
        if (threadIdx.x == 0) {
            v[s] = x0 - beta;
            if (gi == 0) { piv[a0 + s] = p; diag[a0 + s] = beta; }
        }
        __syncthreads();
        // 3. this CTA's share of the open columns.  Its warps take contiguous runs of equal
        // length (within one column), two columns at a time and a single column at the end
        // of an odd run, so a warp never waits for a neighbour by more than one column.
        const int lo = (int)(((int64_t)gi * nopen) / G), hi = (int)(((int64_t)(gi + 1) * nopen) / G);
        unsigned long long wbest = 0;
        const bool lo16 = lane < 16;       // paired bookkeeping: lanes 0-15 column j0, 16-31 j1
        auto columns = [&](auto two_c, int j0, int j1) {
            constexpr bool TWO = decltype(two_c)::value;
            T* col0 = Y + (int64_t)j0 * r;
            T* col1 = Y + (int64_t)j1 * r;
            T w0 = 0, w1 = 0, w0b = 0, w1b = 0;      // two accumulators per column: shorter FMA chains
            int i = s + lane;
            for (; i + 32 * (U - 1) < r; i += 32 * U) {
                T vv[U], xa[U], xb[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    vv[u] = conj_(v[i + 32 * u]);
                    xa[u] = ldcg_(col0 + i + 32 * u);
                    if constexpr (TWO) xb[u] = ldcg_(col1 + i + 32 * u);
                }
#pragma unroll
                for (int u = 0; u < U; u += 2) {
                    w0 = fma_(vv[u], xa[u], w0);
                    w0b = fma_(vv[u + 1], xa[u + 1], w0b);
                    if constexpr (TWO) {
                        w1 = fma_(vv[u], xb[u], w1);
                        w1b = fma_(vv[u + 1], xb[u + 1], w1b);
                    }
                }
            }
            for (; i < r; i += 32) {
                const T vv = conj_(v[i]);
                w0 = fma_(vv, ldcg_(col0 + i), w0);
                if constexpr (TWO) w1 = fma_(vv, ldcg_(col1 + i), w1);
            }
            w0 += w0b;
            T tw0, tw1 = 0;
            if constexpr (TWO) {
                w1 += w1b;
                // both sums in one butterfly: lanes 0-15 end with w0's, 16-31 with w1's
                T wp = (lo16 ? w0 : w1) + shfl_xor_(lo16 ? w1 : w0, 16);
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) wp += shfl_xor_(wp, o);
                const T twp = tau * wp;
                tw0 = shfl_(twp, 0);
                tw1 = shfl_(twp, 16);
            } else {
                tw0 = tau * warp_sum(w0);
            }
            T rs0 = 0, rs1 = 0;                // row s after the update (lane 0)
            i = s + lane;
            for (; i + 32 * (U - 1) < r; i += 32 * U) {
                T vv[U], xa[U], xb[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    vv[u] = v[i + 32 * u];
                    xa[u] = ldcg_(col0 + i + 32 * u);
                    if constexpr (TWO) xb[u] = ldcg_(col1 + i + 32 * u);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    xa[u] = fma_(-vv[u], tw0, xa[u]);
                    col0[i + 32 * u] = xa[u];
                    if constexpr (TWO) {
                        xb[u] = fma_(-vv[u], tw1, xb[u]);
                        col1[i + 32 * u] = xb[u];
                    }
                }
                if (i == s) {
                    rs0 = xa[0];
                    if constexpr (TWO) rs1 = xb[0];
                }
            }
            for (; i < r; i += 32) {
                const T vv = v[i];
                const T xa = fma_(-vv, tw0, ldcg_(col0 + i));
                col0[i] = xa;
                if (i == s) rs0 = xa;
                if constexpr (TWO) {
                    const T xb = fma_(-vv, tw1, ldcg_(col1 + i));
                    col1[i] = xb;
                    if (i == s) rs1 = xb;
                }
            }
            // downdated squared norms (R_sj is row s of column j): both columns in one
            // instruction when there are two
            const T r0 = shfl_(rs0, 0);
            const T r1 = TWO ? shfl_(rs1, 0) : r0;
            const int jj = (TWO && !lo16) ? j1 : j0;
            double nv = ldcg_(nrm + jj) - abs2d((TWO && !lo16) ? r1 : r0);
            const unsigned need = __ballot_sync(0xffffffffu, nv < 1e-4 * ldcg_(ref + jj));
            if (need & 0x00010001u) {
                __syncwarp();                  // the recomputation reads the warp's stores
                for (int c = 0; c < (TWO ? 2 : 1); ++c) {
                    if (!(need & (1u << (16 * c)))) continue;
                    const T* col = c == 0 ? col0 : col1;
                    double q = 0.0;
                    for (int i2 = s + 1 + lane; i2 < r; i2 += 32) q += abs2d(ldcg_(col + i2));
                    q = warp_sum(q);
                    if (!TWO || (lane >> 4) == c) nv = q;
                    if (lane == 16 * c) ref[jj] = q;
                }
            }
            if (lane == 0 || (TWO && lane == 16)) nrm[jj] = nv;
            const unsigned long long kq = pivot_key(nv, jj);
            wbest = kq > wbest ? kq : wbest;
        };
        // BT: eight columns per warp pass.  The lanes' partial dot products of the eight are
        // summed by recursive halving (lane l ends with column (l >> 2) & 7: 9 FP64 adds for
        // eight columns instead of 5 per pair), and the per-column bookkeeping (tau w, row s of
        // R, the norm downdate, the key) runs once per column on lanes 0, 4, .., 28, so the
        // FP64 pipe spends its time on the dot-product and update FMAs.
        auto group8 = [&](int t0, int ng) {
            T* cp[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) cp[c] = Y + (int64_t)alist[t0 + (c < ng ? c : 0)] * r;
            T acc[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = T(0);
            int i = s + lane;
            for (; i + 32 < r; i += 64) {
                const T va = conj_(v[i]), vb = conj_(v[i + 32]);
                T xa[8], xb[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    xa[c] = c < ng ? ldcg_(cp[c] + i) : T(0);
                    xb[c] = c < ng ? ldcg_(cp[c] + i + 32) : T(0);
                }
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[c] = fma_(vb, xb[c], fma_(va, xa[c], acc[c]));
            }
            if (i < r) {
                const T va = conj_(v[i]);
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    if (c < ng) acc[c] = fma_(va, ldcg_(cp[c] + i), acc[c]);
            }
            // recursive halving over lanes 16, 8, 4, then the last two levels
            const bool h4 = (lane >> 4) & 1, h3 = (lane >> 3) & 1, h2 = (lane >> 2) & 1;
            T q4[4], q2[2];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const T snd = h4 ? acc[q] : acc[4 + q];
                q4[q] = (h4 ? acc[4 + q] : acc[q]) + shfl_xor_(snd, 16);
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const T snd = h3 ? q4[q] : q4[2 + q];
                q2[q] = (h3 ? q4[2 + q] : q4[q]) + shfl_xor_(snd, 8);
            }
            T w = (h2 ? q2[1] : q2[0]) + shfl_xor_(h2 ? q2[0] : q2[1], 4);
            w += shfl_xor_(w, 2);
            w += shfl_xor_(w, 1);
            const int cme = (lane >> 2) & 7;
            const bool book = (lane & 3) == 0 && cme < ng;
            const T twm = tau * w;
            T tw[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) tw[c] = shfl_(twm, c << 2);
            // row s of R for this lane's column (the update below computes the same value)
            int jme = 0;
            double nv = 0.0;
            bool need = false;
            if (book) {
                jme = alist[t0 + cme];
                const T rsj = fma_(-v[s], twm, ldcg_(Y + (int64_t)jme * r + s));
                nv = ldcg_(nrm + jme) - abs2d(rsj);
                need = nv < 1e-4 * ldcg_(ref + jme);
            }
            // the update of the eight columns
            i = s + lane;
            for (; i + 32 < r; i += 64) {
                const T va = v[i], vb = v[i + 32];
                T xa[8], xb[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    xa[c] = c < ng ? ldcg_(cp[c] + i) : T(0);
                    xb[c] = c < ng ? ldcg_(cp[c] + i + 32) : T(0);
                }
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    if (c < ng) {
                        cp[c][i] = fma_(-va, tw[c], xa[c]);
                        cp[c][i + 32] = fma_(-vb, tw[c], xb[c]);
                    }
            }
            if (i < r) {
                const T va = v[i];
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    if (c < ng) cp[c][i] = fma_(-va, tw[c], ldcg_(cp[c] + i));
            }
            // norms that fell below 1e-4 of their reference: recomputed from the updated rows,
            // the whole warp on each such column in turn
            unsigned rec = __ballot_sync(0xffffffffu, need);
            if (rec) {
                __syncwarp();                  // the recomputation reads the warp's stores
                while (rec) {
                    const int src = __ffs(rec) - 1;
                    rec &= rec - 1;
                    const int jq = __shfl_sync(0xffffffffu, jme, src);
                    const T* col = Y + (int64_t)jq * r;
                    double q = 0.0;
                    for (int i2 = s + 1 + lane; i2 < r; i2 += 32) q += abs2d(ldcg_(col + i2));
                    q = warp_sum(q);
                    if (lane == src) {
                        nv = q;
                        ref[jq] = q;
                    }
                }
            }
            if (book) {
                nrm[jme] = nv;
                const unsigned long long kq = pivot_key(nv, jme);
                wbest = kq > wbest ? kq : wbest;
            }
        };
        {
            const int C = hi - lo;
            const int wlo = lo + (int)(((int64_t)warp * C) / NW), whi = lo + (int)(((int64_t)(warp + 1) * C) / NW);
            if constexpr (BT) {
                for (int t = wlo; t < whi; t += 8) group8(t, min(8, whi - t));
            } else {
                int t = wlo;
                for (; t + 1 < whi; t += 2) columns(std::true_type{}, alist[t], alist[t + 1]);
                if (t < whi) columns(std::false_type{}, alist[t], alist[t]);
            }
        }
        wbest = block_max_u64<NT>(wbest, kred);
        if (threadIdx.x == 0) kb[((s + 1) & 1) * G + gi] = wbest;
        k = s + 1;
    }
    if (gi == 0 && threadIdx.x == 0) kout[b] = k;
}

#define RS_CPQR_PARAMS                                                                                               \
    int G0, const int32_t *__restrict__ cta_off, const int64_t *__restrict__ act_off,                                \
        const int32_t *__restrict__ nnear, int P, const int64_t *__restrict__ y_off, T *__restrict__ Yall, double eps, \
        int32_t *__restrict__ kout, int32_t *__restrict__ piv, T *__restrict__ diag, unsigned int *__restrict__ bar, \
        unsigned long long *__restrict__ keys, int *__restrict__ status, long long spin,                            \
        double *__restrict__ nrm_all, double *__restrict__ ref_all, int *__restrict__ gwork, int gstride
#define RS_CPQR_PASS G0, cta_off, act_off, nnear, P, y_off, Yall, eps, kout, piv, diag, bar, keys, status, spin, \
                     nrm_all, ref_all, gwork, gstride

template <int NT, int U, bool GL, class T, bool BT = false>
__global__ void __launch_bounds__(NT) cpqr_kernel(RS_CPQR_PARAMS)
{
    cpqr_body<NT, U, GL, T, BT>(RS_CPQR_PASS);
}

// The same body with registers capped for five CTAs per SM (variant 6).
template <int NT, int U, bool GL, class T>
__global__ void __launch_bounds__(NT, 5) cpqr_occ_kernel(RS_CPQR_PARAMS)
{
    cpqr_body<NT, U, GL, T, false>(RS_CPQR_PASS);
}

template <class T>
static size_t cpqr_shm(int max_r, int max_m, bool global_lists)
{
    return (global_lists ? 0 : sizeof(int) * (size_t)(2 * max_m + 2)) + sizeof(T) * (size_t)max_r + 64;
}

// The open-column lists go to global memory when asked (variant 3) or when shared memory cannot
// hold them with the Householder vector.
template <class T>
static bool cpqr_global(int max_r, int max_m, int deep)
{
    return deep == 3 || cpqr_shm<T>(max_r, max_m, false) > 227 * 1024;
}

template <class T>
size_t cpqr_gwork_ints(int max_r, int max_m, int deep, int ctas)
{
    return cpqr_global<T>(max_r, max_m, deep) ? (size_t)ctas * (size_t)(2 * max_m + 2) : 0;
}

template <int U, bool GL, class T, bool BT, bool OCC = false>
static cudaError_t launch_cpqr_u(cudaStream_t st, int nb, int G, const int32_t* cta_off, int ctas,
                                 const int64_t* act_off, const int32_t* nnear, int P, const int64_t* y_off, T* Y,
                                 double eps, int32_t* kout, int32_t* piv, T* diag, unsigned int* bar,
                                 unsigned long long* keys, int* status, long long spin_limit, size_t shm, double* nrm,
                                 double* ref, int* gwork, int gstride)
{
    constexpr int NT = 256;
    auto fn = OCC ? cpqr_occ_kernel<NT, U, GL, T> : cpqr_kernel<NT, U, GL, T, BT>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e != cudaSuccess) return e;
    count_launches(1);
    if (!cta_off && G == 1) {
        fn<<<nb, NT, shm, st>>>(1, nullptr, act_off, nnear, P, y_off, Y, eps, kout, piv, diag, bar, keys, status,
                                spin_limit, nrm, ref, gwork, gstride);
        return cudaGetLastError();
    }
    int g0 = cta_off ? nb : G;
    void* args[] = {(void*)&g0, (void*)&cta_off, (void*)&act_off, (void*)&nnear, (void*)&P, (void*)&y_off, (void*)&Y,
                    (void*)&eps, (void*)&kout, (void*)&piv, (void*)&diag, (void*)&bar, (void*)&keys, (void*)&status,
                    (void*)&spin_limit, (void*)&nrm, (void*)&ref, (void*)&gwork, (void*)&gstride};
    return cudaLaunchCooperativeKernel((void*)fn, dim3((unsigned)(cta_off ? ctas : nb * G)), dim3(NT), args, shm, st);
}

// The kernel instance of a variant: deep 0 (U = 4), 1 (U = 8), 3 (global lists), 5 (eight
// columns per warp pass, U unused) and 6 (U = 2, registers capped for five CTAs per SM: more
// boxes in flight per SM to cover each one's per-step latency) of cpqr_kernel.
template <class T>
static const void* cpqr_fn(int deep, bool glob)
{
    constexpr int NT = 256;
    if (deep == 5) return glob ? (const void*)cpqr_kernel<NT, 4, true, T, true> : (const void*)cpqr_kernel<NT, 4, false, T, true>;
    if (deep == 6) return glob ? (const void*)cpqr_occ_kernel<NT, 2, true, T> : (const void*)cpqr_occ_kernel<NT, 2, false, T>;
    if (glob) return deep == 1 ? (const void*)cpqr_kernel<NT, 8, true, T> : (const void*)cpqr_kernel<NT, 4, true, T>;
    return deep == 1 ? (const void*)cpqr_kernel<NT, 8, false, T> : (const void*)cpqr_kernel<NT, 4, false, T>;
}

template <class T>
cudaError_t launch_cpqr(cudaStream_t st, int nb, int G, const int32_t* cta_off, int ctas, int deep,
                        const int64_t* act_off, const int32_t* nnear, int P, const int64_t* y_off, T* Y, double eps,
                        int32_t* kout, int32_t* piv, T* diag, unsigned int* bar, unsigned long long* keys,
                        int* status, long long spin_limit, int max_r, int max_m, double* nrm, double* ref, T* wv,
                        int* gwork)
{
    if (nb <= 0) return cudaSuccess;
    if (deep == 2) {
        if (!wv) return cudaErrorInvalidValue;
        return launch_cpqr_la<T>(st, nb, G, cta_off, ctas, act_off, nnear, P, y_off, Y, eps, kout, piv, diag, bar,
                                 keys, status, spin_limit, max_r, max_m, nrm, ref, wv);
    }
    const bool glob = cpqr_global<T>(max_r, max_m, deep);
    if (glob && !gwork) return cudaErrorInvalidValue;
    const size_t shm = cpqr_shm<T>(max_r, max_m, glob);
    if (shm > 227 * 1024) return cudaErrorInvalidValue;     // the Householder vector alone does not fit
    int* gw = glob ? gwork : nullptr;
    const int gstride = 2 * max_m + 2;
#define RS_CPQR_ARGS st, nb, G, cta_off, ctas, act_off, nnear, P, y_off, Y, eps, kout, piv, diag, bar, keys, status, \
                     spin_limit, shm, nrm, ref, gw, gstride
    if (deep == 5)
        return glob ? launch_cpqr_u<4, true, T, true>(RS_CPQR_ARGS) : launch_cpqr_u<4, false, T, true>(RS_CPQR_ARGS);
    if (deep == 6)
        return glob ? launch_cpqr_u<2, true, T, false, true>(RS_CPQR_ARGS) : launch_cpqr_u<2, false, T, false, true>(RS_CPQR_ARGS);
    if (glob)
        return deep == 1 ? launch_cpqr_u<8, true, T, false>(RS_CPQR_ARGS) : launch_cpqr_u<4, true, T, false>(RS_CPQR_ARGS);
    return deep == 1 ? launch_cpqr_u<8, false, T, false>(RS_CPQR_ARGS) : launch_cpqr_u<4, false, T, false>(RS_CPQR_ARGS);
#undef RS_CPQR_ARGS
}

template <class T>
int cpqr_max_ctas(int max_r, int max_m, int G, int deep)
{
    constexpr int NT = 256;
    (void)G;
    if (deep == 2) return cpqr_la_max_ctas<T>(max_r, max_m);
    if (deep == 7 || deep == 8) return cpqr_bl_max_ctas<T>(max_r, max_m, deep == 7 ? 16 : 8);
    const bool glob = cpqr_global<T>(max_r, max_m, deep);
    const size_t shm = cpqr_shm<T>(max_r, max_m, glob);
    if (shm > 227 * 1024) return 0;
    const void* fn = cpqr_fn<T>(deep, glob);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) != cudaSuccess) return 0;
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, shm) != cudaSuccess) return 0;
    return per_sm * sms;
}

// ------------------------------------------------------------------ T = R11^{-1} R12
// One CTA per (box, group of nc residual columns): back substitution over the columns of R11
// (a = k-1 .. 0).  The group's right-hand sides live in shared memory; the R11 column of the
// next step is fetched into a second shared buffer while the current step updates, so each
// step costs two CTA barriers and no dependent global load.
template <int NT, class T>
__global__ void __launch_bounds__(NT) id_T_kernel(const int64_t* __restrict__ act_off, const int32_t* __restrict__ kk,
        const int32_t* __restrict__ nnear, int P, const int64_t* __restrict__ y_off, const T* __restrict__ Yall,
        const int32_t* __restrict__ piv, const T* __restrict__ diag, const int32_t* __restrict__ skpos,
        const int32_t* __restrict__ rscol, const int64_t* __restrict__ t_off, T* __restrict__ Tout, int NC,
        int rglobal)
{
    extern __shared__ double ys_raw[];
    const int b = blockIdx.x;
    const int64_t a0 = act_off[b];
    const int m = (int)(act_off[b + 1] - a0);
    const int k = kk[b];
    const int nres = m - k;
    const int cb = blockIdx.y * NC;
    if (cb >= nres || k == 0) return;
    const int nc = min(NC, nres - cb);
    const int r = nnear[b] + P;
    const T* Y = Yall + y_off[b];
    T* Tb = Tout + t_off[b];
    T* ys = (T*)ys_raw;                 // nc x k right-hand sides, then solutions
    T* rc = ys + (size_t)NC * k;        // 2 x k: R11 columns of the current and next step (none
                                        // when rglobal: the columns are read from Y in place)
    __shared__ T tq[64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int NW = NT / 32;
    for (int q = warp; q < nc; q += NW) {
        const T* col = Y + (int64_t)rscol[a0 + cb + q] * r;
        for (int i = lane; i < k; i += 32) ys[(size_t)q * k + i] = col[i];
    }
    if (!rglobal) {
        const T* Ra = Y + (int64_t)piv[a0 + k - 1] * r;
        for (int i = threadIdx.x; i < k; i += NT) rc[(size_t)((k - 1) & 1) * k + i] = Ra[i];
    }
    __syncthreads();
    for (int a = k - 1; a >= 0; --a) {
        const T* cur = rglobal ? Y + (int64_t)piv[a0 + a] * r : rc + (size_t)(a & 1) * k;
        if (threadIdx.x < nc) {
            const T t = ys[(size_t)threadIdx.x * k + a] / diag[a0 + a];
            tq[threadIdx.x] = t;
            Tb[(int64_t)(cb + threadIdx.x) * k + skpos[a0 + a]] = t;
        }
        if (a > 0 && !rglobal) {
            T* nxt = rc + (size_t)((a - 1) & 1) * k;
            const T* Rn = Y + (int64_t)piv[a0 + a - 1] * r;
            for (int i = threadIdx.x; i < a - 1 + 1; i += NT) nxt[i] = Rn[i];
        }
        __syncthreads();
        // every thread takes rows i of all nc columns (no warp idles when nc < NW)
        for (int i = threadIdx.x; i < a; i += NT) {
            const T c = cur[i];
            for (int q = 0; q < nc; ++q) ys[(size_t)q * k + i] = fma_(-tq[q], c, ys[(size_t)q * k + i]);
        }
        __syncthreads();
    }
}

template <class T>
static int id_T_cols(int max_k)
{
    const size_t budget = 160 * 1024;
    const size_t per = sizeof(T) * (size_t)std::max(max_k, 1);
    int nc = (int)std::min<size_t>(32, budget / per > 2 ? budget / per - 2 : 1);
    return std::max(nc, 1);
}

template <class T>
cudaError_t launch_id_T(cudaStream_t st, int nb, const int64_t* act_off, const int32_t* kk, const int32_t* nnear,
                        int P, const int64_t* y_off, const T* Y, const int32_t* piv, const T* diag,
                        const int32_t* skpos, const int32_t* rscol, const int64_t* t_off, T* Tout, int max_cols,
                        int max_k)
{
    constexpr int NT = 256;
    if (nb <= 0 || max_cols <= 0 || max_k <= 0) return cudaSuccess;
    // columns per CTA: as many as shared memory allows, fewer when that leaves the launch short of
    // about four CTAs per SM (the top levels: few boxes, long back substitutions)
    int NC = id_T_cols<T>(max_k);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = 4 * (int64_t)std::max(sms, 1);
    const int64_t nc_fill = ((int64_t)nb * max_cols + want - 1) / want;
    NC = (int)std::max<int64_t>(1, std::min<int64_t>(NC, nc_fill));
    // a skeleton too large for the two R11 column buffers: the columns are read from Y in place
    int rglobal = 0;
    size_t shm = sizeof(T) * (size_t)(NC + 2) * (size_t)max_k;
    if (shm > 227 * 1024) {
        rglobal = 1;
        shm = sizeof(T) * (size_t)NC * (size_t)max_k;
    }
    if (shm > 227 * 1024) return cudaErrorInvalidValue;     // skeleton too large for one CTA's buffers
    cudaError_t e = cudaFuncSetAttribute(id_T_kernel<NT, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)nb, (unsigned)((max_cols + NC - 1) / NC));
    count_launches(1);
    id_T_kernel<NT, T><<<grid, NT, shm, st>>>(act_off, kk, nnear, P, y_off, Y, piv, diag, skpos, rscol, t_off, Tout,
                                              NC, rglobal);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ F assembly
template <class T>
__global__ void __launch_bounds__(256) assemble_F_kernel(int leaf, const int32_t* __restrict__ act,
        const int64_t* __restrict__ act_off, const int32_t* __restrict__ perm, const double* __restrict__ a,
        const int64_t* __restrict__ phi_off, T* __restrict__ Phi, const int32_t* __restrict__ child_k,
        const int64_t* __restrict__ child_e_off, const T* __restrict__ childE, KernelK K)
{
    const int b = blockIdx.y;
    const int64_t a0 = act_off[b];
    const int m = (int)(act_off[b + 1] - a0);
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * m) return;
    const int q = (int)(e / m), p = (int)(e - (int64_t)q * m);     // column-major (p row, q col)
    const int i = perm[a0 + p], j = perm[a0 + q];                  // natural positions
    const int gi = act[a0 + i], gj = act[a0 + j];
    T v;
    if (leaf) {
        v = (i == j) ? kdiag<T>(K, a, gi) : kentry<T>(K, gi, gj);
    } else {
        const int k1 = child_k[2 * b], k2 = child_k[2 * b + 1];
        if (i < k1 && j < k1) v = childE[child_e_off[2 * b] + (int64_t)j * k1 + i];
        else if (i >= k1 && j >= k1) v = childE[child_e_off[2 * b + 1] + (int64_t)(j - k1) * k2 + (i - k1)];
        else v = kentry<T>(K, gi, gj);
    }
    Phi[phi_off[b] + e] = v;
}

template <class T>
cudaError_t launch_assemble_F(cudaStream_t st, int nb, bool leaf, const int32_t* act, const int64_t* act_off,
                              const int32_t* perm, const double* a, const int64_t* phi_off, T* Phi,
                              const int32_t* child_k, const int64_t* child_e_off, const T* childE, KernelK K,
                              int max_m)
{
    if (nb <= 0 || max_m <= 0) return cudaSuccess;
    const int64_t ent = (int64_t)max_m * max_m;
    dim3 grid((unsigned)((ent + 255) / 256), (unsigned)nb);
    count_launches(1);
    assemble_F_kernel<T><<<grid, 256, 0, st>>>(leaf ? 1 : 0, act, act_off, perm, a, phi_off, Phi, child_k, child_e_off,
                                               childE, K);
    return cudaGetLastError();
}

#define RS_INST_FACTOR(T)                                                                                              \
    template cudaError_t launch_assemble_Y<T>(cudaStream_t, int, const int32_t*, const int64_t*, const int32_t*,     \
                                              const int64_t*, const double*, const double*, int, const int64_t*, T*, \
                                              KernelK, int);                                                        \
    template cudaError_t launch_cpqr<T>(cudaStream_t, int, int, const int32_t*, int, int, const int64_t*,            \
                                        const int32_t*, int, const int64_t*, T*, double, int32_t*, int32_t*, T*,    \
                                        unsigned int*, unsigned long long*, int*, long long, int, int, double*,     \
                                        double*, T*, int*);                                                         \
    template int cpqr_max_ctas<T>(int, int, int, int);                                                               \
    template size_t cpqr_gwork_ints<T>(int, int, int, int);                                                          \
    template cudaError_t launch_id_T<T>(cudaStream_t, int, const int64_t*, const int32_t*, const int32_t*, int,      \
                                        const int64_t*, const T*, const int32_t*, const T*, const int32_t*,         \
                                        const int32_t*, const int64_t*, T*, int, int);                              \
    template cudaError_t launch_assemble_F<T>(cudaStream_t, int, bool, const int32_t*, const int64_t*,              \
                                              const int32_t*, const double*, const int64_t*, T*, const int32_t*,     \
                                              const int64_t*, const T*, KernelK, int);
RS_INST_FACTOR(double)
RS_INST_FACTOR(float)
RS_INST_FACTOR(cplx<double>)
RS_INST_FACTOR(cplx<float>)

}  // namespace rs
