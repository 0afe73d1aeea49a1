// k_cpqr_la.cu -- column-pivoted QR of Y (Sec. 2.1, Eq. 2.1), look-ahead variant: each step
// reads and writes every open column once, where the plain variant (k_factor.cu) reads it
// twice (dot product, then update).  Same layout, outputs and group scheme as cpqr_kernel.
//
// With v_s the Householder vector of step s and w_j = v_s^H y_j in wv[j] (y_j: column j
// after the steps before s), pass s
//   - applies reflector s, y_j <- y_j - tau_s v_s w_j (rows >= s), and in the same sweep
//   - takes w'_j = v_{s+1}^H y_j (rows >= s+1), row s+1 of the column after reflector s+1,
//     R_{s+1,j} = y_j[s+1] - tau_{s+1} v_{s+1}[s+1] w'_j, and the downdated squared norm
//     |y_j|^2 - |R_{s+1,j}|^2 (recomputed from the data once below 1e-4 of the value it was
//     last computed from), whose largest key names the pivot of step s+2.
// Before pass s, after one group barrier, every CTA builds v_{s+1} from the pivot column
// p_{s+1} as pass s-1 left it, y_p - tau_s v_s wv[p] (rows >= s+1), and CTA 0 writes its row s
// (an entry of R); p_{s+1} then leaves the open list.  The rank test ends the loop in all CTAs
// at the same step; when it fails, one more barrier lets every CTA finish reading that column
// before the last pass updates it.
#include "k_common.cuh"

namespace rs {

template <int NT, class T>
__global__ void __launch_bounds__(NT) cpqr_la_kernel(int G0, const int32_t* __restrict__ cta_off,
        const int64_t* __restrict__ act_off, const int32_t* __restrict__ nnear, int P,
        const int64_t* __restrict__ y_off, T* __restrict__ Yall, double eps, int32_t* __restrict__ kout,
        int32_t* __restrict__ piv, T* __restrict__ diag, unsigned int* __restrict__ bar,
        unsigned long long* __restrict__ keys, int* __restrict__ status, long long spin,
        double* __restrict__ nrm_all, double* __restrict__ ref_all, T* __restrict__ wv_all)
{
    constexpr int NW = NT / 32;
    constexpr int U = 4;
    extern __shared__ double smem[];
    __shared__ double dred[NW + 1];
    __shared__ unsigned long long kred[NW];
    __shared__ unsigned long long s_key;
    using R = typename sc_traits<T>::real;

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
    T* __restrict__ wv = wv_all + a0;
    int* alist = (int*)smem;                  // m: open columns (same order in every CTA)
    int* apos = alist + m;                    // m: position of a column in alist
    T* va = (T*)(apos + m);                   // r: v of the reflector being applied (2m ints keep
    T* vb = va + r;                           //    it 8-byte aligned); r: v of the next step

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool lo16 = lane < 16;
    unsigned long long* kb = keys + 2 * (cta_off ? (int64_t)cta_off[b] : (int64_t)b * G);   // [2][G], by parity
    unsigned int nbar = 0;
    R tau_a = R(0), tau_b = R(0);

    auto barrier = [&]() -> bool {
        if (G > 1) return group_sync(bar + b, (++nbar) * (unsigned)G, status, spin);
        __syncthreads();
        return true;
    };
    auto group_pivot = [&](int par) -> int {
        if (warp == 0) {
            unsigned long long t = 0;
            for (int q = lane; q < G; q += 32) {
                const unsigned long long u = G > 1 ? __ldcg(kb + par * G + q) : kb[par * G + q];
                t = u > t ? u : t;
            }
            t = warp_max_u64(t);
            if (lane == 0) s_key = t;
        }
        __syncthreads();
        return (int)(KEY_MASK - (s_key & KEY_MASK));
    };
    // Householder vector from x = v[s..r) (in place): alpha = |x|, v_s = x0 - beta with
    // beta = -(x0 / |x0|) alpha, tau = 2 / |v|^2
    auto householder = [&](const T* v, int s, double a2, T& beta, R& tau) -> double {
        const double alpha = sqrt(a2);
        const T x0 = v[s];
        const double ax0 = absd(x0);
        if constexpr (is_cplx<T>::value) beta = (ax0 > 0.0) ? rscale<T>(-alpha / ax0, x0) : T(R(-alpha));
        else beta = (T)(((double)x0 < 0.0) ? alpha : -alpha);
        tau = (R)(alpha > 0.0 ? 1.0 / (alpha * (alpha + ax0)) : 0.0);
        return alpha;
    };
    // the downdate of one or two columns after a dot product d (lanes 0-15 column j0, 16-31
    // j1 when TWO): R = y1 - tbv d, nv = |y|^2 - |R|^2, recomputed from the data below 1e-4 of
    // the reference; stores wv, nrm (and ref) and returns the key of this lane's column
    auto downdate = [&](auto two_c, int j0, int j1, T d, T y1, T tbv, const T* vv, R tau, int from,
                        const T* col0, const T* col1) -> unsigned long long {
        constexpr bool TWO = decltype(two_c)::value;
        const int jj = (TWO && !lo16) ? j1 : j0;
        const T rj = y1 - tbv * d;
        double nv = ldcg_(nrm + jj) - abs2d(rj);
        const unsigned need = __ballot_sync(0xffffffffu, nv < 1e-4 * ldcg_(ref + jj));
        if (need & 0x00010001u) {
            __syncwarp();                      // the recomputation reads the warp's stores
            for (int c = 0; c < (TWO ? 2 : 1); ++c) {
                if (!(need & (1u << (16 * c)))) continue;
                const T* col = c == 0 ? col0 : col1;
                const T dc = shfl_(d, 16 * c);
                const T td = tau * dc;
                double q = 0.0;
                for (int i2 = from + lane; i2 < r; i2 += 32) q += abs2d(fma_(-vv[i2], td, ldcg_(col + i2)));
                q = warp_sum(q);
                if (!TWO || (lane >> 4) == c) nv = q;
                if (lane == 16 * c) ref[jj] = q;
            }
        }
        if (lane == 0 || (TWO && lane == 16)) {
            nrm[jj] = nv;
            wv[jj] = d;
        }
        return pivot_key(nv, jj);
    };

    for (int j = threadIdx.x; j < m; j += NT) { alist[j] = j; apos[j] = j; }
    {
        // initial squared norms of a static share, and its best key for step 0
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
    if (kmax <= 0) goto done;
    {
        // step 0: pivot and reflector from the raw column
        if (!barrier()) return;
        const int p = group_pivot(0);
        if (p < 0 || p >= m) { if (threadIdx.x == 0) atomicOr(status, DEV_BADSIZE); goto done; }
        const T* colp = Y + (int64_t)p * r;
        double part = 0.0;
        for (int i = threadIdx.x; i < r; i += NT) {
            const T x = ldcg_(colp + i);
            va[i] = x;
            part += abs2d(x);
        }
        const double a2 = block_sum<NT>(part, dred);
        T beta;
        alpha0 = householder(va, 0, a2, beta, tau_a);
        if (!(alpha0 > 0.0)) goto done;
        __syncthreads();
        if (threadIdx.x == 0) {
            va[0] = va[0] - beta;
            if (gi == 0) { piv[a0] = p; diag[a0] = beta; }
            const int t = apos[p], lst = alist[nopen - 1];
            alist[t] = lst;
            apos[lst] = t;
        }
        --nopen;
        __syncthreads();
        // pass -1: w_j = v_0^H y_j (rows >= 0), R_{0,j} = y_j[0] - tau_0 v_0[0] w_j, downdate
        const int lo = (int)(((int64_t)gi * nopen) / G), hi = (int)(((int64_t)(gi + 1) * nopen) / G);
        const int C = hi - lo;
        const int wlo = lo + (int)(((int64_t)warp * C) / NW), whi = lo + (int)(((int64_t)(warp + 1) * C) / NW);
        unsigned long long wbest = 0;
        const T tbv = tau_a * va[0];
        auto dot0 = [&](auto two_c, int j0, int j1) {
            constexpr bool TWO = decltype(two_c)::value;
            const T* col0 = Y + (int64_t)j0 * r;
            const T* col1 = Y + (int64_t)j1 * r;
            T d0 = 0, d1 = 0, d0b = 0, d1b = 0, y0a = 0, y0b = 0;
            int i = lane;
            for (; i + 32 * (U - 1) < r; i += 32 * U) {
                T vv[U], xa[U], xb[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    vv[u] = conj_(va[i + 32 * u]);
                    xa[u] = ldcg_(col0 + i + 32 * u);
                    if constexpr (TWO) xb[u] = ldcg_(col1 + i + 32 * u);
                }
                if (i == 0) { y0a = xa[0]; if constexpr (TWO) y0b = xb[0]; }
#pragma unroll
                for (int u = 0; u < U; u += 2) {
                    d0 = fma_(vv[u], xa[u], d0);
                    d0b = fma_(vv[u + 1], xa[u + 1], d0b);
                    if constexpr (TWO) {
                        d1 = fma_(vv[u], xb[u], d1);
                        d1b = fma_(vv[u + 1], xb[u + 1], d1b);
                    }
                }
            }
            for (; i < r; i += 32) {
                const T vv = conj_(va[i]);
                const T xa = ldcg_(col0 + i);
                if (i == 0) y0a = xa;
                d0 = fma_(vv, xa, d0);
                if constexpr (TWO) {
                    const T xb = ldcg_(col1 + i);
                    if (i == 0) y0b = xb;
                    d1 = fma_(vv, xb, d1);
                }
            }
            d0 += d0b;
            T d, y1;
            if constexpr (TWO) {
                d1 += d1b;
                d = (lo16 ? d0 : d1) + shfl_xor_(lo16 ? d1 : d0, 16);
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) d += shfl_xor_(d, o);
                const T ya = shfl_(y0a, 0), yb = shfl_(y0b, 0);
                y1 = lo16 ? ya : yb;
            } else {
                d = warp_sum(d0);
                y1 = shfl_(y0a, 0);
            }
            const unsigned long long kq = downdate(two_c, j0, j1, d, y1, tbv, va, tau_a, 1, col0, col1);
            wbest = kq > wbest ? kq : wbest;
        };
        int t = wlo;
        for (; t + 1 < whi; t += 2) dot0(std::true_type{}, alist[t], alist[t + 1]);
        if (t < whi) dot0(std::false_type{}, alist[t], alist[t]);
        wbest = block_max_u64<NT>(wbest, kred);
        if (threadIdx.x == 0) kb[G + gi] = wbest;
    }
    for (int s = 0;; ++s) {
        // the pivot of step s+1 and its reflector (or the end of the factorisation)
        if (!barrier()) return;
        bool last = s + 1 >= kmax;
        if (!last) {
            const int p = group_pivot((s + 1) & 1);
            if (p < 0 || p >= m) { if (threadIdx.x == 0) atomicOr(status, DEV_BADSIZE); goto done; }
            const T* colp = Y + (int64_t)p * r;
            const T tw = tau_a * ldcg_(wv + p);
            double part = 0.0;
            for (int i = s + 1 + threadIdx.x; i < r; i += NT) {
                const T x = fma_(-va[i], tw, ldcg_(colp + i));
                vb[i] = x;
                part += abs2d(x);
            }
            const double a2 = block_sum<NT>(part, dred);
            T beta;
            const double alpha = householder(vb, s + 1, a2, beta, tau_b);
            if (!(alpha > eps * alpha0)) {
                last = true;
                if (!barrier()) return;      // every CTA is done reading column p
            } else {
                __syncthreads();
                if (threadIdx.x == 0) {
                    vb[s + 1] = vb[s + 1] - beta;
                    if (gi == 0) {
                        piv[a0 + s + 1] = p;
                        diag[a0 + s + 1] = beta;
                        T* ys = Y + (int64_t)p * r + s;
                        *ys = fma_(-va[s], tw, ldcg_(ys));      // R_{s,p}
                    }
                    const int t = apos[p], lst = alist[nopen - 1];
                    alist[t] = lst;
                    apos[lst] = t;
                }
                --nopen;
                __syncthreads();
            }
        }
        // pass s over this CTA's share of the open columns: equal runs per warp, two columns at
        // a time, a single column at the end of an odd run
        const int lo = (int)(((int64_t)gi * nopen) / G), hi = (int)(((int64_t)(gi + 1) * nopen) / G);
        const int C = hi - lo;
        const int wlo = lo + (int)(((int64_t)warp * C) / NW), whi = lo + (int)(((int64_t)(warp + 1) * C) / NW);
        unsigned long long wbest = 0;
        const T tbv = last ? T(0) : tau_b * vb[s + 1];
        auto cols = [&](auto two_c, int j0, int j1) {
            constexpr bool TWO = decltype(two_c)::value;
            T* col0 = Y + (int64_t)j0 * r;
            T* col1 = Y + (int64_t)j1 * r;
            const T tw0 = tau_a * ldcg_(wv + j0);
            const T tw1 = TWO ? tau_a * ldcg_(wv + j1) : T(0);
            T d0 = 0, d1 = 0, d0b = 0, d1b = 0, y1a = 0, y1b = 0;
            int i = s + lane;
            // first block: row s takes the update only; row s+1 is captured (lane 1, u = 0)
            if (i + 32 * (U - 1) < r) {
                T xa[U], xb[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    xa[u] = fma_(-va[i + 32 * u], tw0, ldcg_(col0 + i + 32 * u));
                    col0[i + 32 * u] = xa[u];
                    if constexpr (TWO) {
                        xb[u] = fma_(-va[i + 32 * u], tw1, ldcg_(col1 + i + 32 * u));
                        col1[i + 32 * u] = xb[u];
                    }
                }
                if (!last) {
                    y1a = xa[0];
                    if constexpr (TWO) y1b = xb[0];
                    const T v0 = lane == 0 ? T(0) : conj_(vb[i]);
                    d0 = v0 * xa[0];
                    if constexpr (TWO) d1 = v0 * xb[0];
#pragma unroll
                    for (int u = 1; u < U; ++u) {
                        const T vv = conj_(vb[i + 32 * u]);
                        d0 = fma_(vv, xa[u], d0);
                        if constexpr (TWO) d1 = fma_(vv, xb[u], d1);
                    }
                }
                i += 32 * U;
                if (last) {
                    for (; i + 32 * (U - 1) < r; i += 32 * U) {
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const T vv = va[i + 32 * u];
                            col0[i + 32 * u] = fma_(-vv, tw0, ldcg_(col0 + i + 32 * u));
                            if constexpr (TWO) col1[i + 32 * u] = fma_(-vv, tw1, ldcg_(col1 + i + 32 * u));
                        }
                    }
                } else {
                    for (; i + 32 * (U - 1) < r; i += 32 * U) {
                        T x0[U], x1[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            x0[u] = ldcg_(col0 + i + 32 * u);
                            if constexpr (TWO) x1[u] = ldcg_(col1 + i + 32 * u);
                        }
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const T vv = va[i + 32 * u];
                            x0[u] = fma_(-vv, tw0, x0[u]);
                            col0[i + 32 * u] = x0[u];
                            if constexpr (TWO) {
                                x1[u] = fma_(-vv, tw1, x1[u]);
                                col1[i + 32 * u] = x1[u];
                            }
                        }
#pragma unroll
                        for (int u = 0; u < U; u += 2) {
                            const T w0 = conj_(vb[i + 32 * u]), w1 = conj_(vb[i + 32 * u + 32]);
                            d0 = fma_(w0, x0[u], d0);
                            d0b = fma_(w1, x0[u + 1], d0b);
                            if constexpr (TWO) {
                                d1 = fma_(w0, x1[u], d1);
                                d1b = fma_(w1, x1[u + 1], d1b);
                            }
                        }
                    }
                }
            }
            // the rows left over (and all rows of a short column)
            for (; i < r; i += 32) {
                const T vv = va[i];
                const T xa = fma_(-vv, tw0, ldcg_(col0 + i));
                col0[i] = xa;
                T xb = 0;
                if constexpr (TWO) {
                    xb = fma_(-vv, tw1, ldcg_(col1 + i));
                    col1[i] = xb;
                }
                if (!last) {
                    if (i == s + 1) { y1a = xa; y1b = xb; }
                    if (i > s) {
                        const T w = conj_(vb[i]);
                        d0 = fma_(w, xa, d0);
                        if constexpr (TWO) d1 = fma_(w, xb, d1);
                    }
                }
            }
            if (last) return;
            d0 += d0b;
            T d, y1;
            if constexpr (TWO) {
                d1 += d1b;
                d = (lo16 ? d0 : d1) + shfl_xor_(lo16 ? d1 : d0, 16);
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) d += shfl_xor_(d, o);
                const T ya = shfl_(y1a, 1), yb = shfl_(y1b, 1);
                y1 = lo16 ? ya : yb;
            } else {
                d = warp_sum(d0);
                y1 = shfl_(y1a, 1);
            }
            const unsigned long long kq = downdate(two_c, j0, j1, d, y1, tbv, vb, tau_b, s + 2, col0, col1);
            wbest = kq > wbest ? kq : wbest;
        };
        int t = wlo;
        for (; t + 1 < whi; t += 2) cols(std::true_type{}, alist[t], alist[t + 1]);
        if (t < whi) cols(std::false_type{}, alist[t], alist[t]);
        if (last) { k = s + 1; break; }
        wbest = block_max_u64<NT>(wbest, kred);
        if (threadIdx.x == 0) kb[((s + 2) & 1) * G + gi] = wbest;
        T* tmp = va; va = vb; vb = tmp;
        tau_a = tau_b;
    }
done:
    if (gi == 0 && threadIdx.x == 0) kout[b] = k;
}

template <class T>
static size_t cpqr_la_shm(int max_r, int max_m)
{
    return sizeof(int) * (size_t)(2 * max_m + 2) + sizeof(T) * 2 * (size_t)max_r + 64;
}

template <class T>
cudaError_t launch_cpqr_la(cudaStream_t st, int nb, int G, const int32_t* cta_off, int ctas, const int64_t* act_off,
                           const int32_t* nnear, int P, const int64_t* y_off, T* Y, double eps, int32_t* kout,
                           int32_t* piv, T* diag, unsigned int* bar, unsigned long long* keys, int* status,
                           long long spin_limit, int max_r, int max_m, double* nrm, double* ref, T* wv)
{
    constexpr int NT = 256;
    if (nb <= 0) return cudaSuccess;
    const size_t shm = cpqr_la_shm<T>(max_r, max_m);
    cudaError_t e = cudaFuncSetAttribute(cpqr_la_kernel<NT, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e != cudaSuccess) return e;
    count_launches(1);
    if (!cta_off && G == 1) {
        cpqr_la_kernel<NT, T><<<nb, NT, shm, st>>>(1, nullptr, act_off, nnear, P, y_off, Y, eps, kout, piv, diag, bar,
                                                   keys, status, spin_limit, nrm, ref, wv);
        return cudaGetLastError();
    }
    int g0 = cta_off ? nb : G;
    void* args[] = {(void*)&g0, (void*)&cta_off, (void*)&act_off, (void*)&nnear, (void*)&P, (void*)&y_off, (void*)&Y,
                    (void*)&eps, (void*)&kout, (void*)&piv, (void*)&diag, (void*)&bar, (void*)&keys, (void*)&status,
                    (void*)&spin_limit, (void*)&nrm, (void*)&ref, (void*)&wv};
    return cudaLaunchCooperativeKernel((void*)cpqr_la_kernel<NT, T>, dim3((unsigned)(cta_off ? ctas : nb * G)),
                                       dim3(NT), args, shm, st);
}

template <class T>
int cpqr_la_max_ctas(int max_r, int max_m)
{
    constexpr int NT = 256;
    const size_t shm = cpqr_la_shm<T>(max_r, max_m);
    if (shm > 227 * 1024) return 0;
    if (cudaFuncSetAttribute(cpqr_la_kernel<NT, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) !=
        cudaSuccess)
        return 0;
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cpqr_la_kernel<NT, T>, NT, shm) != cudaSuccess) return 0;
    return per_sm * sms;
}

#define RS_INST_CPQR_LA(T)                                                                                            \
    template cudaError_t launch_cpqr_la<T>(cudaStream_t, int, int, const int32_t*, int, const int64_t*,              \
                                           const int32_t*, int, const int64_t*, T*, double, int32_t*, int32_t*, T*, \
                                           unsigned int*, unsigned long long*, int*, long long, int, int, double*,  \
                                           double*, T*);                                                            \
    template int cpqr_la_max_ctas<T>(int, int);
RS_INST_CPQR_LA(double)
RS_INST_CPQR_LA(float)
RS_INST_CPQR_LA(cplx<double>)
RS_INST_CPQR_LA(cplx<float>)

}  // namespace rs
