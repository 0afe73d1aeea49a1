// k_cpqr_cl.cu -- column-pivoted QR (Sec. 2.1, Eq. 2.1) of boxes small enough to live in the
// shared memory of one thread-block cluster.
//
// One cluster of C CTAs per box.  CTA c holds the columns [c m / C, (c+1) m / C) of the box's Y
// (all r rows, column-major with a padded stride) in its shared memory for the whole
// factorization: Y is read from HBM once and R is written back once, and no step touches HBM.
// Each step:
//   1. after one cluster barrier, every CTA reads the C best pivot keys (one per CTA, written
//      in its own shared memory at the end of the previous step) through distributed shared
//      memory and takes the same maximum: the pivot column p and the CTA that holds it;
//   2. every CTA copies column p (rows s..r-1) from the owner's shared memory into its own and
//      forms the same Householder vector with the same arithmetic (so all CTAs agree on the
//      rank test bit for bit); the owner drops p from its list of open columns;
//   3. every CTA applies the reflector to its own open columns, one column per thread and
//      the rows split over groups of threads (no cross-lane reduction, so the FP64 pipe does
//      only the dot-product and update FMAs plus one short sum per column), downdates the
//      squared column norms (recomputed from the data once below 1e-4 of the value they were
//      last computed from) and writes its best key for the next step.
// The pivot rule (largest key, lowest column on ties, keys as in the other CPQR kernels) and
// the rank rule (|R_ss| > eps |R_00|) are those of cpqr_kernel, so the skeletons agree with
// it.  Results: kout (rank), piv (pivot order), diag (R_ss), and rows 0..k-1 of every column of
// Y hold R, as cpqr_kernel leaves them.  All CTAs of a cluster run the same number of steps
// (the loop bounds and the rank test are uniform), so every cluster barrier is reached by all.
#include <cooperative_groups.h>

#include "k_common.cuh"

namespace cg = cooperative_groups;

namespace rs {

// Shared-memory layout of one CTA (bytes), for at most `ncmax` columns of stride `ld`.
template <class T>
struct ClLayout {
    size_t y, v, part, tw, nrm, ref, open, pos, rec, total;
    __host__ __device__ ClLayout(int ncmax, int ld, int nt)
    {
        size_t o = 0;
        auto take = [&](size_t bytes) { const size_t at = o; o = (o + bytes + 15) & ~(size_t)15; return at; };
        y = take(sizeof(T) * (size_t)ncmax * (size_t)ld);
        v = take(sizeof(T) * (size_t)ld);
        part = take(sizeof(T) * (size_t)nt);
        tw = take(sizeof(T) * (size_t)ncmax);
        nrm = take(sizeof(double) * (size_t)ncmax);
        ref = take(sizeof(double) * (size_t)ncmax);
        open = take(sizeof(int) * (size_t)ncmax);
        pos = take(sizeof(int) * (size_t)ncmax);
        rec = take(sizeof(int) * (size_t)ncmax);
        total = o;
    }
};

template <int NT, class T>
__global__ void __launch_bounds__(NT) cpqr_cl_kernel(int C, const int64_t* __restrict__ act_off,
        const int32_t* __restrict__ nnear, int P, const int64_t* __restrict__ y_off, T* __restrict__ Yall,
        double eps, int32_t* __restrict__ kout, int32_t* __restrict__ piv, T* __restrict__ diag,
        int* __restrict__ status, int ncmax, int ld)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ unsigned long long keys[2];          // this CTA's best key, by step parity
    __shared__ unsigned long long kred[NT / 32];
    __shared__ double dred[NT / 32 + 1];
    __shared__ unsigned long long s_key;
    __shared__ int s_nrec;                            // columns whose norm is recomputed

    cg::cluster_group cluster = cg::this_cluster();
    const int c = (int)cluster.block_rank();
    const int b = (int)(blockIdx.x / (unsigned)C);
    const int64_t a0 = act_off[b];
    const int m = (int)(act_off[b + 1] - a0);
    const int r = nnear[b] + P;
    const int j0 = (int)(((int64_t)c * m) / C), j1 = (int)(((int64_t)(c + 1) * m) / C);
    const int nc = j1 - j0;
    T* __restrict__ Yg = Yall + y_off[b];

    const ClLayout<T> Lo(ncmax, ld, NT);
    T* __restrict__ Ys = (T*)(smraw + Lo.y);
    T* __restrict__ v = (T*)(smraw + Lo.v);
    T* __restrict__ part = (T*)(smraw + Lo.part);
    T* __restrict__ tw = (T*)(smraw + Lo.tw);
    double* __restrict__ nrm = (double*)(smraw + Lo.nrm);
    double* __restrict__ ref = (double*)(smraw + Lo.ref);
    int* __restrict__ open = (int*)(smraw + Lo.open);
    int* __restrict__ pos = (int*)(smraw + Lo.pos);
    int* __restrict__ rec = (int*)(smraw + Lo.rec);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int NW = NT / 32;
    using R = typename sc_traits<T>::real;

    // load the slice (coalesced along each column), open list, initial norms and keys; whether
    // the box fits is decided per box, so all CTAs of the cluster take the same path
    const bool fits = (m + C - 1) / C <= ncmax && r <= ld;
    if (fits) {
        const int64_t tot = (int64_t)nc * r;
        for (int64_t e = threadIdx.x; e < tot; e += NT) {
            const int jl = (int)(e / r), i = (int)(e - (int64_t)jl * r);
            Ys[(int64_t)jl * ld + i] = Yg[(int64_t)(j0 + jl) * r + i];
        }
        for (int q = threadIdx.x; q < nc; q += NT) { open[q] = q; pos[q] = q; }
    } else if (threadIdx.x == 0) {
        atomicOr(status, DEV_BADSIZE);
    }
    __syncthreads();
    unsigned long long best = 0;
    if (fits) {
        for (int jl = warp; jl < nc; jl += NW) {
            double q = 0.0;
            for (int i = lane; i < r; i += 32) q += abs2d(Ys[(int64_t)jl * ld + i]);
            q = warp_sum(q);
            if (lane == 0) { nrm[jl] = q; ref[jl] = q; }
            const unsigned long long kq = pivot_key(q, j0 + jl);
            best = kq > best ? kq : best;
        }
    }
    best = block_max_u64<NT>(best, kred);
    if (threadIdx.x == 0) keys[0] = best;
    cluster.sync();

    int nopen = fits ? nc : 0;
    const int kmax = fits ? min(r, m) : 0;
    int k = 0;
    double alpha0 = 0.0;
    for (int s = 0; s < kmax; ++s) {
        // 1. the cluster's pivot
        if (warp == 0) {
            unsigned long long t = 0;
            if (lane < C) {
                const unsigned long long* rk = cluster.map_shared_rank(&keys[s & 1], lane);
                t = *(volatile const unsigned long long*)rk;
            }
            t = warp_max_u64(t);
            if (lane == 0) s_key = t;
        }
        __syncthreads();
        const unsigned long long bk = s_key;
        const int p = (int)(KEY_MASK - (bk & KEY_MASK));
        if (p < 0 || p >= m) {                   // uniform: every CTA read the same keys
            if (threadIdx.x == 0 && c == 0) atomicOr(status, DEV_BADSIZE);
            break;
        }
        int owner = 0;
        for (int q = 1; q < C; ++q)
            if ((int)(((int64_t)q * m) / C) <= p) owner = q;
        const int lp = p - (int)(((int64_t)owner * m) / C);
        // 2. the Householder vector from the owner's copy of column p (rows s..r-1)
        const T* colp = cluster.map_shared_rank(Ys + (int64_t)lp * ld, owner);
        double part2 = 0.0;
        for (int i = s + threadIdx.x; i < r; i += NT) {
            const T x = colp[i];
            v[i] = x;
            part2 += abs2d(x);
        }
        if (owner == c && threadIdx.x == 0) {
            const int t = pos[lp], last = open[nopen - 1];
            open[t] = last;
            pos[last] = t;
        }
        if (owner == c) --nopen;
        const double a2 = block_sum<NT>(part2, dred);       // its barriers also order v and open[]
        const double alpha = sqrt(a2);
        if (s == 0) alpha0 = alpha;
        if (!(alpha > eps * alpha0)) break;                 // uniform (same data, same order)
        const T x0 = v[s];
        const double ax0 = absd(x0);
        T beta;
        if constexpr (is_cplx<T>::value) beta = (ax0 > 0.0) ? rscale<T>(-alpha / ax0, x0) : T(R(-alpha));
        else beta = (T)(((double)x0 < 0.0) ? alpha : -alpha);
        const R tau = (R)(1.0 / (alpha * (alpha + ax0)));   // 2 / |v|^2
        __syncthreads();
        if (threadIdx.x == 0) {
            v[s] = x0 - beta;
            if (c == 0) { piv[a0 + s] = p; diag[a0 + s] = beta; }
        }
        __syncthreads();
        // 3. this CTA's open columns: thread -> (slot, row group); slot q is open[q]
        const int NS = max(nopen, 1);
        const int RG = min(32, max(1, NT / NS));
        const int slot = (int)threadIdx.x % NS, rg = (int)threadIdx.x / NS;
        const bool act = nopen > 0 && rg < RG;
        const int rlo = s + (int)(((int64_t)(r - s) * rg) / RG), rhi = s + (int)(((int64_t)(r - s) * (rg + 1)) / RG);
        const int jl = act ? open[slot] : 0;
        T* __restrict__ col = Ys + (int64_t)jl * ld;
        if (act) {
            T w0 = T(0), w1 = T(0), w2 = T(0), w3 = T(0);
            int i = rlo;
            for (; i + 3 < rhi; i += 4) {
                w0 = fma_(conj_(v[i]), col[i], w0);
                w1 = fma_(conj_(v[i + 1]), col[i + 1], w1);
                w2 = fma_(conj_(v[i + 2]), col[i + 2], w2);
                w3 = fma_(conj_(v[i + 3]), col[i + 3], w3);
            }
            for (; i < rhi; ++i) w0 = fma_(conj_(v[i]), col[i], w0);
            part[rg * NS + slot] = (w0 + w1) + (w2 + w3);
        }
        if (threadIdx.x == 0) s_nrec = 0;
        __syncthreads();
        if (nopen > 0 && threadIdx.x < nopen) {
            T w = part[threadIdx.x];
            for (int q = 1; q < RG; ++q) w += part[q * NS + threadIdx.x];
            const T t = tau * w;
            tw[threadIdx.x] = t;
            const int jq = open[threadIdx.x];
            const T rsj = fma_(-v[s], t, Ys[(int64_t)jq * ld + s]);   // row s after the update
            const double nv = nrm[jq] - abs2d(rsj);
            nrm[jq] = nv;
            if (nv < 1e-4 * ref[jq]) rec[atomicAdd(&s_nrec, 1)] = jq;
        }
        __syncthreads();
        if (act) {
            const T t = tw[slot];
            int i = rlo;
            for (; i + 3 < rhi; i += 4) {
                const T y0 = fma_(-v[i], t, col[i]);
                const T y1 = fma_(-v[i + 1], t, col[i + 1]);
                const T y2 = fma_(-v[i + 2], t, col[i + 2]);
                const T y3 = fma_(-v[i + 3], t, col[i + 3]);
                col[i] = y0;
                col[i + 1] = y1;
                col[i + 2] = y2;
                col[i + 3] = y3;
            }
            for (; i < rhi; ++i) col[i] = fma_(-v[i], t, col[i]);
        }
        __syncthreads();
        // norms that fell below 1e-4 of their reference: recomputed from the updated rows
        // s+1..r-1, one warp per column
        const int nrec = s_nrec;
        if (nrec > 0) {
            for (int q = warp; q < nrec; q += NW) {
                const int jq = rec[q];
                const T* cq = Ys + (int64_t)jq * ld;
                double acc = 0.0;
                for (int i = s + 1 + lane; i < r; i += 32) acc += abs2d(cq[i]);
                acc = warp_sum(acc);
                if (lane == 0) { nrm[jq] = acc; ref[jq] = acc; }
            }
            __syncthreads();
        }
        best = 0;
        if (nopen > 0 && threadIdx.x < nopen) {
            const int jq = open[threadIdx.x];
            best = pivot_key(nrm[jq], j0 + jq);
        }
        best = block_max_u64<NT>(best, kred);
        if (threadIdx.x == 0) keys[(s + 1) & 1] = best;
        k = s + 1;
        cluster.sync();
    }
    // no CTA leaves (and frees the shared memory others read) before all are done
    cluster.sync();
    if (fits) {
        const int kr = min(k, r);
        const int64_t tot = (int64_t)nc * kr;
        for (int64_t e = threadIdx.x; e < tot; e += NT) {
            const int q = (int)(e / kr), i = (int)(e - (int64_t)q * kr);
            Yg[(int64_t)(j0 + q) * r + i] = Ys[(int64_t)q * ld + i];
        }
    }
    if (c == 0 && threadIdx.x == 0) kout[b] = k;
}

namespace {
constexpr int CL_NT = 256;
constexpr size_t CL_SMEM_MAX = 227 * 1024;

int cl_stride(int max_r) { return max_r | 1; }     // odd: columns start in different banks
}  // namespace

// Launch configuration of variant 4 for boxes up to max_r x max_m with clusters of C CTAs:
// sets the kernel's attributes and fills cfg (its attribute array in attr); returns the
// clusters that can be resident at once (0: this C cannot be launched for these sizes).
template <class T>
static int cl_config(int C, int max_r, int max_m, cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, int& ncmax,
                     int& ld)
{
    ld = cl_stride(max_r);
    ncmax = (max_m + C - 1) / C;
    if (C < 2 || C > 16 || ncmax > CL_NT) return 0;
    const size_t shm = ClLayout<T>(ncmax, ld, CL_NT).total;
    if (shm > CL_SMEM_MAX - 2048) return 0;
    auto fn = cpqr_cl_kernel<CL_NT, T>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) != cudaSuccess ||
        (C > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
        cudaGetLastError();
        return 0;
    }
    cfg = cudaLaunchConfig_t{};
    cfg.blockDim = dim3(CL_NT);
    cfg.dynamicSmemBytes = shm;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((unsigned)(C * 64));
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return clusters;
}

// Cluster size for a launch whose largest box is max_r x max_m (0: no size fits).  The
// smallest C in 2, 4, 8, 16 that keeps two CTAs per SM resident (so that one box's serial part
// of a step overlaps another box's updates); failing that, the C with the most CTAs resident
// at once, the smaller on a tie (fewer CTAs per box to keep in step).
template <class T>
int cpqr_cl_cluster(int max_r, int max_m)
{
    if (max_r <= 0 || max_m <= 0) return 0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int best = 0, best_ctas = 0;
    for (int C = 2; C <= 16; C *= 2) {
        cudaLaunchConfig_t cfg;
        cudaLaunchAttribute attr[1];
        int ncmax = 0, ld = 0;
        const int ctas = cl_config<T>(C, max_r, max_m, cfg, attr, ncmax, ld) * C;
        if (ctas >= 2 * sms) return C;
        if (ctas > best_ctas) { best = C; best_ctas = ctas; }
    }
    return best;
}

template <class T>
cudaError_t launch_cpqr_cl(cudaStream_t st, int nb, int C, const int64_t* act_off, const int32_t* nnear, int P,
                           const int64_t* y_off, T* Y, double eps, int32_t* kout, int32_t* piv, T* diag, int* status,
                           int max_r, int max_m)
{
    if (nb <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    int ncmax = 0, ld = 0;
    if (cl_config<T>(C, max_r, max_m, cfg, attr, ncmax, ld) < 1) return cudaErrorInvalidConfiguration;
    cfg.gridDim = dim3((unsigned)(nb * C));
    cfg.stream = st;
    count_launches(1);
    return cudaLaunchKernelEx(&cfg, cpqr_cl_kernel<CL_NT, T>, C, act_off, nnear, P, y_off, Y, eps, kout, piv, diag,
                              status, ncmax, ld);
}

#define RS_INST_CPQR_CL(T)                                                                                             \
    template int cpqr_cl_cluster<T>(int, int);                                                                         \
    template cudaError_t launch_cpqr_cl<T>(cudaStream_t, int, int, const int64_t*, const int32_t*, int,              \
                                           const int64_t*, T*, double, int32_t*, int32_t*, T*, int*, int, int);
RS_INST_CPQR_CL(double)
RS_INST_CPQR_CL(float)
RS_INST_CPQR_CL(cplx<double>)
RS_INST_CPQR_CL(cplx<float>)

}  // namespace rs
