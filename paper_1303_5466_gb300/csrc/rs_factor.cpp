// rs_factor.cpp -- rs_factor / rs_solve: host orchestration of the per-level CUDA kernels.
//
// Factor (Algorithm 1, level by level, every box of a level in one launch):
//   ID phase   (l = d..1): Y assembly -> column-pivoted QR -> T = R11^{-1} R12
//   inverse    (l = d..1): F' = Pi^T F Pi -> Phi = F'^{-1} (Gauss-Jordan) ->
//              W = Phi L, E^{-1} = R W (grouped GEMMs) -> E (Gauss-Jordan); root: F_root^{-1}
// Solve (Algorithm 6 as the recursion of Eqs. 2.10-2.12), nrhs columns per launch.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <map>
#include <chrono>
#include <cmath>
#include <functional>
#include <memory>
#include <string>
#include <vector>

#include "rs_host.h"

namespace rs {

namespace {

using Clock = std::chrono::steady_clock;
double ms_since(Clock::time_point t0) { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }

template <class T>
int upload(DevMem& d, const std::vector<T>& h, cudaStream_t st)
{
    RS_CUDA(d.alloc(sizeof(T) * (h.empty() ? 1 : h.size())));
    if (!h.empty()) RS_CUDA(cudaMemcpyAsync(d.p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st));
    return RS_OK;
}

template <class T>
std::vector<int32_t> to32(const std::vector<T>& v)
{
    std::vector<int32_t> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = (int32_t)v[i];
    return o;
}

// Event pair around one kernel launch when opts.profile is set; the elapsed time and the
// launch's algorithmic work are added to the class sums by prof_flush after a sync.
struct ProfScope {
    rs_op* op;
    int cls;
    cudaStream_t st;
    double work, bytes;
    int level;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    static cudaEvent_t take(rs_op* o)
    {
        if (!o->ev_pool.empty()) {
            cudaEvent_t e = o->ev_pool.back();
            o->ev_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        o->ev_all.push_back(e);
        return e;
    }
    ProfScope(rs_op* o, int c, cudaStream_t s, double w, double b = 0.0, int lvl = -1)
        : op(o), cls(c), st(s), work(w), bytes(b), level(lvl)
    {
        if (!op->opts.profile) return;
        e0 = take(op);
        e1 = take(op);
        if (e0 && e1) cudaEventRecord(e0, st);
    }
    ~ProfScope()
    {
        if (!e0 || !e1) return;
        cudaEventRecord(e1, st);
        op->pending.push_back({cls, level, e0, e1, work, bytes});
    }
};

void prof_flush(rs_op* op)
{
    for (const ProfRec& r : op->pending) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) {
            op->prof_ms[r.cls] += ms;
            op->prof_work[r.cls] += r.work;
            op->prof_bytes[r.cls] += r.bytes;
            op->prof_n[r.cls] += 1;
            if (r.level >= 0) {
                std::vector<double>& v = op->prof_level_ms[r.cls];
                if ((int)v.size() <= r.level) v.resize(r.level + 1, 0.0);
                v[r.level] += ms;
            }
        }
        op->ev_pool.push_back(r.e0);
        op->ev_pool.push_back(r.e1);
    }
    op->pending.clear();
}

int check_status(rs_op* op, cudaStream_t st)
{
    RS_CUDA(cudaStreamSynchronize(st));
    prof_flush(op);
    int s = 0;
    RS_CUDA(cudaMemcpy(&s, op->d_status.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (s & DEV_TIMEOUT) return fail(RS_E_TIMEOUT, "a device-side wait exceeded spin_limit");
    if (s & DEV_SINGULAR) return fail(RS_E_SINGULAR, "pivot below 1e3 unit roundoff times the largest earlier pivot");
    if (s & DEV_BADSIZE) return fail(RS_E_CUDA, "a kernel found an out-of-range index and stopped");
    return RS_OK;
}

}  // namespace

// Pick the CTA group size per box for a cooperative kernel (capacity(G): co-resident CTAs
// when each box takes G CTAs, 0 if such a CTA does not fit on an SM).  Start from the smallest
// G whose CTAs fit; keep it when the boxes alone fill the GPU.  Otherwise take up to
// max_cols / 32 CTAs per box (and 1024), as many as stay co-resident, preferring a total
// that loads every SM with the same number of CTAs: a group runs at the pace of its slowest
// CTA, so CTAs that share an SM with one more neighbour than the others hold back the group.
int choose_group(int nb, int max_cols, const std::function<int(int)>& capacity)
{
    const int gmax = std::max(1, std::min(max_cols / 32, 1024));
    int g0 = 1;
    while (g0 < gmax && capacity(g0) <= 0) ++g0;
    const int cap0 = capacity(g0);
    if (cap0 <= 0 || g0 == gmax || nb * g0 >= cap0) return g0;
    int G = std::min(gmax, cap0 / std::max(nb, 1));
    while (G > g0 && nb * G > capacity(G)) --G;
    G = std::max(G, g0);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess || sms <= 0)
        return G;
    // evenness of the per-SM load of T CTAs: T / (sms * ceil(T / sms))
    auto even = [&](int g) {
        const double T = (double)nb * g;
        return T / (sms * std::ceil(T / sms));
    };
    int best = G;
    for (int g = G - 1; g >= g0 && g >= G / 2; --g)
        if (even(g) > even(best) + 0.02) best = g;
    return best;
}

std::vector<int32_t> proportional_groups(int total, const std::vector<double>& work, const std::vector<int>& cap)
{
    const int nb = (int)work.size();
    double W = 0.0;
    for (double w : work) W += w;
    std::vector<int> gb(nb);
    int used = 0;
    for (int b = 0; b < nb; ++b) {
        gb[b] = std::max(1, std::min(cap[b], W > 0.0 ? (int)std::floor(total * work[b] / W) : 1));
        used += gb[b];
    }
    while (used < total) {              // the rest to the groups with the most work per CTA
        int best = -1;
        for (int b = 0; b < nb; ++b)
            if (gb[b] < cap[b] && (best < 0 || work[b] / gb[b] > work[best] / gb[best])) best = b;
        if (best < 0) break;
        ++gb[best];
        ++used;
    }
    std::vector<int32_t> off(nb + 1, 0);
    for (int b = 0; b < nb; ++b) off[b + 1] = off[b] + gb[b];
    return off;
}

namespace {

// Workspace of the ID phase, released when rs_factor returns.
struct IdWork {
    DevMem near, near_off, geo, y_off, nn, piv, diag, skpos, rscol, Y, keys, norms, cta_off, gwork, blk;
};

template <class T>
int run_gj(rs_op* op, cudaStream_t st, int nb, const DevMem& dm, const DevMem& doff, T* A,
           const std::vector<int64_t>& sizes, const std::vector<int64_t>& size_off, int max_m, int cls, int level)
{
    if (max_m <= 0) return RS_OK;
    DevMem& d_ipoff = op->t_ipoff;      // kept by the op: a freed buffer would synchronise the device
    RS_CUDA(d_ipoff.alloc(sizeof(int64_t) * nb));
    RS_CUDA(cudaMemcpyAsync(d_ipoff.p, size_off.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice, st));
    const int64_t tot = size_off[nb];
    RS_CUDA(op->d_ipiv.alloc(sizeof(int32_t) * (tot + 1)));
    RS_CUDA(op->d_pivrow.alloc(sizeof(int) * 2 * (size_t)gj_panel_width() * nb));
    RS_CUDA(op->d_bar.alloc(sizeof(unsigned int) * nb));
    RS_CUDA(cudaMemsetAsync(op->d_bar.p, 0, sizeof(unsigned int) * nb, st));
    // one CTA per panel of columns at most
    const int G = choose_group(nb, max_m * 32 / gj_panel_width(), [&](int) { return gj_max_ctas<T>(max_m, nb); });
    double work = 0.0;
    for (int b = 0; b < nb; ++b) work += 2.0 * (double)sizes[b] * (double)sizes[b] * (double)sizes[b];
    ProfScope ps(op, cls, st, work, 2.0 * sizeof(T) * (double)size_off[nb], level);
    if (op->opts.per_box) {                 // one matrix per launch, each with the whole GPU
        for (int b = 0; b < nb; ++b) {
            const int mb = (int)sizes[b];
            if (mb <= 0) continue;
            const int Gb = choose_group(1, mb * 32 / gj_panel_width(), [&](int) { return gj_max_ctas<T>(mb, 1); });
            RS_CUDA(launch_gj_inverse<T>(st, 1, Gb, dm.as<int32_t>() + b, doff.as<int64_t>() + b, A,
                                         op->d_ipiv.as<int32_t>(), d_ipoff.as<int64_t>() + b,
                                         op->d_pivrow.as<int>() + 2 * (int64_t)gj_panel_width() * b,
                                         op->d_bar.as<unsigned int>() + b, op->d_status.as<int>(),
                                         (long long)op->opts.spin_limit, mb));
        }
        return check_status(op, st);
    }
    RS_CUDA(launch_gj_inverse<T>(st, nb, G, dm.as<int32_t>(), doff.as<int64_t>(), A, op->d_ipiv.as<int32_t>(),
                              d_ipoff.as<int64_t>(), op->d_pivrow.as<int>(), op->d_bar.as<unsigned int>(),
                              op->d_status.as<int>(), (long long)op->opts.spin_limit, max_m));
    return check_status(op, st);
}

// Symmetric sweep inverse of a level's SPD blocks (real kernels only).  *not_spd is set, and
// the status word cleared, when a block is not positive definite to working accuracy: the
// blocks are then partly swept and the caller rebuilds them for run_gj.  While op->defer_spd
// is set the launch returns without waiting: the status word is read once after the whole
// inverse phase, which is redone with Gauss-Jordan if any sweep found a block not SPD.
// The sweep in panels of 64 with its rank-64 updates on the digit-slice GEMM (FP64).
int run_sweep_bl(rs_op* op, cudaStream_t st, int nb, const DevMem& dm, const DevMem& doff, double* A,
                 const std::vector<int64_t>& sizes, const std::vector<int64_t>& moff, int max_m, int cls, int level)
{
    std::vector<int64_t> qoff;
    std::vector<std::vector<GemmProb>> gx, gu;
    const size_t qn = sweep_bl_plan(nb, sizes, max_m, qoff, gx, gu, moff);
    const int steps = (int)gx.size();
    // every step's descriptors and exponent offsets in one array each
    std::vector<GemmProb> ax, au;
    std::vector<int64_t> ex, eu;
    struct StepL { size_t px, pu, ex, eu; OzPlan x, u; int nx, nu; };
    std::vector<StepL> sl(steps);
    int64_t max_lines = 1, max_digits = 1;
    for (int q = 0; q < steps; ++q) {
        std::vector<int64_t> eo;
        StepL& z = sl[q];
        z.px = ax.size(); z.ex = ex.size(); z.nx = (int)gx[q].size();
        z.x = gemm_oz_plan(gx[q], eo);
        ax.insert(ax.end(), gx[q].begin(), gx[q].end());
        ex.insert(ex.end(), eo.begin(), eo.end());
        z.pu = au.size(); z.eu = eu.size(); z.nu = (int)gu[q].size();
        z.u = gemm_oz_plan(gu[q], eo);
        au.insert(au.end(), gu[q].begin(), gu[q].end());
        eu.insert(eu.end(), eo.begin(), eo.end());
        max_lines = std::max(max_lines, std::max(z.x.lines, z.u.lines));
        max_digits = std::max(max_digits, std::max(z.x.digits, z.u.digits));
    }
    int rc;
    if ((rc = upload(op->t_blq, qoff, st))) return rc;
    if ((rc = upload(op->t_blgx, ax, st))) return rc;
    if ((rc = upload(op->t_blgu, au, st))) return rc;
    if ((rc = upload(op->t_blex, ex, st))) return rc;
    if ((rc = upload(op->t_bleu, eu, st))) return rc;
    RS_CUDA(op->t_blQ.alloc(sizeof(double) * (qn + 1)));
    RS_CUDA(op->t_blX.alloc(sizeof(double) * (qn + 1)));
    RS_CUDA(op->t_blD.alloc(sizeof(double) * 64 * 64 * (size_t)nb));
    RS_CUDA(op->t_blmp.alloc(sizeof(double) * (size_t)nb));
    RS_CUDA(op->t_ozx.alloc(sizeof(int) * (size_t)max_lines));
    RS_CUDA(op->t_ozd.alloc(2 * (size_t)(max_digits + 8)));
    RS_CUDA(cudaMemsetAsync(op->t_blmp.p, 0, sizeof(double) * (size_t)nb, st));
    double work = 0.0;
    for (int b = 0; b < nb; ++b) work += (double)sizes[b] * (double)sizes[b] * (double)sizes[b];
    ProfScope ps(op, cls, st, work, 2.0 * sizeof(double) * (double)moff[nb], level);
    for (int q = 0; q < steps; ++q) {
        const StepL& z = sl[q];
        RS_CUDA(launch_sweep_bl_panel(st, nb, 64 * q, max_m, dm.as<int32_t>(), doff.as<int64_t>(), A,
                                      op->t_blq.as<int64_t>(), op->t_blQ.as<double>(), op->t_blD.as<double>(),
                                      op->t_blmp.as<double>(), op->d_status.as<int>()));
        RS_CUDA(launch_gemm_oz(st, op->t_blgx.as<GemmProb>() + z.px, z.nx, z.x, op->t_blex.as<int64_t>() + z.ex,
                               op->t_ozx.as<int>(), op->t_ozd.p, op->t_blQ.as<double>(), op->t_blD.as<double>(),
                               op->t_blX.as<double>(), op->t_blX.as<double>()));
        RS_CUDA(launch_gemm_oz(st, op->t_blgu.as<GemmProb>() + z.pu, z.nu, z.u, op->t_bleu.as<int64_t>() + z.eu,
                               op->t_ozx.as<int>(), op->t_ozd.p, op->t_blX.as<double>(), op->t_blQ.as<double>(), A,
                               A));
        RS_CUDA(launch_sweep_bl_write(st, nb, 64 * q, max_m, dm.as<int32_t>(), doff.as<int64_t>(), A,
                                      op->t_blq.as<int64_t>(), op->t_blX.as<double>(), op->t_blD.as<double>()));
    }
    RS_CUDA(launch_sweep_finish<double>(st, nb, dm.as<int32_t>(), doff.as<int64_t>(), A, max_m));
    return RS_OK;
}

template <class T>
int run_sweep(rs_op* op, cudaStream_t st, int nb, const DevMem& dm, const DevMem& doff, T* A,
              const std::vector<int64_t>& sizes, const std::vector<int64_t>& size_off, int max_m, int cls,
              int level, bool* not_spd, const std::vector<int64_t>* moff = nullptr)
{
    *not_spd = false;
    if (max_m <= 0) return RS_OK;
    if constexpr (std::is_same<T, double>::value) {
        if (moff && op->opts.gemm_form == 1 && !op->opts.per_box) {
            int rc;
            if ((rc = run_sweep_bl(op, st, nb, dm, doff, A, sizes, *moff, max_m, cls, level))) return rc;
            if (op->defer_spd) return RS_OK;
            RS_CUDA(cudaStreamSynchronize(st));
            prof_flush(op);
            int s = 0;
            RS_CUDA(cudaMemcpy(&s, op->d_status.p, sizeof(int), cudaMemcpyDeviceToHost));
            if (s & DEV_NOT_SPD) {
                RS_CUDA(cudaMemsetAsync(op->d_status.p, 0, sizeof(int), st));
                op->stats.spd_fallbacks += 1;
                *not_spd = true;
                return RS_OK;
            }
            return check_status(op, st);
        }
    }
    if constexpr (is_cplx<T>::value) {
        return fail(RS_E_INVALID, "the symmetric sweep is for real kernels");
    } else {
        // panel width: the autotuner's for this launch shape (or the candidate being timed)
        const std::string skey = tune_key("sweep", (int)sizeof(T), nb, max_m, 0);
        const int NB = g_trial.sweep_nb > 0       ? g_trial.sweep_nb
                       : op->opts.sweep_panel > 0 ? op->opts.sweep_panel
                                                  : (int)tune_get(skey + ".nb", (double)sweep_panel_width());
        std::vector<int64_t> pb_off(nb);
        for (int b = 0; b < nb; ++b) pb_off[b] = 2 * (int64_t)NB * size_off[b];
        DevMem& d_pboff = op->t_pboff;
        int rc;
        if ((rc = upload(d_pboff, pb_off, st))) return rc;
        RS_CUDA(op->d_pb.alloc(sizeof(T) * 2 * (size_t)NB * (size_t)(size_off[nb] + 1)));
        RS_CUDA(op->d_bar.alloc(sizeof(unsigned int) * nb));
        RS_CUDA(cudaMemsetAsync(op->d_bar.p, 0, sizeof(unsigned int) * nb, st));
        // panels are dealt back and forth, so a group of G CTAs wants at least 2G panels
        const int cap = sweep_max_ctas<T>(NB);
        int G = choose_group(nb, max_m * 16 / NB, [&](int) { return cap; });
        // the autotuner's group scale for this launch shape (or the candidate being timed)
        const double gs = g_trial.sweep_gscale >= 0.0 ? g_trial.sweep_gscale : tune_get(skey + ".gscale", 1.0);
        if (G > 1 && gs > 0.0 && gs < 1.0) G = std::max(1, (int)std::lround(G * gs));
        double work = 0.0;
        for (int b = 0; b < nb; ++b) work += (double)sizes[b] * (double)sizes[b] * (double)sizes[b];
        // matrices of one launch differ in size: CTAs in proportion to m^3, at most m / 16 each
        std::vector<int32_t> cta_off;
        DevMem& d_cta = op->t_cta;
        if (G > 1 && nb > 1) {
            std::vector<double> wgt(nb);
            std::vector<int> capb(nb);
            for (int b = 0; b < nb; ++b) {
                wgt[b] = (double)sizes[b] * (double)sizes[b] * (double)sizes[b];
                capb[b] = std::max(1, (int)(sizes[b] / (2 * NB)));
            }
            cta_off = proportional_groups(nb * G, wgt, capb);
            if ((rc = upload(d_cta, cta_off, st))) return rc;
        }
        if (op->opts.per_box) {             // one matrix per launch, each with the whole GPU
            ProfScope ps(op, cls, st, work, 2.0 * sizeof(T) * (double)size_off[nb], level);
            for (int b = 0; b < nb; ++b) {
                const int mb = (int)sizes[b];
                if (mb <= 0) continue;
                const int Gb = choose_group(1, mb * 16 / NB, [&](int) { return cap; });
                RS_CUDA(launch_sweep_inverse<T>(st, 1, Gb, nullptr, Gb, dm.as<int32_t>() + b, doff.as<int64_t>() + b,
                                                A, op->d_pb.as<T>(), d_pboff.as<int64_t>() + b,
                                                op->d_bar.as<unsigned int>() + b, op->d_status.as<int>(),
                                                (long long)op->opts.spin_limit, mb, NB));
            }
        } else {
            ProfScope ps(op, cls, st, work, 2.0 * sizeof(T) * (double)size_off[nb], level);
            RS_CUDA(launch_sweep_inverse<T>(st, nb, G, cta_off.empty() ? nullptr : d_cta.as<int32_t>(),
                                            cta_off.empty() ? nb * G : cta_off[nb], dm.as<int32_t>(),
                                            doff.as<int64_t>(), A, op->d_pb.as<T>(), d_pboff.as<int64_t>(),
                                            op->d_bar.as<unsigned int>(), op->d_status.as<int>(),
                                            (long long)op->opts.spin_limit, max_m, NB));
        }
        if (op->defer_spd) return RS_OK;
        RS_CUDA(cudaStreamSynchronize(st));
        prof_flush(op);
        int s = 0;
        RS_CUDA(cudaMemcpy(&s, op->d_status.p, sizeof(int), cudaMemcpyDeviceToHost));
        if (s & DEV_NOT_SPD) {
            RS_CUDA(cudaMemsetAsync(op->d_status.p, 0, sizeof(int), st));
            op->stats.spd_fallbacks += 1;
            *not_spd = true;
            return RS_OK;
        }
        return check_status(op, st);
    }
}

// Whether the inverses of this operator go through the symmetric sweep first.
bool use_sweep(const rs_op* op) { return op->kind == RS_LAPLACE && op->opts.spd_inverse != 0; }

// ID phase of one level (Sec. 2.2 proxy ID, Eq. 2.1).
// The ID phase of one level whose index sets (L.m, act, nn, nearv and their offsets) are
// filled: Y assembly with kernel K and proxy circles geo (centre x, y, radius per box),
// column-pivoted QR, skeleton bookkeeping and T.
template <class T>
int id_core(rs_op* op, Level& L, IdWork& w, cudaStream_t st, const KernelK& K, const std::vector<double>& geo)
{
    const int P = op->opts.proxy_points;
    int rc;
    const int nb = L.nb;
    L.r.resize(nb);
    std::vector<int64_t> y_off(nb + 1, 0);
    int64_t max_entries = 0;
    L.max_m = L.max_r = 0;
    for (int b = 0; b < nb; ++b) {
        L.r[b] = L.nn[b] + P;
        y_off[b + 1] = y_off[b] + L.r[b] * L.m[b];
        max_entries = std::max(max_entries, L.r[b] * L.m[b]);
        L.max_m = std::max<int>(L.max_m, (int)L.m[b]);
        L.max_r = std::max<int>(L.max_r, (int)L.r[b]);
    }
    if (max_entries > (int64_t)INT32_MAX) return fail(RS_E_INVALID, "box too large");
    if ((rc = upload(L.d_act, to32(L.act), st))) return rc;
    if ((rc = upload(L.d_act_off, L.act_off, st))) return rc;
    if ((rc = upload(L.d_m, to32(L.m), st))) return rc;
    if ((rc = upload(w.near, to32(L.nearv), st))) return rc;
    if ((rc = upload(w.near_off, L.near_off, st))) return rc;
    if ((rc = upload(w.geo, geo, st))) return rc;
    if ((rc = upload(w.y_off, y_off, st))) return rc;
    if ((rc = upload(w.nn, to32(L.nn), st))) return rc;
    RS_CUDA(w.Y.alloc(sizeof(T) * (size_t)(y_off[nb] + 1)));
    {
    ProfScope ps(op, RS_PROF_ASSEMBLE_Y, st, (double)y_off[nb], sizeof(T) * (double)y_off[nb]);
    const bool pb = op->opts.per_box != 0;
    for (int b0 = 0; b0 < nb; b0 += pb ? 1 : nb) {
        const int cnt = pb ? 1 : nb;
        RS_CUDA(launch_assemble_Y<T>(st, cnt, L.d_act.as<int32_t>(), L.d_act_off.as<int64_t>() + b0,
                                     w.near.as<int32_t>(), w.near_off.as<int64_t>() + b0, w.geo.as<double>() + 3 * b0,
                                     op->d_ucirc.as<double>(), P, w.y_off.as<int64_t>() + b0, w.Y.as<T>(), K,
                                     pb ? (int)(L.r[b0] * L.m[b0]) : (int)max_entries));
    }
    }
    const int64_t sum_m = L.act_off[nb];
    RS_CUDA(w.piv.alloc(sizeof(int32_t) * (sum_m + 1)));
    RS_CUDA(w.diag.alloc(sizeof(T) * (sum_m + 1)));
    RS_CUDA(L.d_k.alloc(sizeof(int32_t) * nb));
    RS_CUDA(op->d_bar.alloc(sizeof(unsigned int) * nb));
    RS_CUDA(cudaMemsetAsync(op->d_bar.p, 0, sizeof(unsigned int) * nb, st));
    // The autotuner's settings for this level (or the candidate being timed).  With a batch
    // budget, boxes whose Y fit together in that many 96 MB units go to one launch each, and
    // each launch takes the whole GPU: the passes of a step then stream from L2 rather than
    // HBM (all boxes of a big level at once spill L2 and re-read every trailing matrix from HBM
    // at every step), at the price of fewer CTAs per box.  Untuned: one launch per level.
    const std::string tkey = tune_key("cpqr", (int)sizeof(T), nb, L.max_m, L.max_r);
    const double gs = g_trial.cpqr_gscale >= 0.0 ? g_trial.cpqr_gscale : tune_get(tkey + ".gscale", 1.0);
    int deep_set = g_trial.cpqr_deep >= 0         ? g_trial.cpqr_deep
                   : op->opts.cpqr_variant >= 0 ? op->opts.cpqr_variant
                                                : (int)tune_get(tkey + ".deep", -1.0);
    // the blocked forms (7, 8) take real scalars and boxes whose lists fit shared memory
    if ((deep_set == 7 || deep_set == 8) && !cpqr_bl_fits<T>(L.max_r, L.max_m)) deep_set = -1;
    const double batch_bytes =
        96.0 * (1 << 20) * (g_trial.cpqr_batch >= 0.0 ? g_trial.cpqr_batch : tune_get(tkey + ".batch", 0.0));
    std::vector<int> b_start(1, 0);
    if (op->opts.per_box) {
        for (int b = 1; b < nb; ++b) b_start.push_back(b);
    } else if (batch_bytes > 0.0) {
        double tot = 0.0;
        for (int b = 0; b < nb; ++b) tot += (double)sizeof(T) * (double)L.r[b] * (double)L.m[b];
        const int nbat = std::max(1, std::min(nb, (int)std::ceil(tot / batch_bytes)));
        for (int q = 1; q < nbat; ++q) b_start.push_back((int)(((int64_t)q * nb) / nbat));
    }
    b_start.push_back(nb);
    const int nbat = (int)b_start.size() - 1;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    struct Batch {
        int b0, nb, G, ctas, deep, max_r, max_m, cl;
        size_t cta_pos;
    };
    std::vector<Batch> bats;
    std::vector<int32_t> cta_all;
    size_t max_keys = 1;
    for (int q = 0; q < nbat; ++q) {
        Batch B{};
        B.b0 = b_start[q];
        B.nb = b_start[q + 1] - b_start[q];
        for (int b = B.b0; b < B.b0 + B.nb; ++b) {
            B.max_r = std::max<int>(B.max_r, (int)L.r[b]);
            B.max_m = std::max<int>(B.max_m, (int)L.m[b]);
        }
        // variant 4: boxes that fit the shared memory of one cluster stay there for the whole
        // factorization (when asked for, or picked by the autotuner)
        B.cl = 0;
        if (!op->opts.per_box && deep_set == 4) B.cl = cpqr_cl_cluster<T>(B.max_r, B.max_m);
        if (B.cl > 0) {
            B.G = 1;
            B.ctas = B.nb * B.cl;
            B.deep = 4;
            B.cta_pos = (size_t)-1;
            bats.push_back(B);
            continue;
        }
        // the open columns are re-split every step, so a group may take one CTA per 16 columns
        // (sized for the co-residency of the variant when one is set)
        const bool streaming = deep_set >= 0 && deep_set != 4;      // variants 0-3 and 5-8
        const int var = streaming ? deep_set : 0;
        int G = choose_group(B.nb, 2 * B.max_m, [&](int g) { return cpqr_max_ctas<T>(B.max_r, B.max_m, g, var); });
        if (G > 1 && gs > 0.0 && gs < 1.0) G = std::max(1, (int)std::lround(G * gs));
        // gs > 1 (large boxes, few per launch): more CTAs than one per 16 columns, so that more
        // warps -- and more loads in flight -- share each SM, within co-residency
        double cap_scale = 1.0;
        if (G > 1 && gs > 1.0) {
            const int capc = cpqr_max_ctas<T>(B.max_r, B.max_m, G, var);
            const int G2 = std::min((int)std::lround(G * gs), capc / std::max(B.nb, 1));
            if (G2 > G) {
                cap_scale = (double)G2 / (double)G;
                G = G2;
            }
        }
        B.G = G;
        // The boxes of a batch differ in work (boundary boxes have fewer near rows, ranks
        // differ), and a group runs at its own pace: deal the same CTA total in proportion to
        // each box's work, r m^2, so the groups finish together (at most one CTA per 16 columns).
        B.cta_pos = cta_all.size();
        if (G > 1 && B.nb > 1) {
            std::vector<double> wgt(B.nb);
            std::vector<int> cap(B.nb);
            for (int b = 0; b < B.nb; ++b) {
                wgt[b] = (double)L.r[B.b0 + b] * (double)L.m[B.b0 + b] * (double)L.m[B.b0 + b];
                cap[b] = std::max(1, (int)(cap_scale * (double)(2 * L.m[B.b0 + b] / 32)));
            }
            const std::vector<int32_t> off = proportional_groups(B.nb * G, wgt, cap);
            cta_all.insert(cta_all.end(), off.begin(), off.end());
            B.ctas = off[B.nb];
        } else {
            B.cta_pos = (size_t)-1;
            B.ctas = B.nb * G;
        }
        // few CTAs per SM: each warp keeps twice the rows in flight.  FP64 levels of many
        // small boxes (one or two CTAs each) take the blocked form with panels of 8 steps:
        // measured 9-19% faster there at 512^2, slower where a box spreads over more CTAs (its
        // two group barriers per step then wait on the slowest of them) and in FP32
        B.deep = (G > 1 && B.ctas <= 2 * sms) ? 1 : 0;
        if (std::is_same<T, double>::value && G <= 2 && B.max_r <= 704 && cpqr_bl_fits<T>(B.max_r, B.max_m)) B.deep = 8;
        if (streaming) B.deep = deep_set;
        // a group of several CTAs must stay co-resident
        if (B.deep && (G > 1 || B.cta_pos != (size_t)-1) && B.ctas > cpqr_max_ctas<T>(B.max_r, B.max_m, G, B.deep))
            B.deep = 0;
        max_keys = std::max(max_keys, (size_t)(2 * B.ctas));
        bats.push_back(B);
    }
    if (!cta_all.empty()) {
        int rc2;
        if ((rc2 = upload(w.cta_off, cta_all, st))) return rc2;
    }
    RS_CUDA(w.keys.alloc(sizeof(unsigned long long) * max_keys));
    size_t gw_ints = 0;        // open-column lists in global memory (boxes too large for shared)
    for (const Batch& B : bats)
        if (!B.cl) gw_ints = std::max(gw_ints, cpqr_gwork_ints<T>(B.max_r, B.max_m, B.deep, B.ctas));
    if (gw_ints) RS_CUDA(w.gwork.alloc(sizeof(int) * gw_ints));
    size_t bl_bytes = 0;       // V, F and group partials of the blocked forms
    for (const Batch& B : bats)
        if (!B.cl && (B.deep == 7 || B.deep == 8))
            bl_bytes = std::max(bl_bytes, cpqr_bl_bytes<T>(B.nb, B.max_r, sum_m, B.ctas, B.deep == 7 ? 16 : 8));
    if (bl_bytes) RS_CUDA(w.blk.alloc(bl_bytes));
    // squared norms, their references, and (look-ahead variant) the dot products v^H y_j
    const size_t nrm_dbl = 2 * (size_t)(sum_m + 1), wv_dbl = ((size_t)(sum_m + 1) * sizeof(T) + 7) / 8;
    RS_CUDA(w.norms.alloc(sizeof(double) * (nrm_dbl + wv_dbl)));
    {
        // the rank is known only afterwards: the work is added once k is read back
        ProfScope ps(op, RS_PROF_CPQR, st, 0.0, 0.0, L.l);
        for (const Batch& B : bats) {
            if (B.cl) {
                RS_CUDA(launch_cpqr_cl<T>(st, B.nb, B.cl, L.d_act_off.as<int64_t>() + B.b0, w.nn.as<int32_t>() + B.b0, P,
                                          w.y_off.as<int64_t>() + B.b0, w.Y.as<T>(), op->eps,
                                          L.d_k.as<int32_t>() + B.b0, w.piv.as<int32_t>(), w.diag.as<T>(),
                                          op->d_status.as<int>(), B.max_r, B.max_m));
                continue;
            }
            if (B.deep == 7 || B.deep == 8) {
                RS_CUDA(launch_cpqr_bl<T>(st, B.nb, B.G,
                                          B.cta_pos == (size_t)-1 ? nullptr : w.cta_off.as<int32_t>() + B.cta_pos,
                                          B.ctas, B.deep == 7 ? 16 : 8, L.d_act_off.as<int64_t>() + B.b0,
                                          w.nn.as<int32_t>() + B.b0, P, w.y_off.as<int64_t>() + B.b0, w.Y.as<T>(),
                                          op->eps, L.d_k.as<int32_t>() + B.b0, w.piv.as<int32_t>(), w.diag.as<T>(),
                                          op->d_bar.as<unsigned int>() + B.b0, w.keys.as<unsigned long long>(),
                                          op->d_status.as<int>(), (long long)op->opts.spin_limit, B.max_r, B.max_m,
                                          sum_m, w.norms.as<double>(), w.norms.as<double>() + sum_m + 1, w.blk.p));
                continue;
            }
            RS_CUDA(launch_cpqr<T>(st, B.nb, B.G,
                                   B.cta_pos == (size_t)-1 ? nullptr : w.cta_off.as<int32_t>() + B.cta_pos, B.ctas,
                                   B.deep, L.d_act_off.as<int64_t>() + B.b0, w.nn.as<int32_t>() + B.b0, P,
                                   w.y_off.as<int64_t>() + B.b0, w.Y.as<T>(), op->eps, L.d_k.as<int32_t>() + B.b0,
                                   w.piv.as<int32_t>(), w.diag.as<T>(), op->d_bar.as<unsigned int>() + B.b0,
                                   w.keys.as<unsigned long long>(), op->d_status.as<int>(),
                                   (long long)op->opts.spin_limit, B.max_r, B.max_m, w.norms.as<double>(),
                                   w.norms.as<double>() + sum_m + 1, (T*)(w.norms.as<double>() + nrm_dbl),
                                   gw_ints ? w.gwork.as<int>() : nullptr));
        }
    }
    if ((rc = check_status(op, st))) return rc;
    std::vector<int32_t> k32(nb), piv(sum_m);
    RS_CUDA(cudaMemcpy(k32.data(), L.d_k.p, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost));
    RS_CUDA(cudaMemcpy(piv.data(), w.piv.p, sizeof(int32_t) * sum_m, cudaMemcpyDeviceToHost));
    // skeleton ascending in grid index, residual ascending in local index
    L.k.assign(nb, 0);
    L.k_off.assign(nb + 1, 0);
    L.perm.assign(sum_m, 0);
    L.skel.clear();
    std::vector<int32_t> skpos(sum_m, 0), rscol(sum_m, 0);
    L.t_off.assign(nb + 1, 0);
    L.max_k = 0;
    int max_res = 0;
    for (int b = 0; b < nb; ++b) {
        const int64_t a0 = L.act_off[b];
        const int m = (int)L.m[b], k = k32[b];
        if (k < 0 || k > m) return fail(RS_E_CUDA, "bad rank from the ID kernel");
        L.k[b] = k;
        L.k_off[b + 1] = L.k_off[b] + k;
        std::vector<int> order(k);
        for (int a = 0; a < k; ++a) order[a] = a;
        std::sort(order.begin(), order.end(),
                  [&](int x, int y) { return L.act[a0 + piv[a0 + x]] < L.act[a0 + piv[a0 + y]]; });
        std::vector<char> is_sk(m, 0);
        for (int q = 0; q < k; ++q) {
            const int a = order[q];
            const int loc = piv[a0 + a];
            if (loc < 0 || loc >= m || is_sk[loc]) return fail(RS_E_CUDA, "bad pivot from the ID kernel");
            is_sk[loc] = 1;
            skpos[a0 + a] = q;
            L.perm[a0 + q] = loc;
            L.skel.push_back(L.act[a0 + loc]);
        }
        int c = 0;
        for (int loc = 0; loc < m; ++loc)
            if (!is_sk[loc]) { rscol[a0 + c] = loc; L.perm[a0 + k + c] = loc; ++c; }
        L.t_off[b + 1] = L.t_off[b] + (int64_t)k * (m - k);
        L.max_k = std::max(L.max_k, k);
        max_res = std::max(max_res, m - k);
    }
    double cpqr_work = 0.0, t_work = 0.0;
    for (int b = 0; b < nb; ++b) {
        const double m = (double)L.m[b], k = (double)L.k[b], r = (double)L.r[b];
        cpqr_work += 4.0 * r * m * k - 2.0 * k * k * (r + m) + 4.0 * k * k * k / 3.0;
        t_work += k * k * (m - k);
    }
    op->prof_work[RS_PROF_CPQR] += op->opts.profile ? cpqr_work : 0.0;
    if ((rc = upload(L.d_perm, L.perm, st))) return rc;
    if ((rc = upload(w.skpos, skpos, st))) return rc;
    if ((rc = upload(w.rscol, rscol, st))) return rc;
    if ((rc = upload(L.d_t_off, L.t_off, st))) return rc;
    if ((rc = upload(L.d_k_off, L.k_off, st))) return rc;
    RS_CUDA(L.d_T.alloc(sizeof(T) * (size_t)(L.t_off[nb] + 1)));
    {
    ProfScope ps(op, RS_PROF_ID_T, st, t_work, sizeof(T) * (double)L.t_off[nb]);
    const bool pb = op->opts.per_box != 0;
    if constexpr (std::is_same<T, double>::value) {
        if (!pb && op->opts.gemm_form == 1) {
            // blocks of 64 rows of R11, the updates on the digit-slice GEMM
            std::vector<int64_t> rgoff;
            std::vector<std::vector<GemmProb>> gs;
            const size_t rgn = idt_bl_plan(nb, L.m, L.k, L.max_k, rgoff, gs);
            std::vector<GemmProb> ag;
            std::vector<int64_t> eg;
            struct StepI { size_t pg, eg; OzPlan pl; int n; };
            std::vector<StepI> si(gs.size());
            int64_t max_lines = 1, max_digits = 1, max_km = 0, max_kres = 0;
            for (size_t q = 0; q < gs.size(); ++q) {
                std::vector<int64_t> eo;
                si[q].pg = ag.size(); si[q].eg = eg.size(); si[q].n = (int)gs[q].size();
                si[q].pl = gemm_oz_plan(gs[q], eo);
                ag.insert(ag.end(), gs[q].begin(), gs[q].end());
                eg.insert(eg.end(), eo.begin(), eo.end());
                max_lines = std::max(max_lines, si[q].pl.lines);
                max_digits = std::max(max_digits, si[q].pl.digits);
            }
            for (int b = 0; b < nb; ++b) {
                max_km = std::max<int64_t>(max_km, L.k[b] * L.m[b]);
                max_kres = std::max<int64_t>(max_kres, L.k[b] * (L.m[b] - L.k[b]));
            }
            if ((rc = upload(op->t_idrg, rgoff, st))) return rc;
            if ((rc = upload(op->t_idg, ag, st))) return rc;
            if ((rc = upload(op->t_ide, eg, st))) return rc;
            RS_CUDA(op->t_idR.alloc(sizeof(double) * (rgn + 1)));
            RS_CUDA(op->t_ozx.alloc(sizeof(int) * (size_t)max_lines));
            RS_CUDA(op->t_ozd.alloc(2 * (size_t)(max_digits + 8)));
            RS_CUDA(launch_idt_gather(st, nb, max_km, L.d_act_off.as<int64_t>(), L.d_k.as<int32_t>(), w.nn.as<int32_t>(),
                                      P, w.y_off.as<int64_t>(), w.Y.as<double>(), w.piv.as<int32_t>(),
                                      w.diag.as<double>(), w.rscol.as<int32_t>(), op->t_idrg.as<int64_t>(),
                                      op->t_idR.as<double>()));
            for (size_t q = 0; q < gs.size(); ++q) {
                RS_CUDA(launch_idt_solve(st, nb, (int)q, max_res, L.d_act_off.as<int64_t>(), L.d_k.as<int32_t>(),
                                         op->t_idrg.as<int64_t>(), op->t_idR.as<double>()));
                if (si[q].n > 0)
                    RS_CUDA(launch_gemm_oz(st, op->t_idg.as<GemmProb>() + si[q].pg, si[q].n, si[q].pl,
                                           op->t_ide.as<int64_t>() + si[q].eg, op->t_ozx.as<int>(), op->t_ozd.p,
                                           op->t_idR.as<double>(), op->t_idR.as<double>(), op->t_idR.as<double>(),
                                           op->t_idR.as<double>()));
            }
            RS_CUDA(launch_idt_scatter(st, nb, max_kres, L.d_act_off.as<int64_t>(), L.d_k.as<int32_t>(),
                                       w.skpos.as<int32_t>(), op->t_idrg.as<int64_t>(), op->t_idR.as<double>(),
                                       L.d_t_off.as<int64_t>(), L.d_T.as<double>()));
        }
    }
    const bool idt_bl = std::is_same<T, double>::value && !pb && op->opts.gemm_form == 1;
    for (int b0 = 0; !idt_bl && b0 < nb; b0 += pb ? 1 : nb) {
        const int cnt = pb ? 1 : nb;
        RS_CUDA(launch_id_T<T>(st, cnt, L.d_act_off.as<int64_t>() + b0, L.d_k.as<int32_t>() + b0,
                               w.nn.as<int32_t>() + b0, P, w.y_off.as<int64_t>() + b0, w.Y.as<T>(),
                               w.piv.as<int32_t>(), w.diag.as<T>(), w.skpos.as<int32_t>(), w.rscol.as<int32_t>(),
                               L.d_t_off.as<int64_t>() + b0, L.d_T.as<T>(),
                               pb ? (int)(L.m[b0] - L.k[b0]) : max_res, pb ? (int)L.k[b0] : L.max_k));
    }
    }
    // no synchronisation: the next level's CPQR status check covers this launch too
    RS_CUDA(cudaGetLastError());
    return RS_OK;
}

// Proxy circle of every box of level L (centre x, y and radius; Sec. 2.2).
std::vector<double> box_geo(const rs_op* op, const Level& L)
{
    std::vector<double> geo(3 * (size_t)L.nb);
    const double hh = 0.5 * op->K.h;
    for (int b = 0; b < L.nb; ++b) {
        const BoxInt bi = box_int(op->n, L.l, b);
        geo[3 * b] = (double)((2 * bi.bx + 1) * bi.wx) * hh;
        geo[3 * b + 1] = (double)((2 * bi.by + 1) * bi.wy) * hh;
        geo[3 * b + 2] = (op->opts.proxy_radius_factor * (double)std::max(bi.wx, bi.wy)) * hh;
    }
    return geo;
}

// Translation-invariant modes (a and b constant, so A depends only on the offset between grid
// points; Sec. 5, one set of matrix blocks per level).  The level's ID phase runs on a few
// "factored" boxes, and every box of the level takes the rank, skeleton positions and T of
// its class (L.ti_cls, representatives L.ti_rep).
//   Mode 1 (the paper's one set per level): one template, box 0 with all eight same-level
//     neighbours present -- translates of its active set in the order (dy, dx) = (-1,-1),
//     (-1,0), (-1,1), (0,-1), (0,1), (1,-1), (1,0), (1,1), also where they fall outside the
//     unit square, their points strictly inside the proxy circle as near rows.  Every box's
//     real near rows are rows of this Y (translated) and its proxy rows the same, so the
//     skeleton positions and T serve all boxes.  The template lives on an extended lattice of
//     side 3n, box 0 shifted by (n, n): the entries depend only on offsets, so the grid kernels
//     evaluate it unchanged (no offset table; the Helmholtz scaling is the constant s0).
//   Mode 2 (the per-box factorization without its repeats): boxes whose active points, near
//     points and children's classes are translates of one another have translated Y and F,
//     hence the same ID, F^{-1} and E; one box per class is factored (with its real rows).
template <class T>
int id_level_ti(rs_op* op, Level& L, const Level* child, IdWork& w, cudaStream_t st)
{
    const int64_t n = op->n;
    const int nb = L.nb;
    Level& TL = op->ti_lev[L.l];
    TL.l = L.l;
    std::vector<double> geo;
    KernelK K = op->K;
    if (op->opts.translation_invariant == 1) {
        const int64_t ne = 3 * n;
        const int64_t m = L.m[0];
        const BoxInt bi = box_int(n, L.l, 0);
        L.ti_cls.assign(nb, 0);
        L.ti_rep = {0};
        TL.nb = 1;
        TL.m = {m};
        TL.act.resize(m);
        for (int64_t p = 0; p < m; ++p) {
            const int64_t g = L.act[p];
            TL.act[p] = (g % n + n) + ne * (g / n + n);
        }
        TL.act_off = {0, m};
        const int64_t cx2 = (2 * bi.bx + 1) * bi.wx, cy2 = (2 * bi.by + 1) * bi.wy;     // units of h/2
        const double R2 = op->opts.proxy_radius_factor * (double)std::max(bi.wx, bi.wy);
        TL.nearv.clear();
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                if (ox == 0 && oy == 0) continue;
                for (int64_t p = 0; p < m; ++p) {
                    const int64_t i1 = L.act[p] % n + ox * bi.wx, i2 = L.act[p] / n + oy * bi.wy;
                    const int64_t dx = 2 * i1 + 1 - cx2, dy = 2 * i2 + 1 - cy2;
                    if (!((double)(dx * dx + dy * dy) < R2 * R2)) continue;
                    TL.nearv.push_back((i1 + n) + ne * (i2 + n));
                }
            }
        TL.nn = {(int64_t)TL.nearv.size()};
        TL.near_off = {0, (int64_t)TL.nearv.size()};
        geo = box_geo(op, TL);
        geo[0] += (double)n * op->K.h;
        geo[1] += (double)n * op->K.h;
        K.n = (int)ne;
        K.tab = nullptr;
        K.s = nullptr;
        K.s0 = op->ti_s0;
    } else {
        // classes: the active and near points relative to the box's first active point, and
        // the children's classes (exact keys: equal keys mean translated Y and F)
        std::map<std::vector<int64_t>, int> key_of;
        L.ti_cls.assign(nb, 0);
        L.ti_rep.clear();
        std::vector<int64_t> key;
        for (int b = 0; b < nb; ++b) {
            const int64_t a0 = L.act_off[b], a1 = L.act_off[b + 1], g0 = L.act[a0];
            key.clear();
            key.push_back(a1 - a0);
            key.push_back(L.near_off[b + 1] - L.near_off[b]);
            if (child) {
                key.push_back(child->ti_cls[2 * b]);
                key.push_back(child->ti_cls[2 * b + 1]);
            }
            for (int64_t p = a0; p < a1; ++p) key.push_back(L.act[p] - g0);
            for (int64_t q = L.near_off[b]; q < L.near_off[b + 1]; ++q) key.push_back(L.nearv[q] - g0);
            auto it = key_of.find(key);
            if (it == key_of.end()) {
                it = key_of.emplace(key, (int)L.ti_rep.size()).first;
                L.ti_rep.push_back(b);
            }
            L.ti_cls[b] = it->second;
        }
        const int nc = (int)L.ti_rep.size();
        TL.nb = nc;
        TL.m.resize(nc);
        TL.nn.resize(nc);
        TL.act_off.assign(nc + 1, 0);
        TL.near_off.assign(nc + 1, 0);
        TL.act.clear();
        TL.nearv.clear();
        const std::vector<double> g_all = box_geo(op, L);
        geo.resize(3 * (size_t)nc);
        for (int c = 0; c < nc; ++c) {
            const int b = L.ti_rep[c];
            TL.m[c] = L.m[b];
            TL.nn[c] = L.nn[b];
            TL.act.insert(TL.act.end(), L.act.begin() + L.act_off[b], L.act.begin() + L.act_off[b + 1]);
            TL.nearv.insert(TL.nearv.end(), L.nearv.begin() + L.near_off[b], L.nearv.begin() + L.near_off[b + 1]);
            TL.act_off[c + 1] = (int64_t)TL.act.size();
            TL.near_off[c + 1] = (int64_t)TL.nearv.size();
            for (int q = 0; q < 3; ++q) geo[3 * c + q] = g_all[3 * b + q];
        }
    }
    int rc = id_core<T>(op, TL, w, st, K, geo);
    if (rc) return rc;
    // every box: its class's rank, skeleton positions and T
    L.r.resize(nb);
    L.k.resize(nb);
    L.k_off.assign(nb + 1, 0);
    L.t_off.assign(nb + 1, 0);
    for (int b = 0; b < nb; ++b) {
        const int c = L.ti_cls[b];
        L.r[b] = TL.r[c];
        if (op->opts.translation_invariant == 1) L.nn[b] = TL.nn[c];
        L.k[b] = TL.k[c];
        L.k_off[b + 1] = L.k_off[b] + L.k[b];
        L.t_off[b] = TL.t_off[c];
    }
    L.t_off[nb] = TL.t_off[TL.nb];
    L.perm.resize(L.act.size());
    L.skel.resize(L.k_off[nb]);
    for (int b = 0; b < nb; ++b) {
        const int c = L.ti_cls[b];
        const int64_t a0 = L.act_off[b], m = L.m[b], t0 = TL.act_off[c];
        if (m != TL.m[c]) return fail(RS_E_CUDA, "translation-invariant mode: boxes of a class differ in size");
        const int64_t sh = L.act[a0] - L.act[L.act_off[L.ti_rep[c]]];
        for (int64_t p = 0; p < m; ++p) {
            if (op->opts.translation_invariant == 2 && L.act[a0 + p] - TL.act[t0 + p] != sh)
                return fail(RS_E_CUDA, "translation-invariant mode: not a translate");
            L.perm[a0 + p] = TL.perm[t0 + p];
        }
        for (int64_t a = 0; a < L.k[b]; ++a) L.skel[L.k_off[b] + a] = L.act[a0 + TL.perm[t0 + a]];
    }
    L.max_m = TL.max_m;
    L.max_k = TL.max_k;
    L.max_r = TL.max_r;
    if ((rc = upload(L.d_act, to32(L.act), st))) return rc;
    if ((rc = upload(L.d_act_off, L.act_off, st))) return rc;
    if ((rc = upload(L.d_m, to32(L.m), st))) return rc;
    if ((rc = upload(L.d_k, to32(L.k), st))) return rc;
    if ((rc = upload(L.d_perm, L.perm, st))) return rc;
    if ((rc = upload(L.d_k_off, L.k_off, st))) return rc;
    return upload(L.d_t_off, L.t_off, st);
}

template <class T>
int id_level(rs_op* op, Level& L, const Level* child, IdWork& w, cudaStream_t st)
{
    int rc = level_sets(op->n, op->d, L.l, child ? child->k.data() : nullptr, child ? child->skel.data() : nullptr,
                        op->opts.proxy_radius_factor, L.m, L.act, L.act_off, L.nn, L.nearv, L.near_off);
    if (rc) return rc;
    if (op->opts.translation_invariant) return id_level_ti<T>(op, L, child, w, st);
    return id_core<T>(op, L, w, st, op->K, box_geo(op, L));
}

// What F assembly reads of the child level: per box b of the level being inverted, the rank
// and E offset of its children at 2b and 2b + 1, and the children's E storage.
struct ChildRef {
    const int32_t* k = nullptr;
    const int64_t* e_off = nullptr;
    const void* E = nullptr;
};

// Inversion phase of one level (Algorithm 1 with the E of Algorithm 2).
template <class T>
int inverse_level(rs_op* op, Level& L, const ChildRef& cref, cudaStream_t st)
{
    const int nb = L.nb;
    L.phi_off.assign(nb + 1, 0);
    L.e_off.assign(nb + 1, 0);
    L.w_off.assign(nb + 1, 0);
    for (int b = 0; b < nb; ++b) {
        L.phi_off[b + 1] = L.phi_off[b] + L.m[b] * L.m[b];
        L.e_off[b + 1] = L.e_off[b] + L.k[b] * L.k[b];
        L.w_off[b + 1] = L.w_off[b] + L.m[b] * L.k[b];
    }
    int rc;
    if ((rc = upload(L.d_phi_off, L.phi_off, st))) return rc;
    RS_CUDA(L.d_Phi.alloc(sizeof(T) * (size_t)(L.phi_off[nb] + 1)));
    const bool leaf = (L.l == op->d);
    auto assemble = [&]() -> int {
        ProfScope ps(op, RS_PROF_ASSEMBLE_F, st, (double)L.phi_off[nb], sizeof(T) * (double)L.phi_off[nb]);
        const bool pb = op->opts.per_box != 0;
        for (int b0 = 0; b0 < nb; b0 += pb ? 1 : nb) {
            RS_CUDA(launch_assemble_F<T>(st, pb ? 1 : nb, leaf, L.d_act.as<int32_t>(), L.d_act_off.as<int64_t>() + b0,
                                         L.d_perm.as<int32_t>(), op->d_a.as<double>(),
                                         L.d_phi_off.as<int64_t>() + b0, L.d_Phi.as<T>(),
                                         cref.k ? cref.k + 2 * b0 : nullptr,
                                         cref.e_off ? cref.e_off + 2 * b0 : nullptr,
                                         (const T*)cref.E, op->K,
                                         pb ? (int)L.m[b0] : L.max_m));
        }
        return RS_OK;
    };
    if ((rc = assemble())) return rc;
    const int cls_f = L.l == 0 ? RS_PROF_INV_ROOT : RS_PROF_INV_F;
    bool redo = true;
    if (use_sweep(op)) {
        if ((rc = run_sweep<T>(op, st, nb, L.d_m, L.d_phi_off, L.d_Phi.as<T>(), L.m, L.act_off, L.max_m, cls_f, L.l,
                               &redo, &L.phi_off)))
            return rc;
        if (redo && (rc = assemble())) return rc;
    }
    if (redo && (rc = run_gj<T>(op, st, nb, L.d_m, L.d_phi_off, L.d_Phi.as<T>(), L.m, L.act_off, L.max_m, cls_f, L.l)))
        return rc;
    if (L.l == 0) return RS_OK;
    // W = Phi[:, :k] + Phi[:, k:] T^T ;  E^{-1} = W[:k, :] + T W[k:, :]
    if ((rc = upload(L.d_e_off, L.e_off, st))) return rc;
    RS_CUDA(L.d_E.alloc(sizeof(T) * (size_t)(L.e_off[nb] + 1)));
    // scratch kept by the op across levels (freeing it would synchronise the device)
    DevMem& W = op->t_W;
    DevMem& d_p1 = op->t_p1;
    DevMem& d_p2 = op->t_p2;
    RS_CUDA(W.alloc(sizeof(T) * (size_t)(L.w_off[nb] + 1)));
    // with the symmetric sweep, E^{-1} (symmetric) is needed on and below the diagonal only:
    // p2l takes those tiles; p2 (all tiles) serves the Gauss-Jordan path and its fallback
    const bool sym = use_sweep(op);
    // FP64: the products from digit slices on the tensor cores (opts.gemm_form), batched launches
    const bool use_oz = std::is_same<T, double>::value && op->opts.gemm_form == 1 && !op->opts.per_box;
    auto run_oz = [&](std::vector<GemmProb> q, DevMem& dq, DevMem& de, const T* A, const T* B, T* C,
                      const T* C0) -> int {
        if constexpr (std::is_same<T, double>::value) {
            std::vector<int64_t> eo;
            const OzPlan pl = gemm_oz_plan(q, eo);
            int rc2;
            if ((rc2 = upload(dq, q, st))) return rc2;
            if ((rc2 = upload(de, eo, st))) return rc2;
            RS_CUDA(op->t_ozx.alloc(sizeof(int) * (size_t)(pl.lines + 1)));
            RS_CUDA(op->t_ozd.alloc(2 * (size_t)(pl.digits + 8)));
            RS_CUDA(launch_gemm_oz(st, dq.as<GemmProb>(), (int)q.size(), pl, de.as<int64_t>(), op->t_ozx.as<int>(),
                                   op->t_ozd.p, A, B, C, C0));
            return RS_OK;
        } else {
            (void)q; (void)dq; (void)de; (void)A; (void)B; (void)C; (void)C0;
            return fail(RS_E_INVALID, "digit-product GEMM for FP64 only");
        }
    };
    std::vector<GemmProb> p1, p2, p2l;
    int64_t t1 = 0, t2 = 0, t2l = 0;
    for (int b = 0; b < nb; ++b) {
        const int m = (int)L.m[b], k = (int)L.k[b];
        if (k == 0) continue;
        GemmProb g{};
        g.M = m; g.N = k; g.K = m - k; g.ta = 0; g.tb = 1;
        g.lda = m; g.ldb = std::max(k, 1); g.ldc = m; g.ldc0 = m;
        g.a_off = L.phi_off[b] + (int64_t)k * m; g.b_off = L.t_off[b]; g.c_off = L.w_off[b]; g.c0_off = L.phi_off[b];
        g.alpha = 1.0; g.beta = 1.0;
        g.tiles_m = (m + 63) / 64; g.tiles_n = (k + 63) / 64; g.tile0 = t1;
        t1 += (int64_t)g.tiles_m * g.tiles_n;
        p1.push_back(g);
        GemmProb h{};
        h.M = k; h.N = k; h.K = m - k; h.ta = 0; h.tb = 0;
        h.lda = std::max(k, 1); h.ldb = m; h.ldc = k; h.ldc0 = m;
        h.a_off = L.t_off[b]; h.b_off = L.w_off[b] + k; h.c_off = L.e_off[b]; h.c0_off = L.w_off[b];
        h.alpha = 1.0; h.beta = 1.0;
        h.tiles_m = (k + 63) / 64; h.tiles_n = (k + 63) / 64; h.tile0 = t2;
        t2 += (int64_t)h.tiles_m * h.tiles_n;
        p2.push_back(h);
        GemmProb hl = h;
        hl.lower = 1;
        hl.tile0 = t2l;
        t2l += (int64_t)h.tiles_m * (h.tiles_m + 1) / 2;
        p2l.push_back(hl);
    }
    if (!p1.empty()) {
        if ((rc = upload(d_p1, p1, st))) return rc;
        if ((rc = upload(d_p2, sym ? p2l : p2, st))) return rc;
        double work = 0.0;
        for (int b = 0; b < nb; ++b) {
            const double m = (double)L.m[b], k = (double)L.k[b];
            work += 2.0 * m * (m - k) * k + (sym ? k * (k + 1.0) * (m - k) : 2.0 * k * (m - k) * k);
        }
        ProfScope ps(op, RS_PROF_GEMM_E, st, work,
                     sizeof(T) * (double)(L.phi_off[nb] + 2 * L.w_off[nb] + L.e_off[nb]));
        if (op->opts.per_box) {             // one box per launch: descriptors starting at tile 0
            std::vector<GemmProb> q1 = p1, q2 = sym ? p2l : p2;
            for (auto& g : q1) g.tile0 = 0;
            for (auto& g : q2) g.tile0 = 0;
            if ((rc = upload(op->t_q1, q1, st))) return rc;
            if ((rc = upload(op->t_q2, q2, st))) return rc;
            for (size_t i = 0; i < q1.size(); ++i) {
                const int64_t n2 = q2[i].lower ? (int64_t)q2[i].tiles_m * (q2[i].tiles_m + 1) / 2
                                               : (int64_t)q2[i].tiles_m * q2[i].tiles_n;
                RS_CUDA(launch_gemm<T>(st, op->t_q1.as<GemmProb>() + i, 1, (int64_t)q1[i].tiles_m * q1[i].tiles_n,
                                       L.d_Phi.as<T>(), L.d_T.as<T>(), W.as<T>(), L.d_Phi.as<T>()));
                RS_CUDA(launch_gemm<T>(st, op->t_q2.as<GemmProb>() + i, 1, n2, L.d_T.as<T>(), W.as<T>(),
                                       L.d_E.as<T>(), W.as<T>()));
            }
        } else if (use_oz) {
            if ((rc = run_oz(p1, op->t_oz1, op->t_ozo1, L.d_Phi.as<T>(), L.d_T.as<T>(), W.as<T>(), L.d_Phi.as<T>())))
                return rc;
            if ((rc = run_oz(sym ? p2l : p2, op->t_oz2, op->t_ozo2, L.d_T.as<T>(), W.as<T>(), L.d_E.as<T>(), W.as<T>())))
                return rc;
        } else {
            RS_CUDA(launch_gemm<T>(st, d_p1.as<GemmProb>(), (int)p1.size(), t1, L.d_Phi.as<T>(), L.d_T.as<T>(),
                                   W.as<T>(), L.d_Phi.as<T>()));
            RS_CUDA(launch_gemm<T>(st, d_p2.as<GemmProb>(), (int)p2.size(), sym ? t2l : t2, L.d_T.as<T>(), W.as<T>(),
                                   L.d_E.as<T>(), W.as<T>()));
        }
    }
    DevMem& d_k32 = op->t_k32;
    if ((rc = upload(d_k32, to32(L.k), st))) return rc;
    redo = true;
    if (use_sweep(op)) {
        if ((rc = run_sweep<T>(op, st, nb, d_k32, L.d_e_off, L.d_E.as<T>(), L.k, L.k_off, L.max_k, RS_PROF_INV_E,
                               L.l, &redo, &L.e_off)))
            return rc;
        if (redo && !p1.empty()) {   // E^{-1} again from W, all tiles (the sweep overwrote it)
            if (use_oz) {
                if ((rc = run_oz(p2, op->t_oz2, op->t_ozo2, L.d_T.as<T>(), W.as<T>(), L.d_E.as<T>(), W.as<T>())))
                    return rc;
            } else {
                if ((rc = upload(d_p2, p2, st))) return rc;
                RS_CUDA(launch_gemm<T>(st, d_p2.as<GemmProb>(), (int)p2.size(), t2, L.d_T.as<T>(), W.as<T>(),
                                       L.d_E.as<T>(), W.as<T>()));
            }
        }
    }
    if (!redo) return RS_OK;
    return run_gj<T>(op, st, nb, d_k32, L.d_e_off, L.d_E.as<T>(), L.k, L.k_off, L.max_k, RS_PROF_INV_E, L.l);
}

ChildRef child_ref(const Level* child)
{
    ChildRef c;
    if (child) {
        c.k = child->d_k.as<int32_t>();
        c.e_off = child->d_e_off.as<int64_t>();
        c.E = child->d_E.p;
    }
    return c;
}

template <class T>
int inverse_level(rs_op* op, Level& L, const Level* child, cudaStream_t st)
{
    return inverse_level<T>(op, L, child_ref(child), st);
}

// Translation-invariant modes: the inversion phase on the level's factored boxes (the
// template, or one box per class), each F assembled from its representative's own active
// points and children; then every box takes its class's F^{-1}, E and T offsets.
template <class T>
int inverse_level_ti(rs_op* op, int l, cudaStream_t st)
{
    Level& L = op->lev[l];
    Level& TL = op->ti_lev[l];
    const int nb = L.nb, nc = TL.nb;
    int rc;
    if (op->opts.translation_invariant == 1) {      // the template's Y was on the extended lattice
        TL.act.assign(L.act.begin(), L.act.begin() + TL.m[0]);
        if ((rc = upload(TL.d_act, to32(TL.act), st))) return rc;
    }
    ChildRef cref;
    if (l < op->d) {
        const Level& C = op->lev[l + 1];
        std::vector<int32_t> ck(2 * (size_t)nc);
        std::vector<int64_t> ce(2 * (size_t)nc);
        for (int c = 0; c < nc; ++c)
            for (int i = 0; i < 2; ++i) {
                const int cb = 2 * L.ti_rep[c] + i;
                ck[2 * c + i] = (int32_t)C.k[cb];
                ce[2 * c + i] = C.e_off[cb];
            }
        if ((rc = upload(op->t_ck, ck, st))) return rc;
        if ((rc = upload(op->t_ce, ce, st))) return rc;
        cref.k = op->t_ck.as<int32_t>();
        cref.e_off = op->t_ce.as<int64_t>();
        cref.E = C.d_E.p;
    }
    if ((rc = inverse_level<T>(op, TL, cref, st))) return rc;
    L.phi_off.assign(nb + 1, 0);
    L.e_off.assign(nb + 1, 0);
    L.w_off.assign(nb + 1, 0);
    for (int b = 0; b < nb; ++b) {
        L.phi_off[b] = TL.phi_off[L.ti_cls[b]];
        L.e_off[b] = TL.e_off[L.ti_cls[b]];
        L.w_off[b] = TL.w_off[L.ti_cls[b]];
    }
    L.phi_off[nb] = TL.phi_off[nc];
    L.e_off[nb] = TL.e_off[nc];
    L.w_off[nb] = TL.w_off[nc];
    L.d_Phi = std::move(TL.d_Phi);
    L.d_E = std::move(TL.d_E);
    L.d_T = std::move(TL.d_T);
    if ((rc = upload(L.d_phi_off, L.phi_off, st))) return rc;
    return upload(L.d_e_off, L.e_off, st);
}

void add_mv(std::vector<MatvecProb>& v, std::vector<int64_t>& blk, int64_t& nblk, int rows, int cols, int ld, int trans,
            int64_t a_off, int64_t x_off, int64_t y_off, double alpha, double beta)
{
    const int out_n = trans ? cols : rows;
    if (out_n <= 0) return;      // an empty inner dimension still writes beta * y (zeros)
    MatvecProb p{};
    p.rows = rows; p.cols = cols; p.ld = std::max(ld, 1); p.trans = trans;
    p.a_off = a_off; p.x_off = x_off; p.y_off = y_off; p.alpha = alpha; p.beta = beta;
    v.push_back(p);
    blk.push_back(nblk);
    nblk += (out_n + 63) / 64;
}

// Upload a descriptor set, with blocks of rb output entries (matvec_rows_per_block of its
// 64-entry block count: small sets get smaller blocks, so the launch still fills the GPU).
int upload_mv(DevMem& d, DevMem& db, int& n, int64_t& nblk, int& rb, std::vector<MatvecProb>& v,
              std::vector<int64_t>& blk, int64_t total, cudaStream_t st, double* work = nullptr,
              std::vector<int64_t>* keep = nullptr)
{
    n = (int)v.size();
    rb = matvec_rows_per_block(total);
    nblk = 0;
    for (size_t i = 0; i < v.size(); ++i) {
        blk[i] = nblk;
        nblk += ((v[i].trans ? v[i].cols : v[i].rows) + rb - 1) / rb;
    }
    if (work) {
        *work = 0.0;
        for (const MatvecProb& p : v) *work += (double)p.rows * (double)p.cols;
    }
    int rc;
    if ((rc = upload(d, v, st))) return rc;
    if (keep) {
        *keep = blk;
        keep->push_back(nblk);
    }
    return upload(db, blk, st);
}

// Index maps and matvec descriptors of the solve for one level.
int solve_plan(rs_op* op, Level& L, const Level* child, cudaStream_t st)
{
    const int nb = L.nb;
    L.sum_m = L.act_off[nb];
    L.sum_k = L.l == 0 ? 0 : L.k_off[nb];
    int rc;
    if (L.l == op->d) {
        std::vector<int64_t> idx(L.sum_m);
        for (int b = 0; b < nb; ++b)
            for (int64_t p = 0; p < L.m[b]; ++p)
                idx[L.act_off[b] + p] = op->input_of_g[L.act[L.act_off[b] + L.perm[L.act_off[b] + p]]];
        if ((rc = upload(L.d_idx_leaf, idx, st))) return rc;
    } else if (L.l > 0) {
        std::vector<int64_t> idx(L.sum_m);
        for (int b = 0; b < nb; ++b)
            for (int64_t p = 0; p < L.m[b]; ++p)
                idx[L.act_off[b] + p] = child->k_off[2 * b] + L.perm[L.act_off[b] + p];
        if ((rc = upload(L.d_idx_up, idx, st))) return rc;
    }
    if (L.l == 0) {
        std::vector<MatvecProb> v;
        std::vector<int64_t> blk;
        int64_t n = 0;
        add_mv(v, blk, n, (int)L.m[0], (int)L.m[0], (int)L.m[0], 0, 0, 0, 0, 1.0, 0.0);
        return upload_mv(L.d_mv_phi, L.d_mv_phi_blk, L.n_mv_phi, L.b_mv_phi, L.rb_phi, v, blk, n, st, &L.mvw_phi,
                         &L.h_blk_phi);
    }
    std::vector<int64_t> isk(L.sum_k);
    for (int b = 0; b < nb; ++b)
        for (int64_t a = 0; a < L.k[b]; ++a) isk[L.k_off[b] + a] = L.act_off[b] + a;
    if ((rc = upload(L.d_idx_sk, isk, st))) return rc;
    std::vector<MatvecProb> vphi, vT, vE, vTt;
    std::vector<int64_t> bphi, bT, bE, bTt;
    int64_t nphi = 0, nT = 0, nE = 0, nTt = 0;
    for (int b = 0; b < nb; ++b) {
        if (!L.cmp.empty() && L.cmp[b]) continue;   // applied through its compressed forms
        const int m = (int)L.m[b], k = (int)L.k[b];
        add_mv(vphi, bphi, nphi, m, m, m, 0, L.phi_off[b], L.act_off[b], L.act_off[b], 1.0, 0.0);
        if (m - k > 0) add_mv(vT, bT, nT, k, m - k, k, 0, L.t_off[b], L.act_off[b] + k, L.k_off[b], 1.0, 1.0);
        add_mv(vE, bE, nE, k, k, k, 0, L.e_off[b], L.k_off[b], L.k_off[b], 1.0, 0.0);
        if (m - k > 0) add_mv(vTt, bTt, nTt, k, m - k, k, 1, L.t_off[b], L.k_off[b], L.act_off[b] + k, 1.0, 0.0);
    }
    if ((rc = upload_mv(L.d_mv_phi, L.d_mv_phi_blk, L.n_mv_phi, L.b_mv_phi, L.rb_phi, vphi, bphi, nphi, st,
                        &L.mvw_phi, &L.h_blk_phi)))
        return rc;
    if ((rc = upload_mv(L.d_mv_T, L.d_mv_T_blk, L.n_mv_T, L.b_mv_T, L.rb_T, vT, bT, nT, st, &L.mvw_T, &L.h_blk_T)))
        return rc;
    if ((rc = upload_mv(L.d_mv_E, L.d_mv_E_blk, L.n_mv_E, L.b_mv_E, L.rb_E, vE, bE, nE, st, &L.mvw_E, &L.h_blk_E)))
        return rc;
    return upload_mv(L.d_mv_Tt, L.d_mv_Tt_blk, L.n_mv_Tt, L.b_mv_Tt, L.rb_Tt, vTt, bTt, nTt, st, &L.mvw_Tt,
                     &L.h_blk_Tt);
}

void compute_stats(rs_op* op)
{
    rs_stats& s = op->stats;
    s.depth = op->d;
    s.n_side = op->n;
    s.root_m = op->lev[0].m[0];
    double ff = 0.0, sw = 0.0;
    // an SPD inverse by the symmetric sweep does m^3 flops, Gauss-Jordan 2 m^3
    const double inv = (use_sweep(op) && s.spd_fallbacks == 0) ? 1.0 : 2.0;
    int64_t bytes = 0, cboxes = 0, replaced = 0;
    for (int l = 1; l <= op->d; ++l) {
        const Level& L = op->lev[l];
        std::vector<char> fac(L.nb, 1);                 // boxes factored (one per class)
        if (op->opts.translation_invariant) {
            fac.assign(L.nb, 0);
            for (int b : L.ti_rep) fac[b] = 1;
        }
        for (int b = 0; b < L.nb; ++b) {
            const double m = (double)L.m[b], k = (double)L.k[b], r = (double)L.r[b];
            if (!fac[b]) continue;
            ff += 4.0 * r * m * k - 2.0 * k * k * (r + m) + 4.0 * k * k * k / 3.0;   // CPQR, k steps
            ff += k * k * (m - k);                                                // T = R11^{-1} R12
            if (op->opts.forward_only) continue;
            ff += inv * m * m * m;                                                // F^{-1}
            ff += 2.0 * m * (m - k) * k;                                          // W
            ff += (inv == 1.0) ? k * (k + 1.0) * (m - k) : 2.0 * k * (m - k) * k;  // E^{-1} (lower only if SPD)
            ff += inv * k * k * k;                                                // E
            if (!L.cmp.empty() && L.cmp[b]) {
                ++cboxes;
                replaced += (int64_t)(m * m + k * k + k * (m - k)) * op->esz;
            }
        }
        // entries read by one apply: Phi, E up and down, T and T^T, dense and compressed parts
        sw += 2.0 * L.mvw_phi + L.mvw_T + 2.0 * L.mvw_E + L.mvw_Tt;
        sw += 2.0 * L.p_phi.work + L.p_T.work + 2.0 * L.p_E.work + L.p_Tt.work;
        if (!L.dense_freed)
            bytes += (L.phi_off.back() + L.e_off.back() + L.t_off.back()) * op->esz;
        bytes += L.act_off.back() * 8 + L.nb * 64;
    }
    const double m0 = (double)op->lev[0].m[0];
    if (!op->opts.forward_only) {
        ff += inv * m0 * m0 * m0;
        sw += m0 * m0;
        bytes += (int64_t)(m0 * m0 * op->esz);
    }
    bytes += op->cstore_n * op->esz;
    s.flops_factor = ff;
    s.flops_solve_per_rhs = 2.0 * sw;
    s.bytes_solve = op->esz * sw;
    s.bytes_factors = bytes;
    s.compressed_boxes = cboxes;
    s.bytes_compressed = op->cstore_n * op->esz;
    s.bytes_dense_replaced = replaced;
}

}  // namespace

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool on_other_device(const void* p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type != cudaMemoryTypeDevice) return false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.device != dev;
}

// Algorithm 1 over all levels in storage precision T: IDs (d..1), inverses (d..1), root.
template <class T>
int factor_levels(rs_op* op, cudaStream_t st, Clock::time_point t0)
{
    int rc;
    {
        IdWork w;
        for (int l = op->d; l >= 1; --l)
            if ((rc = id_level<T>(op, op->lev[l], l < op->d ? &op->lev[l + 1] : nullptr, w, st))) return rc;
    }
    op->stats.ms_tree = ms_since(t0);
    auto t1 = Clock::now();
    const bool fwd_only = op->opts.forward_only != 0;
    // the per-box inverse phase runs without a host round trip per sweep: one status check
    // after the root, and a rerun with pivoted Gauss-Jordan if a block was not SPD
    op->defer_spd = use_sweep(op) && !op->opts.per_box && !op->opts.translation_invariant && !fwd_only;
    for (int l = op->d; l >= 1; --l) {
        const Level* child = l < op->d ? &op->lev[l + 1] : nullptr;
        if (fwd_only) {             // the tree build alone: no F^{-1}, no E
            Level& L = op->lev[l];
            L.phi_off.assign(L.nb + 1, 0);
            L.e_off.assign(L.nb + 1, 0);
            L.w_off.assign(L.nb + 1, 0);
            continue;
        }
        rc = op->opts.translation_invariant ? inverse_level_ti<T>(op, l, st)
                                            : inverse_level<T>(op, op->lev[l], child, st);
        if (rc) return rc;
    }
    // root: active set = skeletons of (1,0) then (1,1), natural order
    Level& R = op->lev[0];
    const Level& L1 = op->lev[1];
    R.m = {L1.k[0] + L1.k[1]};
    R.k = {0};
    R.act = L1.skel;
    R.act_off = {0, R.m[0]};
    R.perm.resize(R.m[0]);
    for (int64_t i = 0; i < R.m[0]; ++i) R.perm[i] = (int32_t)i;
    R.max_m = (int)R.m[0];
    if ((rc = upload(R.d_act, to32(R.act), st))) return rc;
    if ((rc = upload(R.d_act_off, R.act_off, st))) return rc;
    if ((rc = upload(R.d_perm, R.perm, st))) return rc;
    if ((rc = upload(R.d_m, to32(R.m), st))) return rc;
    if (fwd_only) R.phi_off = {0, 0};
    else if ((rc = inverse_level<T>(op, R, &op->lev[1], st))) return rc;
    if (op->defer_spd) {
        op->defer_spd = false;
        RS_CUDA(cudaStreamSynchronize(st));
        prof_flush(op);
        int s = 0;
        RS_CUDA(cudaMemcpy(&s, op->d_status.p, sizeof(int), cudaMemcpyDeviceToHost));
        if (s & DEV_NOT_SPD) {
            // every inversion of the phase again, by pivoted Gauss-Jordan (each level's F is
            // rebuilt from the children's new E)
            RS_CUDA(cudaMemsetAsync(op->d_status.p, 0, sizeof(int), st));
            op->opts.spd_inverse = 0;
            for (int l = op->d; l >= 1 && !rc; --l)
                rc = inverse_level<T>(op, op->lev[l], l < op->d ? &op->lev[l + 1] : nullptr, st);
            if (!rc) rc = inverse_level<T>(op, R, &op->lev[1], st);
            op->opts.spd_inverse = 1;
            if (rc) return rc;
            op->stats.spd_fallbacks = 2 * op->d + 1;
        }
        if ((rc = check_status(op, st))) return rc;
    }
    if ((rc = compress_levels<T>(op, st))) return rc;
    for (int l = 0; l <= op->d; ++l)
        if ((rc = solve_plan(op, op->lev[l], l < op->d ? &op->lev[l + 1] : nullptr, st))) return rc;
    RS_CUDA(cudaStreamSynchronize(st));
    op->stats.ms_inverse = ms_since(t1);
    compute_stats(op);
    return RS_OK;
}

int factor_impl(const rs_tree* tree, const rs_kernel* kernel, const double* a, double eps, const rs_opts* opts,
                cudaStream_t st, rs_op** out)
{
    rs_op* op = new (std::nothrow) rs_op();
    if (!op) return fail(RS_E_NOMEM, "host allocation");
    std::unique_ptr<rs_op> guard(op);
    RS_CUDA(cudaGetDevice(&op->device));
    if (opts) op->opts = *opts; else rs_opts_default(&op->opts);
    op->n = tree->n;
    op->N = tree->n * tree->n;
    op->d = tree->d;
    op->kind = kernel ? kernel->kind : RS_LAPLACE;
    op->kappa = kernel ? kernel->kappa : 0.0;
    op->eps = eps;
    op->input_of_g = tree->input_of_g;
    if (op->kind == RS_LAPLACE) {
        if (kernel && kernel->b) return fail(RS_E_INVALID, "b(x) is only used by the Helmholtz kernel");
        if (op->opts.precision != RS_FP64 && op->opts.precision != RS_MIXED_FP32)
            return fail(RS_E_INVALID, "Laplace operators are factored in RS_FP64 or RS_MIXED_FP32");
        op->esz = op->opts.precision == RS_MIXED_FP32 ? (int)sizeof(float) : (int)sizeof(double);
    } else if (op->kind == RS_HELMHOLTZ) {
        if (!(op->kappa > 0.0)) return fail(RS_E_INVALID, "Helmholtz needs kappa > 0");
        if (op->opts.precision == RS_FP64) op->opts.precision = RS_C128;
        if (op->opts.precision != RS_C128 && op->opts.precision != RS_C64_REFINED)
            return fail(RS_E_INVALID, "Helmholtz operators are factored in RS_C128 or RS_C64_REFINED");
        op->esz = op->opts.precision == RS_C64_REFINED ? 2 * (int)sizeof(float) : 2 * (int)sizeof(double);
    } else {
        return fail(RS_E_INVALID, "unknown kernel kind");
    }
    if ((op->opts.precision == RS_MIXED_FP32 || op->opts.precision == RS_C64_REFINED) &&
        !(op->opts.refine_tol > 0.0 && op->opts.refine_max_iter >= 1))
        return fail(RS_E_INVALID, "refined precisions need refine_tol > 0 and refine_max_iter >= 1");
    if (op->opts.proxy_points < 0 || op->opts.proxy_points > 4096 || !(op->opts.proxy_radius_factor > 0.0))
        return fail(RS_E_INVALID, "bad proxy options");
    if (!(eps >= 0.0) || !(eps < 1.0)) return fail(RS_E_INVALID, "eps must be in [0, 1)");
    if (op->opts.spin_limit <= 0) return fail(RS_E_INVALID, "spin_limit must be positive");
    if (op->opts.k_cut < 0) return fail(RS_E_INVALID, "k_cut must be >= 0");
    if (op->opts.k_cut > 0 && op->opts.hss_leaf < 1) return fail(RS_E_INVALID, "hss_leaf must be >= 1");
    if (!(op->opts.hss_eps >= 0.0) || !(op->opts.hss_eps < 1.0)) return fail(RS_E_INVALID, "hss_eps must be in [0, 1)");
    if (op->opts.cpqr_variant < -1 || op->opts.cpqr_variant > 8) return fail(RS_E_INVALID, "cpqr_variant must be -1 .. 8");
    if (op->opts.gemm_form != 0 && op->opts.gemm_form != 1) return fail(RS_E_INVALID, "gemm_form must be 0 or 1");
    if (op->opts.sweep_panel != 0 && op->opts.sweep_panel != 8 && op->opts.sweep_panel != 16)
        return fail(RS_E_INVALID, "sweep_panel must be 0, 8 or 16");
    if (op->opts.forward_only && (op->opts.translation_invariant || op->opts.k_cut > 0 || op->opts.per_box))
        return fail(RS_E_INVALID, "forward_only combines with none of translation_invariant, k_cut, per_box");
    if (op->opts.translation_invariant < 0 || op->opts.translation_invariant > 2)
        return fail(RS_E_INVALID, "translation_invariant must be 0, 1 or 2");
    if (op->opts.translation_invariant) {
        if (op->opts.k_cut > 0) return fail(RS_E_INVALID, "translation_invariant does not combine with k_cut");
        if (op->opts.translation_invariant == 1 && 9 * op->N > (int64_t)INT32_MAX)
            return fail(RS_E_INVALID, "translation_invariant: grid too large");
        for (int64_t i = 1; i < op->N; ++i)
            if ((a && a[i] != a[0]) || (kernel && kernel->b && kernel->b[i] != kernel->b[0]))
                return fail(RS_E_INVALID, "translation_invariant needs constant a(x) and b(x)");
    }
    const double h = 1.0 / (double)op->n;
    op->K.n = (int)op->n;
    op->K.h = h;
    op->K.c0 = -(h * h) / (4.0 * M_PI);
    // diagonal: a_g - (1/2pi) * integral of log|y - x_g| over the h x h cell, whose closed
    // form is h^2 (log h - log(2)/2 - 3/2 + pi/4)
    op->K.self = -(h * h * (std::log(h) - 0.5 * std::log(2.0) - 1.5 + M_PI / 4.0)) / (2.0 * M_PI);
    op->K.kind = op->kind;
    op->K.kappa = op->kappa;
    auto t0 = Clock::now();
    int rc;
    if (op->kind == RS_HELMHOLTZ) {
        // (i/4) * integral of H0^(1)(kappa |y - x|) over the h x h cell centred at x
        double re = 0.0, im = 0.0;
        helmholtz_cell_integral(h, op->kappa, &re, &im);
        op->K.hs_re = -0.25 * im;
        op->K.hs_im = 0.25 * re;
        // symmetric form of Eq. (5.6): s = kappa sqrt(b), grid order and input order
        std::vector<double> sg((size_t)op->N), si((size_t)op->N);
        for (int64_t i = 0; i < op->N; ++i) {
            const double bi = (kernel && kernel->b) ? kernel->b[i] : 1.0;
            if (!(bi > 0.0) || !std::isfinite(bi)) return fail(RS_E_INVALID, "b(x) must be positive and finite");
            si[(size_t)i] = op->kappa * std::sqrt(bi);
        }
        for (int64_t g = 0; g < op->N; ++g) sg[(size_t)g] = si[(size_t)op->input_of_g[g]];
        if ((rc = upload(op->d_s, sg, st))) return rc;
        if ((rc = upload(op->d_s_in, si, st))) return rc;
        op->K.s = op->d_s.as<double>();
        op->ti_s0 = si[0];
    }
    // a in grid order
    std::vector<double> ag(op->N, 1.0);
    if (a)
        for (int64_t g = 0; g < op->N; ++g) ag[g] = a[op->input_of_g[g]];
    if ((rc = upload(op->d_a, ag, st))) return rc;
    if ((rc = kernel_tables(op, st))) return rc;
    const int P = op->opts.proxy_points;
    std::vector<double> uc(2 * (size_t)P + 1);
    for (int q = 0; q < P; ++q) {
        const double ang = (2.0 * M_PI * (double)q) / (double)P;
        uc[q] = std::cos(ang);
        uc[P + q] = std::sin(ang);
    }
    if ((rc = upload(op->d_ucirc, uc, st))) return rc;
    RS_CUDA(op->d_status.alloc(sizeof(int)));
    RS_CUDA(op->d_zero.alloc(sizeof(int64_t)));
    RS_CUDA(cudaMemsetAsync(op->d_zero.p, 0, sizeof(int64_t), st));
    RS_CUDA(cudaMemsetAsync(op->d_status.p, 0, sizeof(int), st));
    op->lev.resize(op->d + 1);
    if (op->opts.translation_invariant) op->ti_lev.resize(op->d + 1);
    for (int l = 0; l <= op->d; ++l) {
        op->lev[l].l = l;
        op->lev[l].nb = 1 << l;
    }
    switch (op->opts.precision) {
        case RS_MIXED_FP32: rc = factor_levels<float>(op, st, t0); break;
        case RS_C128: rc = factor_levels<cplx<double>>(op, st, t0); break;
        case RS_C64_REFINED: rc = factor_levels<cplx<float>>(op, st, t0); break;
        default: rc = factor_levels<double>(op, st, t0); break;
    }
    if (rc) return rc;
    *out = guard.release();
    return RS_OK;
}

SolveLayout solve_layout(const rs_op* op, int64_t nrhs)
{
    SolveLayout Ls;
    const int d = op->d;
    Ls.woff.assign(d + 2, 0);
    Ls.goff.assign(d + 2, 0);
    for (int l = 1; l <= d; ++l) {
        Ls.woff[l + 1] = Ls.woff[l] + op->lev[l].sum_m;
        Ls.goff[l + 1] = Ls.goff[l] + op->lev[l].sum_k;
        Ls.max_m = std::max(Ls.max_m, op->lev[l].sum_m);
        Ls.max_k = std::max(Ls.max_k, op->lev[l].sum_k);
    }
    Ls.max_m = std::max<int64_t>(Ls.max_m, op->lev[0].sum_m);
    Ls.n_w = Ls.woff[d + 1] * nrhs + 1;
    Ls.n_g = Ls.goff[d + 1] * nrhs + 1;
    Ls.n_u = Ls.max_m * nrhs + 1;
    Ls.n_t = Ls.max_k * nrhs + 1;
    int64_t zr = 0;
    for (int l = 1; l <= d; ++l) {
        const Level& L = op->lev[l];
        zr = std::max({zr, L.p_phi.z_rows, L.p_T.z_rows, L.p_E.z_rows, L.p_Tt.z_rows});
    }
    Ls.n_z = zr * nrhs + 1;
    return Ls;
}

namespace {

// The kernel sequence of the inverse apply (Algorithm 6 as the recursion of Eqs. 2.10-2.12)
// in storage type T; f (fd) and x (xd) are FP64 N x nrhs column-major in input order.
template <class T>
int solve_run_t(rs_op* op, const SolveLayout& Ls, const SolveWork& ws, const typename sc_traits<T>::io* fd,
                typename sc_traits<T>::io* xd, int64_t nrhs, cudaStream_t st)
{
    using IO = typename sc_traits<T>::io;
    const int64_t N = op->N;
    const int d = op->d;
    const std::vector<int64_t>& woff = Ls.woff;
    const std::vector<int64_t>& goff = Ls.goff;
    T* W = (T*)ws.w;
    T* Gb = (T*)ws.g;
    T* Ph = (T*)ws.phi;
    T* U = (T*)ws.u;
    T* XO = (T*)ws.out;
    T* Tt = (T*)ws.t;
    T* Z = (T*)ws.z;
    const int nr = (int)nrhs;
    const double esz = (double)sizeof(T);
    int rc;
    // one descriptor set: one launch, or (opts.per_box) one launch per box
    auto mv = [&](const Level& L, const DevMem& probs, const DevMem& blk0, int np, int64_t nblk, int rb,
                  const std::vector<int64_t>& hblk, const T* A, const T* x, T* y) -> int {
        if (!op->opts.per_box || np <= 1) {
            RS_CUDA(launch_matvec<T>(st, probs.as<MatvecProb>(), blk0.as<int64_t>(), np, nblk, A, x, y, nr, rb));
            return RS_OK;
        }
        (void)L;
        for (int i = 0; i < np; ++i)
            RS_CUDA(launch_matvec<T>(st, probs.as<MatvecProb>() + i, op->d_zero.as<int64_t>(), 1, hblk[i + 1] - hblk[i],
                                     A, x, y, nr, rb));
        return RS_OK;
    };
    // compressed boxes (Sec. 3): their part of an apply, from `in` to `out`
    auto run_cprog = [&](const Program& p, const T* in, T* out) -> int {
        if (p.st.empty()) return RS_OK;
        ProfScope ps(op, RS_PROF_SOLVE, st, 2.0 * p.work * (double)nrhs, esz * p.work);
        return run_program<T>(st, p, op->d_cstore.as<T>(), in, out, Z, nr);
    };
    // upward pass
    for (int l = d; l >= 1; --l) {
        Level& L = op->lev[l];
        T* wl = W + woff[l] * nrhs;
        T* gl = Gb + goff[l] * nrhs;
        if (l == d) RS_CUDA(launch_gather_cm<IO, T>(st, L.sum_m, L.d_idx_leaf.as<int64_t>(), fd, N, U, nr));
        else RS_CUDA(launch_gather_rows<T>(st, L.sum_m, L.d_idx_up.as<int64_t>(), Gb + goff[l + 1] * nrhs, U, nr));
        { ProfScope ps(op, RS_PROF_SOLVE, st, 2.0 * L.mvw_phi * (double)nrhs, esz * L.mvw_phi);
        if ((rc = mv(L, L.d_mv_phi, L.d_mv_phi_blk, L.n_mv_phi, L.b_mv_phi, L.rb_phi, L.h_blk_phi,
                     L.d_Phi.as<T>(), U, wl))) return rc; }
        if ((rc = run_cprog(L.p_phi, U, wl))) return rc;
        RS_CUDA(launch_gather_rows<T>(st, L.sum_k, L.d_idx_sk.as<int64_t>(), wl, Tt, nr));
        { ProfScope ps(op, RS_PROF_SOLVE, st, 2.0 * L.mvw_T * (double)nrhs, esz * L.mvw_T);
        if ((rc = mv(L, L.d_mv_T, L.d_mv_T_blk, L.n_mv_T, L.b_mv_T, L.rb_T, L.h_blk_T,
                     L.d_T.as<T>(), wl, Tt))) return rc; }
        if ((rc = run_cprog(L.p_T, wl, Tt))) return rc;
        { ProfScope ps(op, RS_PROF_SOLVE, st, 2.0 * L.mvw_E * (double)nrhs, esz * L.mvw_E);
        if ((rc = mv(L, L.d_mv_E, L.d_mv_E_blk, L.n_mv_E, L.b_mv_E, L.rb_E, L.h_blk_E,
                     L.d_E.as<T>(), Tt, gl))) return rc; }
        if ((rc = run_cprog(L.p_E, Tt, gl))) return rc;
    }
    // root
    {
        Level& R = op->lev[0];
        { ProfScope ps(op, RS_PROF_SOLVE, st, 2.0 * R.mvw_phi * (double)nrhs, esz * R.mvw_phi);
        if ((rc = mv(R, R.d_mv_phi, R.d_mv_phi_blk, R.n_mv_phi, R.b_mv_phi, R.rb_phi, R.h_blk_phi,
                     R.d_Phi.as<T>(), Gb + goff[1] * nrhs, Ph + goff[1] * nrhs))) return rc; }
    }
    // downward pass
    for (int l = 1; l <= d; ++l) {
        Level& L = op->lev[l];
        T* wl = W + woff[l] * nrhs;
        T* gl = Gb + goff[l] * nrhs;
        T* pl = Ph + goff[l] * nrhs;
        RS_CUDA(cudaMemcpyAsync(Tt, gl, sizeof(T) * (size_t)(L.sum_k * nrhs), cudaMemcpyDeviceToDevice, st));
        { ProfScope ps(op, RS_PROF_SOLVE, st, 2.0 * L.mvw_E * (double)nrhs, esz * L.mvw_E);
        if ((rc = mv(L, L.d_mv_E, L.d_mv_E_blk, L.n_mv_E, L.b_mv_E, L.rb_E, L.h_blk_E,
                     L.d_E.as<T>(), pl, Tt))) return rc; }   // beta = 0: Tt = E phi
        if ((rc = run_cprog(L.p_E, pl, Tt))) return rc;
        RS_CUDA(launch_axpby<T>(st, L.sum_k * nrhs, (T)-1, gl, (T)1, Tt));   // Tt = E phi - g
        RS_CUDA(launch_scatter_rows<T>(st, L.sum_k, L.d_idx_sk.as<int64_t>(), Tt, U, nr));
        { ProfScope ps(op, RS_PROF_SOLVE, st, 2.0 * L.mvw_Tt * (double)nrhs, esz * L.mvw_Tt);
        if ((rc = mv(L, L.d_mv_Tt, L.d_mv_Tt_blk, L.n_mv_Tt, L.b_mv_Tt, L.rb_Tt, L.h_blk_Tt,
                     L.d_T.as<T>(), Tt, U))) return rc; }
        if ((rc = run_cprog(L.p_Tt, Tt, U))) return rc;
        { ProfScope ps(op, RS_PROF_SOLVE, st, 2.0 * L.mvw_phi * (double)nrhs, esz * L.mvw_phi);
        if ((rc = mv(L, L.d_mv_phi, L.d_mv_phi_blk, L.n_mv_phi, L.b_mv_phi, L.rb_phi, L.h_blk_phi,
                     L.d_Phi.as<T>(), U, XO))) return rc; }
        if ((rc = run_cprog(L.p_phi, U, XO))) return rc;
        RS_CUDA(launch_axpby<T>(st, L.sum_m * nrhs, (T)1, wl, (T)1, XO));   // x' = w + Phi v
        if (l == d) RS_CUDA(launch_scatter_cm<T, IO>(st, L.sum_m, L.d_idx_leaf.as<int64_t>(), XO, N, xd, nr));
        else RS_CUDA(launch_scatter_rows<T>(st, L.sum_m, L.d_idx_up.as<int64_t>(), XO, Ph + goff[l + 1] * nrhs, nr));
    }
    return RS_OK;
}

}  // namespace

int solve_run(rs_op* op, const SolveLayout& Ls, const SolveWork& ws, const double* fd, double* xd, int64_t nrhs,
              cudaStream_t st, bool profile)
{
    const int saved_profile = op->opts.profile;
    op->opts.profile = profile ? saved_profile : 0;
    int rc;
    switch (op->opts.precision) {
        case RS_MIXED_FP32: rc = solve_run_t<float>(op, Ls, ws, fd, xd, nrhs, st); break;
        case RS_C128: rc = solve_run_t<cplx<double>>(op, Ls, ws, (const cplx<double>*)fd, (cplx<double>*)xd, nrhs, st); break;
        case RS_C64_REFINED: rc = solve_run_t<cplx<float>>(op, Ls, ws, (const cplx<double>*)fd, (cplx<double>*)xd, nrhs, st); break;
        default: rc = solve_run_t<double>(op, Ls, ws, fd, xd, nrhs, st); break;
    }
    op->opts.profile = saved_profile;
    return rc;
}

// Workspace of one inverse apply with nrhs columns (grown on demand); bumps op->ws_gen when a
// buffer moves, which retires the solve graphs captured against the old addresses.
int solve_workspace(rs_op* op, int64_t nrhs, SolveLayout& Ls, SolveWork& ws)
{
    Ls = solve_layout(op, nrhs);
    const size_t e = (size_t)op->esz;
    RS_CUDA(op->s_w.alloc(e * (size_t)Ls.n_w));
    RS_CUDA(op->s_g.alloc(e * (size_t)Ls.n_g));
    RS_CUDA(op->s_phi.alloc(e * (size_t)Ls.n_g));
    RS_CUDA(op->s_u.alloc(e * (size_t)Ls.n_u));
    RS_CUDA(op->s_out.alloc(e * (size_t)Ls.n_u));
    RS_CUDA(op->s_t.alloc(e * (size_t)Ls.n_t));
    RS_CUDA(op->s_z.alloc(e * (size_t)Ls.n_z));
    if (op->kind == RS_HELMHOLTZ) RS_CUDA(op->s_fs.alloc(2 * sizeof(double) * (size_t)(op->N * nrhs)));
    ws = SolveWork{op->s_w.p, op->s_g.p, op->s_phi.p, op->s_u.p, op->s_out.p, op->s_t.p, op->s_z.p};
    const void* now[9] = {op->s_w.p, op->s_g.p, op->s_phi.p, op->s_u.p, op->s_out.p, op->s_t.p, op->s_z.p,
                          op->s_fs.p, nullptr};
    if (memcmp(now, op->ws_ptrs, sizeof(now)) != 0) {
        memcpy(op->ws_ptrs, now, sizeof(now));
        ++op->ws_gen;
    }
    return RS_OK;
}

// The launches of one inverse apply (no allocation, no host synchronisation).
int apply_launch(rs_op* op, const SolveLayout& Ls, const SolveWork& ws, const double* fd, double* xd, int64_t nrhs,
                 cudaStream_t st, bool profile)
{
    if (op->kind != RS_HELMHOLTZ) return solve_run(op, Ls, ws, fd, xd, nrhs, st, profile);
    // symmetric form: x = S (S^{-1} A S)^{-1} S^{-1} f, S = diag(kappa sqrt(b))
    using Z = cplx<double>;
    RS_CUDA(launch_scale_cm<Z>(st, op->N, (int)nrhs, op->d_s_in.as<double>(), -1, (const Z*)fd, op->s_fs.as<Z>()));
    const int rc = solve_run(op, Ls, ws, op->s_fs.as<double>(), xd, nrhs, st, profile);
    if (rc) return rc;
    RS_CUDA(launch_scale_cm<Z>(st, op->N, (int)nrhs, op->d_s_in.as<double>(), 1, (const Z*)xd, (Z*)xd));
    return RS_OK;
}

// One inverse apply with the library's own (growing) workspace; fd, xd device FP64.
int apply_once(rs_op* op, const double* fd, double* xd, int64_t nrhs, cudaStream_t st)
{
    SolveLayout Ls;
    SolveWork ws;
    int rc = solve_workspace(op, nrhs, Ls, ws);
    if (rc) return rc;
    return apply_launch(op, Ls, ws, fd, xd, nrhs, st, op->opts.profile != 0);
}

// One inverse apply replayed from a CUDA graph (captured on first use for this nrhs and
// workspace): f is copied into the staging buffer the graph reads, x out of the one it writes.
int apply_graph(rs_op* op, const double* fd, double* xd, int64_t nrhs, cudaStream_t st)
{
    SolveLayout Ls;
    SolveWork ws;
    int rc = solve_workspace(op, nrhs, Ls, ws);
    if (rc) return rc;
    const size_t io = (op->kind == RS_HELMHOLTZ ? 2 : 1) * sizeof(double) * (size_t)(op->N * nrhs);
    const void* gin0 = op->g_in.p;
    const void* gout0 = op->g_out.p;
    RS_CUDA(op->g_in.alloc(io));
    RS_CUDA(op->g_out.alloc(io));
    if (op->g_in.p != gin0 || op->g_out.p != gout0) ++op->ws_gen;
    RS_CUDA(cudaMemcpyAsync(op->g_in.p, fd, io, cudaMemcpyDeviceToDevice, st));
    rs_op::SolveGraph* g = nullptr;
    for (auto it = op->graphs.begin(); it != op->graphs.end();) {
        if (it->gen != op->ws_gen) {                    // captured against buffers since moved
            cudaGraphExecDestroy(it->exec);
            it = op->graphs.erase(it);
            continue;
        }
        if (it->nrhs == nrhs) g = &*it;
        ++it;
    }
    if (!g) {
        if (op->graphs.size() >= 16) {
            for (auto& e : op->graphs) cudaGraphExecDestroy(e.exec);
            op->graphs.clear();
        }
        if (!op->cap_stream) RS_CUDA(cudaStreamCreateWithFlags(&op->cap_stream, cudaStreamNonBlocking));
        const int64_t l0 = rs_launch_count();
        RS_CUDA(cudaStreamBeginCapture(op->cap_stream, cudaStreamCaptureModeThreadLocal));
        rc = apply_launch(op, Ls, ws, op->g_in.as<double>(), op->g_out.as<double>(), nrhs, op->cap_stream, false);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(op->cap_stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (ec != cudaSuccess) return cuda_fail(ec, "cudaStreamEndCapture (inverse apply)");
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) return cuda_fail(ei, "cudaGraphInstantiate (inverse apply)");
        // the launches were recorded, not made: the count is taken on every replay instead
        const int64_t nl = rs_launch_count() - l0;
        count_launches((int)-nl);
        op->graphs.push_back({nrhs, op->ws_gen, exec, nl});
        g = &op->graphs.back();
    }
    {
        ProfScope ps(op, RS_PROF_SOLVE, st, op->stats.flops_solve_per_rhs * (double)nrhs, op->stats.bytes_solve);
        RS_CUDA(cudaGraphLaunch(g->exec, st));
    }
    count_launches((int)g->launches);
    RS_CUDA(cudaMemcpyAsync(xd, op->g_out.p, io, cudaMemcpyDeviceToDevice, st));
    return RS_OK;
}

// ------------------------------------------------------------------ forward apply
// y = A x through the HSS form of A that the factorization's IDs define: the off-diagonal
// blocks A(I_i, I_j) ~ L_i A(sk_i, sk_j) R_j (Sec. 2.2, the ID of Eq. 2.1 on both sides of the
// symmetric form), nested level by level as in the telescoping form of Eq. 2.9:
//   up:   xh_i = u_i(sk) + T_i u_i(rs), u_i = x(I_i) at a leaf and [xh_c1; xh_c2] above;
//   root: yh of the two level-1 boxes = [A(sk_1, sk_2) xh_2; A(sk_2, sk_1) xh_1];
//   down: z_i = L_i yh_i (z(sk) = yh_i, z(rs) = T_i^T yh_i); above the leaves z_i plus the
//         children's mutual blocks gives yh_c1, yh_c2; at a leaf y(I_i) = A(I_i, I_i) x + z_i.
// The T products reuse the solve's descriptors; the blocks of A are generated on the fly.

int fw_plan(rs_op* op, cudaStream_t st)
{
    if (op->fw_built) return RS_OK;
    const int RB = kblock_rows_per_block();
    auto add = [&](std::vector<KbProb>& v, std::vector<int64_t>& blk, int64_t& nblk, int64_t rows, int64_t cols,
                   int64_t r_off, int64_t c_off, int64_t x_off, int64_t y_off) {
        if (rows <= 0 || cols <= 0) return;
        KbProb p{};
        p.rows = (int)rows; p.cols = (int)cols;
        p.r_off = r_off; p.c_off = c_off; p.x_off = x_off; p.y_off = y_off;
        v.push_back(p);
        blk.push_back(nblk);
        nblk += (rows + RB - 1) / RB;
    };
    int rc;
    for (int l = 0; l < op->d; ++l) {
        Level& P = op->lev[l];
        const Level& C = op->lev[l + 1];
        std::vector<KbProb> v;
        std::vector<int64_t> blk;
        int64_t nblk = 0;
        for (int b = 0; b < P.nb; ++b) {
            const int c1 = 2 * b, c2 = 2 * b + 1;
            add(v, blk, nblk, C.k[c1], C.k[c2], C.k_off[c1], C.k_off[c2], C.k_off[c2], C.k_off[c1]);
            add(v, blk, nblk, C.k[c2], C.k[c1], C.k_off[c2], C.k_off[c1], C.k_off[c1], C.k_off[c2]);
        }
        if ((rc = upload(P.d_fw_pts, to32(C.skel), st))) return rc;
        if ((rc = upload(P.d_fw_sib, v, st))) return rc;
        if ((rc = upload(P.d_fw_sib_blk, blk, st))) return rc;
        P.n_fw_sib = (int)v.size();
        P.b_fw_sib = nblk;
    }
    Level& L = op->lev[op->d];
    std::vector<int64_t> pts(L.act.size());
    std::vector<KbProb> v;
    std::vector<int64_t> blk;
    int64_t nblk = 0;
    for (int b = 0; b < L.nb; ++b) {
        const int64_t a0 = L.act_off[b], m = L.m[b];
        for (int64_t p = 0; p < m; ++p) pts[a0 + p] = L.act[a0 + L.perm[a0 + p]];
        add(v, blk, nblk, m, m, a0, a0, a0, a0);
    }
    if ((rc = upload(L.d_fw_leaf_pts, to32(pts), st))) return rc;
    if ((rc = upload(L.d_fw_leaf, v, st))) return rc;
    if ((rc = upload(L.d_fw_leaf_blk, blk, st))) return rc;
    L.n_fw_leaf = (int)v.size();
    L.b_fw_leaf = nblk;
    op->fw_built = true;
    return RS_OK;
}

template <class T>
int fwd_run_t(rs_op* op, const SolveLayout& Ls, const SolveWork& ws, const typename sc_traits<T>::io* xd,
              typename sc_traits<T>::io* yd, int64_t nrhs, cudaStream_t st)
{
    using IO = typename sc_traits<T>::io;
    const int64_t N = op->N;
    const int d = op->d;
    const std::vector<int64_t>& goff = Ls.goff;
    T* Gb = (T*)ws.g;
    T* Ph = (T*)ws.phi;
    T* U = (T*)ws.u;
    T* Z = (T*)ws.out;
    T* Ud = (T*)ws.w + Ls.woff[d] * nrhs;          // the leaf values of x, kept for the leaf blocks
    const int nr = (int)nrhs;
    const double* a = op->d_a.as<double>();
    auto mv = [&](const DevMem& probs, const DevMem& blk0, int np, int64_t nblk, int rb, const T* A, const T* x,
                  T* y) -> int {
        RS_CUDA(launch_matvec<T>(st, probs.as<MatvecProb>(), blk0.as<int64_t>(), np, nblk, A, x, y, nr, rb));
        return RS_OK;
    };
    int rc;
    for (int l = d; l >= 1; --l) {
        Level& L = op->lev[l];
        T* ul = U;
        if (l == d) {
            RS_CUDA(launch_gather_cm<IO, T>(st, L.sum_m, L.d_idx_leaf.as<int64_t>(), xd, N, Ud, nr));
            ul = Ud;
        } else {
            RS_CUDA(launch_gather_rows<T>(st, L.sum_m, L.d_idx_up.as<int64_t>(), Gb + goff[l + 1] * nrhs, U, nr));
        }
        T* gl = Gb + goff[l] * nrhs;
        RS_CUDA(launch_gather_rows<T>(st, L.sum_k, L.d_idx_sk.as<int64_t>(), ul, gl, nr));
        if ((rc = mv(L.d_mv_T, L.d_mv_T_blk, L.n_mv_T, L.b_mv_T, L.rb_T, L.d_T.as<T>(), ul, gl))) return rc;
    }
    {
        Level& R = op->lev[0];
        RS_CUDA(cudaMemsetAsync(Ph + goff[1] * nrhs, 0, sizeof(T) * (size_t)(op->lev[1].sum_k * nrhs), st));
        RS_CUDA(launch_kblock_mv<T>(st, R.d_fw_sib.as<KbProb>(), R.d_fw_sib_blk.as<int64_t>(), R.n_fw_sib, R.b_fw_sib,
                                    R.d_fw_pts.as<int32_t>(), Gb + goff[1] * nrhs, Ph + goff[1] * nrhs, nr, op->K, a));
    }
    for (int l = 1; l <= d; ++l) {
        Level& L = op->lev[l];
        T* pl = Ph + goff[l] * nrhs;
        RS_CUDA(launch_scatter_rows<T>(st, L.sum_k, L.d_idx_sk.as<int64_t>(), pl, Z, nr));
        if ((rc = mv(L.d_mv_Tt, L.d_mv_Tt_blk, L.n_mv_Tt, L.b_mv_Tt, L.rb_Tt, L.d_T.as<T>(), pl, Z))) return rc;
        if (l < d) {
            T* pc = Ph + goff[l + 1] * nrhs;
            RS_CUDA(launch_scatter_rows<T>(st, L.sum_m, L.d_idx_up.as<int64_t>(), Z, pc, nr));
            RS_CUDA(launch_kblock_mv<T>(st, L.d_fw_sib.as<KbProb>(), L.d_fw_sib_blk.as<int64_t>(), L.n_fw_sib,
                                        L.b_fw_sib, L.d_fw_pts.as<int32_t>(), Gb + goff[l + 1] * nrhs, pc, nr,
                                        op->K, a));
        } else {
            RS_CUDA(launch_kblock_mv<T>(st, L.d_fw_leaf.as<KbProb>(), L.d_fw_leaf_blk.as<int64_t>(), L.n_fw_leaf,
                                        L.b_fw_leaf, L.d_fw_leaf_pts.as<int32_t>(), Ud, Z, nr, op->K, a));
            RS_CUDA(launch_scatter_cm<T, IO>(st, L.sum_m, L.d_idx_leaf.as<int64_t>(), Z, N, yd, nr));
        }
    }
    return RS_OK;
}

int fwd_impl(rs_op* op, const void* x, int64_t nrhs, void* y, cudaStream_t st)
{
    const int64_t N = op->N;
    for (int l = 1; l <= op->d; ++l)
        if (!op->lev[l].cmp.empty())
            for (char c : op->lev[l].cmp)
                if (c) return fail(RS_E_INVALID, "the forward apply needs the dense T of every box (k_cut = 0)");
    const bool dev_x = is_device_ptr(x), dev_y = is_device_ptr(y);
    if (dev_x != dev_y) return fail(RS_E_INVALID, "x and y must both be device or both be host pointers");
    const size_t io = op->kind == RS_HELMHOLTZ ? 2 * sizeof(double) : sizeof(double);
    const double* xd = (const double*)x;
    double* yd = (double*)y;
    if (!dev_x) {
        RS_CUDA(op->s_in.alloc(io * (size_t)(N * nrhs)));
        RS_CUDA(cudaMemcpyAsync(op->s_in.p, x, io * (size_t)(N * nrhs), cudaMemcpyHostToDevice, st));
        xd = op->s_in.as<double>();
        RS_CUDA(op->s_out2.alloc(io * (size_t)(N * nrhs)));
        yd = op->s_out2.as<double>();
    }
    int rc = fw_plan(op, st);
    if (rc) return rc;
    SolveLayout Ls;
    SolveWork ws;
    if ((rc = solve_workspace(op, nrhs, Ls, ws))) return rc;
    using Zc = cplx<double>;
    if (op->kind == RS_HELMHOLTZ) {      // A = S A_s S^{-1}: the symmetric form between two scalings
        RS_CUDA(launch_scale_cm<Zc>(st, N, (int)nrhs, op->d_s_in.as<double>(), -1, (const Zc*)xd, op->s_fs.as<Zc>()));
        xd = op->s_fs.as<double>();
    }
    switch (op->opts.precision) {
        case RS_MIXED_FP32: rc = fwd_run_t<float>(op, Ls, ws, xd, yd, nrhs, st); break;
        case RS_C128: rc = fwd_run_t<cplx<double>>(op, Ls, ws, (const Zc*)xd, (Zc*)yd, nrhs, st); break;
        case RS_C64_REFINED: rc = fwd_run_t<cplx<float>>(op, Ls, ws, (const Zc*)xd, (Zc*)yd, nrhs, st); break;
        default: rc = fwd_run_t<double>(op, Ls, ws, xd, yd, nrhs, st); break;
    }
    if (rc) return rc;
    if (op->kind == RS_HELMHOLTZ)
        RS_CUDA(launch_scale_cm<Zc>(st, N, (int)nrhs, op->d_s_in.as<double>(), 1, (const Zc*)yd, (Zc*)yd));
    if (!dev_x) {
        RS_CUDA(cudaMemcpyAsync(y, yd, io * (size_t)(N * nrhs), cudaMemcpyDeviceToHost, st));
        RS_CUDA(cudaStreamSynchronize(st));
    }
    return RS_OK;
}

int solve_impl(rs_op* op, const void* f, int64_t nrhs, void* x, cudaStream_t st)
{
    const int64_t N = op->N;
    const bool dev_f = is_device_ptr(f), dev_x = is_device_ptr(x);
    if (dev_f != dev_x) return fail(RS_E_INVALID, "f and x must both be device or both be host pointers");
    if (op->opts.profile) {
        op->prof_ms[RS_PROF_SOLVE] = op->prof_work[RS_PROF_SOLVE] = op->prof_bytes[RS_PROF_SOLVE] = 0.0;
        op->prof_n[RS_PROF_SOLVE] = 0;
    }
    const size_t io = op->kind == RS_HELMHOLTZ ? 2 * sizeof(double) : sizeof(double);
    const double* fd = (const double*)f;
    double* xd = (double*)x;
    if (!dev_f) {
        RS_CUDA(op->s_in.alloc(io * (size_t)(N * nrhs)));
        RS_CUDA(cudaMemcpyAsync(op->s_in.p, f, io * (size_t)(N * nrhs), cudaMemcpyHostToDevice, st));
        fd = op->s_in.as<double>();
        RS_CUDA(op->s_out2.alloc(io * (size_t)(N * nrhs)));
        xd = op->s_out2.as<double>();
    }
    const bool refine = op->opts.precision == RS_MIXED_FP32 || op->opts.precision == RS_C64_REFINED;
    int rc = refine ? refine_solve(op, fd, xd, nrhs, st)
                    : op->opts.solve_graph ? apply_graph(op, fd, xd, nrhs, st) : apply_once(op, fd, xd, nrhs, st);
    if (rc && rc != RS_E_NOT_CONVERGED) return rc;
    if (!dev_x) {
        RS_CUDA(cudaMemcpyAsync(x, xd, io * (size_t)(N * nrhs), cudaMemcpyDeviceToHost, st));
        RS_CUDA(cudaStreamSynchronize(st));
    }
    if (op->opts.profile) {
        RS_CUDA(cudaStreamSynchronize(st));
        prof_flush(op);
    }
    return rc;
}

}  // namespace rs

using namespace rs;

extern "C" {

int rs_factor(const rs_tree* tree, const rs_kernel* kernel, const double* a, double eps, const rs_opts* opts,
              void* stream, rs_op** out)
{
    if (!out) return fail(RS_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!tree) return fail(RS_E_INVALID, "tree is NULL");
    return factor_impl(tree, kernel, a, eps, opts, (cudaStream_t)stream, out);
}

int rs_fwd_apply(rs_op* op, const void* x, int64_t nrhs, void* y, void* stream)
{
    if (!op || !x || !y || nrhs < 1) return fail(RS_E_INVALID, "bad argument");
    if (nrhs > (int64_t)1 << 20) return fail(RS_E_INVALID, "nrhs too large");
    if (x == y) return fail(RS_E_INVALID, "y may not alias x");
    int dev = 0;
    RS_CUDA(cudaGetDevice(&dev));
    if (dev != op->device) return fail(RS_E_INVALID, "the current device is not the one the operator was factored on");
    if (on_other_device(x) || on_other_device(y))
        return fail(RS_E_INVALID, "x or y is device memory of another GPU than the operator's");
    return fwd_impl(op, x, nrhs, y, (cudaStream_t)stream);
}

int rs_solve(rs_op* op, const void* f, int64_t nrhs, void* x, void* stream)
{
    if (!op || !f || !x || nrhs < 1) return fail(RS_E_INVALID, "bad argument");
    if (nrhs > (int64_t)1 << 20) return fail(RS_E_INVALID, "nrhs too large");
    if (f == x) return fail(RS_E_INVALID, "x may not alias f");
    if (op->opts.forward_only) return fail(RS_E_INVALID, "a forward-only operator has no inverse");
    int dev = 0;
    RS_CUDA(cudaGetDevice(&dev));
    if (dev != op->device) return fail(RS_E_INVALID, "the current device is not the one the operator was factored on");
    if (on_other_device(f) || on_other_device(x))
        return fail(RS_E_INVALID, "f or x is device memory of another GPU than the operator's");
    return solve_impl(op, f, nrhs, x, (cudaStream_t)stream);
}

int rs_free(rs_op* op)
{
    if (!op) return RS_OK;
    if (op->inflight.load() > 0) return fail(RS_E_INVALID, "the operator is still referenced by a server");
    delete op;
    return RS_OK;
}

int rs_op_profile_level(const rs_op* op, int cls, int level, double* ms)
{
    if (!op || !ms || cls < 0 || cls >= RS_PROF_COUNT || level < 0) return fail(RS_E_INVALID, "bad argument");
    const std::vector<double>& v = op->prof_level_ms[cls];
    *ms = level < (int)v.size() ? v[level] : 0.0;
    return RS_OK;
}

// Autotuner: time whole factorizations under each candidate setting and keep, for every
// level's launch shape, the fastest candidate of each kernel (the levels are independent
// launches, so their choices combine).
int rs_autotune(const rs_tree* tree, const rs_kernel* kernel, const double* a, double eps, const rs_opts* opts,
                void* stream, const char* path, rs_tune_report* report)
{
    if (!tree) return fail(RS_E_INVALID, "tree is NULL");
    rs_opts o;
    if (opts) o = *opts; else rs_opts_default(&o);
    o.profile = 1;
    o.k_cut = 0;
    const cudaStream_t st = (cudaStream_t)stream;
    // candidates: (CPQR group scale, CPQR variant (4 rows, 8 rows, look-ahead, cluster-resident,
    // register-capped, blocked), sweep group
    // scale, CPQR batch budget, sweep panel width); every sweep scale appears, and the CPQR
    // settings are picked per level as one triple, the sweep's as one pair
    const TuneTrial trials[] = {{1.0, 0, 1.0, 0.0}, {1.0, 1, 0.5, 0.0}, {1.0, 0, 0.25, 1.0},
                                {1.0, 1, 1.0, 1.0}, {0.5, 1, 0.5, 2.0}, {1.0, 1, 1.0, 2.0},
                                {1.0, 2, 1.0, 0.0}, {1.0, 2, 0.5, 1.0}, {2.0, 1, 1.0, 0.0}, {3.0, 0, 0.5, 0.0},
                                {1.0, 0, 1.0, 0.0, 16}, {1.0, 1, 0.5, 0.0, 16}, {1.0, 4, 1.0, 0.0},
                                {1.0, 6, 1.0, 0.0}, {1.0, 8, 1.0, 0.0}};
    constexpr int NTR = 15;
    auto timed_factor = [&](rs_op** op, double* ms) -> int {
        auto t0 = std::chrono::steady_clock::now();
        int rc = factor_impl(tree, kernel, a, eps, &o, st, op);
        if (rc) return rc;
        RS_CUDA(cudaStreamSynchronize(st));
        *ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        return RS_OK;
    };
    struct Shape {
        int nb;
        int64_t m, r, k;
    };
    std::vector<Shape> shapes;
    std::vector<std::vector<double>> t_cpqr(NTR), t_f(NTR), t_e(NTR);
    // per-level event times (CPQR, F^{-1} or root, E) of one factorization
    auto level_times = [&](rs_op* op, std::vector<double>& c, std::vector<double>& f, std::vector<double>& e) {
        const int d = op->d;
        c.assign(d + 1, 0.0);
        f.assign(d + 1, 0.0);
        e.assign(d + 1, 0.0);
        for (int l = 0; l <= d; ++l) {
            rs_op_profile_level(op, RS_PROF_CPQR, l, &c[l]);
            rs_op_profile_level(op, l == 0 ? RS_PROF_INV_ROOT : RS_PROF_INV_F, l, &f[l]);
            rs_op_profile_level(op, RS_PROF_INV_E, l, &e[l]);
        }
    };
    double base_ms = 0.0;
    std::vector<double> b_cpqr, b_f, b_e;
    g_trial = TuneTrial();
    {
        rs_op* op = nullptr;
        int rc = timed_factor(&op, &base_ms);
        if (rc) return rc;
        for (int l = 0; l <= op->d; ++l) {
            const Level& L = op->lev[l];
            shapes.push_back({L.nb, (int64_t)L.max_m, (int64_t)L.max_r, (int64_t)L.max_k});
        }
        level_times(op, b_cpqr, b_f, b_e);
        rs_free(op);
    }
    for (int t = 0; t < NTR; ++t) {
        g_trial = trials[t];
        rs_op* op = nullptr;
        double ms = 0.0;
        const int rc = timed_factor(&op, &ms);
        g_trial = TuneTrial();
        if (rc) return rc;
        level_times(op, t_cpqr[t], t_f[t], t_e[t]);
        rs_free(op);
    }
    int keys = 0;
    const int esz = (o.precision == RS_MIXED_FP32) ? 4 : (o.precision == RS_C64_REFINED) ? 8
                    : (kernel && kernel->kind == RS_HELMHOLTZ) ? 16 : 8;
    for (size_t l = 0; l < shapes.size(); ++l) {
        const Shape& S = shapes[l];
        auto best_of = [&](const std::vector<std::vector<double>>& tt) {
            int b = 0;
            for (int t = 1; t < NTR; ++t)
                if (l < tt[t].size() && tt[t][l] < tt[b][l]) b = t;
            return b;
        };
        if (l >= 1) {
            const int b = best_of(t_cpqr);
            const std::string k = tune_key("cpqr", esz, S.nb, S.m, S.r);
            // the built-in setting competes too
            const bool keep = l < b_cpqr.size() && l < t_cpqr[b].size() && b_cpqr[l] <= t_cpqr[b][l];
            tune_set(k + ".gscale", keep ? 1.0 : trials[b].cpqr_gscale);
            tune_set(k + ".deep", keep ? -1.0 : trials[b].cpqr_deep);
            tune_set(k + ".batch", keep ? 0.0 : trials[b].cpqr_batch);
            const int be = best_of(t_e);
            const std::string ke = tune_key("sweep", esz, S.nb, S.k, 0);
            tune_set(ke + ".gscale", trials[be].sweep_gscale);
            tune_set(ke + ".nb", trials[be].sweep_nb > 0 ? trials[be].sweep_nb : sweep_panel_width());
            keys += 5;
        }
        const int bf = best_of(t_f);
        const std::string kf = tune_key("sweep", esz, S.nb, S.m, 0);
        tune_set(kf + ".gscale", trials[bf].sweep_gscale);
        tune_set(kf + ".nb", trials[bf].sweep_nb > 0 ? trials[bf].sweep_nb : sweep_panel_width());
        keys += 2;
    }
    // Each candidate was timed once: check the picks in one factorization on the new table, and
    // give the built-in setting back to every level whose kernel came out more than 3% slower
    // than in the first factorization (a pick that owed its place to a lucky timing).
    {
        rs_op* op = nullptr;
        double ms = 0.0;
        int rc = timed_factor(&op, &ms);
        if (rc) return rc;
        std::vector<double> v_cpqr, v_f, v_e;
        level_times(op, v_cpqr, v_f, v_e);
        rs_free(op);
        for (size_t l = 0; l < shapes.size() && l < v_cpqr.size() && l < b_cpqr.size(); ++l) {
            const Shape& S = shapes[l];
            if (l >= 1 && v_cpqr[l] > 1.03 * b_cpqr[l]) {
                const std::string k = tune_key("cpqr", esz, S.nb, S.m, S.r);
                tune_set(k + ".gscale", 1.0);
                tune_set(k + ".deep", -1.0);
                tune_set(k + ".batch", 0.0);
            }
            if (l >= 1 && v_e[l] > 1.03 * b_e[l]) {
                tune_set(tune_key("sweep", esz, S.nb, S.k, 0) + ".gscale", 1.0);
                tune_set(tune_key("sweep", esz, S.nb, S.k, 0) + ".nb", sweep_panel_width());
            }
            if (v_f[l] > 1.03 * b_f[l]) {
                tune_set(tune_key("sweep", esz, S.nb, S.m, 0) + ".gscale", 1.0);
                tune_set(tune_key("sweep", esz, S.nb, S.m, 0) + ".nb", sweep_panel_width());
            }
        }
    }
    double tuned_ms = 0.0;
    {
        rs_op* op = nullptr;
        int rc = timed_factor(&op, &tuned_ms);
        if (rc) return rc;
        rs_free(op);
    }
    if (path) {
        int rc = rs_tune_save(path);
        if (rc) return rc;
    }
    if (report) {
        report->candidates = NTR;
        report->keys_set = keys;
        report->default_factor_ms = base_ms;
        report->tuned_factor_ms = tuned_ms;
    }
    return RS_OK;
}

int rs_op_profile(const rs_op* op, int cls, double* ms, double* work, double* bytes, int64_t* launches)
{
    if (!op || cls < 0 || cls >= RS_PROF_COUNT) return fail(RS_E_INVALID, "bad op or class");
    if (ms) *ms = op->prof_ms[cls];
    if (work) *work = op->prof_work[cls];
    if (bytes) *bytes = op->prof_bytes[cls];
    if (launches) *launches = op->prof_n[cls];
    return RS_OK;
}

int rs_op_stats(const rs_op* op, rs_stats* out)
{
    if (!op || !out) return fail(RS_E_INVALID, "NULL argument");
    *out = op->stats;
    // the solve workspace as it stands now (grown by rs_solve on demand; rs_solve_noalloc
    // never touches it)
    int64_t ws = 0;
    for (const DevMem* m : {&op->s_u, &op->s_w, &op->s_g, &op->s_phi, &op->s_t, &op->s_z, &op->s_in, &op->s_out,
                            &op->s_out2, &op->s_fs})
        ws += (int64_t)m->cap;
    out->bytes_workspace = ws;
    return RS_OK;
}

static const Level* get_level(const rs_op* op, int level, int box)
{
    if (!op || level < 1 || level > op->d || box < 0 || box >= (1 << level)) return nullptr;
    return &op->lev[level];
}

int rs_op_box_sizes(const rs_op* op, int level, int box, int64_t* m, int64_t* k, int64_t* r, int64_t* nnear)
{
    const Level* L = get_level(op, level, box);
    if (!L) return fail(RS_E_INVALID, "level/box out of range");
    if (m) *m = L->m[box];
    if (k) *k = L->k[box];
    if (r) *r = L->r[box];
    if (nnear) *nnear = L->nn[box];
    return RS_OK;
}

int rs_op_box_indices(const rs_op* op, int level, int box, int which, int64_t* out)
{
    const Level* L = get_level(op, level, box);
    if (!L || !out) return fail(RS_E_INVALID, "level/box out of range");
    if (which == 0) {
        std::copy(L->act.begin() + L->act_off[box], L->act.begin() + L->act_off[box + 1], out);
    } else if (which == 1) {
        if (op->opts.translation_invariant == 1)  // the level's near rows are its template's
            return fail(RS_E_INVALID, "no per-box near list in translation-invariant mode");
        std::copy(L->nearv.begin() + L->near_off[box], L->nearv.begin() + L->near_off[box + 1], out);
    } else if (which == 2) {
        std::copy(L->skel.begin() + L->k_off[box], L->skel.begin() + L->k_off[box + 1], out);
    } else {
        return fail(RS_E_INVALID, "bad `which`");
    }
    return RS_OK;
}

// Copy n entries of the factor storage (FP64 or FP32) at element offset `off` into doubles.
static int fetch(const rs_op* op, const DevMem& d, int64_t off, int64_t n, std::vector<double>& out)
{
    out.assign((size_t)n, 0.0);
    if (n == 0) return RS_OK;
    if (op->kind == RS_HELMHOLTZ) {      // complex storage: n counts doubles (re, im pairs)
        const int64_t e0 = 2 * off;
        if (op->esz == 2 * (int)sizeof(double)) {
            RS_CUDA(cudaMemcpy(out.data(), d.as<double>() + e0, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost));
        } else {
            std::vector<float> t((size_t)n);
            RS_CUDA(cudaMemcpy(t.data(), d.as<float>() + e0, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < t.size(); ++i) out[i] = t[i];
        }
        return RS_OK;
    }
    if (op->esz == (int)sizeof(double)) {
        RS_CUDA(cudaMemcpy(out.data(), d.as<double>() + off, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> t((size_t)n);
        RS_CUDA(cudaMemcpy(t.data(), d.as<float>() + off, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < t.size(); ++i) out[i] = t[i];
    }
    return RS_OK;
}

int rs_op_box_matrix(const rs_op* op, int level, int box, int which, double* out)
{
    const Level* L = get_level(op, level, box);
    if (!L || !out) return fail(RS_E_INVALID, "level/box out of range");
    if (L->dense_freed) return fail(RS_E_INVALID, "the dense blocks of this level were released after compression");
    const int64_t m = L->m[box], k = L->k[box];
    const int c = op->kind == RS_HELMHOLTZ ? 2 : 1;     // doubles per entry
    RS_CUDA(cudaSetDevice(op->device));
    std::vector<double> t;
    int rc;
    if (which == 0) {
        if ((rc = fetch(op, L->d_T, L->t_off[box], c * k * (m - k), t))) return rc;
        for (int64_t i = 0; i < k; ++i)
            for (int64_t j = 0; j < m - k; ++j)
                for (int q = 0; q < c; ++q) out[(i * (m - k) + j) * c + q] = t[(size_t)((j * k + i) * c + q)];
    } else if (which == 1) {
        if ((rc = fetch(op, L->d_Phi, L->phi_off[box], c * m * m, t))) return rc;
        const int32_t* pm = L->perm.data() + L->act_off[box];
        for (int64_t qq = 0; qq < m; ++qq)
            for (int64_t p = 0; p < m; ++p)
                for (int q = 0; q < c; ++q) out[((int64_t)pm[p] * m + pm[qq]) * c + q] = t[(size_t)((qq * m + p) * c + q)];
    } else if (which == 2) {
        if ((rc = fetch(op, L->d_E, L->e_off[box], c * k * k, t))) return rc;
        for (int64_t i = 0; i < k; ++i)
            for (int64_t j = 0; j < k; ++j)
                for (int q = 0; q < c; ++q) out[(i * k + j) * c + q] = t[(size_t)((j * k + i) * c + q)];
    } else {
        return fail(RS_E_INVALID, "bad `which`");
    }
    return RS_OK;
}

int rs_op_root_matrix(const rs_op* op, double* out)
{
    if (!op || !out) return fail(RS_E_INVALID, "NULL argument");
    const Level& R = op->lev[0];
    const int64_t m = R.m[0];
    const int c = op->kind == RS_HELMHOLTZ ? 2 : 1;
    RS_CUDA(cudaSetDevice(op->device));
    std::vector<double> t;
    const int rc = fetch(op, R.d_Phi, 0, c * m * m, t);
    if (rc) return rc;
    for (int64_t qq = 0; qq < m; ++qq)
        for (int64_t p = 0; p < m; ++p)
            for (int q = 0; q < c; ++q) out[(p * m + qq) * c + q] = t[(size_t)((qq * m + p) * c + q)];
    return RS_OK;
}

}  // extern "C"
