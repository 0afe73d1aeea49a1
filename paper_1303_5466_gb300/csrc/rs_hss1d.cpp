// rs_hss1d.cpp -- the extra compression of Sec. 3 for boxes with k > k_cut, built from the
// explicit dense blocks of the factorization:
//   - phi^{sk} and phi^{rs} (the diagonal blocks of Phi = Pi^T F^{-1} Pi) and E in HSS1D form
//     (Sec. 3.2: a binary tree over halving runs of the 1D orders of Sec. 3.1, one ID per node
//     of its block column and transposed block row, and the telescoping form of Eq. 2.9);
//   - phi^{s<-r}, phi^{r<-s} and T in low-rank form (column ID);
//   - the inverse apply (Algorithm 6) then uses these forms for those boxes: each form is
//     applied by a short program of row copies and batched matvecs on a scratch buffer, all
//     forms of a level sharing each launch.
// The IDs run in the factorization's column-pivoted QR and T kernels; the new kernels are in
// k_hss1d.cu.  Also here: the standalone HSS1D entry points (rs_hss1d_*).
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <memory>
#include <new>
#include <numeric>
#include <tuple>

#include "rs_host.h"

namespace rs {

// ------------------------------------------------------------------ orders of Sec. 3.1

// Skeleton points by angle about the box centre, counter-clockwise from the positive x1
// axis; points on one ray by distance, then grid index.  Offsets are integers in units of
// h/2, so every comparison is exact.
std::vector<int> cyclic_order(int64_t n, int l, int64_t j, const int64_t* g, int cnt)
{
    const BoxInt bi = box_int(n, l, j);
    const int64_t cx2 = (2 * bi.bx + 1) * bi.wx, cy2 = (2 * bi.by + 1) * bi.wy;
    struct P { int64_t dx, dy, g; int idx; };
    std::vector<P> v(cnt);
    for (int i = 0; i < cnt; ++i) v[i] = {2 * (g[i] % n) + 1 - cx2, 2 * (g[i] / n) + 1 - cy2, g[i], i};
    auto lower = [](const P& p) { return p.dy < 0 || (p.dy == 0 && p.dx < 0); };   // angle in [pi, 2 pi)
    std::sort(v.begin(), v.end(), [&](const P& a, const P& b) {
        const bool ha = lower(a), hb = lower(b);
        if (ha != hb) return hb;
        const int64_t cr = a.dx * b.dy - a.dy * b.dx;        // > 0: b lies counter-clockwise of a
        if (cr != 0) return cr > 0;
        const int64_t ra = a.dx * a.dx + a.dy * a.dy, rb = b.dx * b.dx + b.dy * b.dy;
        if (ra != rb) return ra < rb;
        return a.g < b.g;
    });
    std::vector<int> o(cnt);
    for (int i = 0; i < cnt; ++i) o[i] = v[i].idx;
    return o;
}

// A box at even depth splits along x1, so the interface between its children runs along x2:
// order by (i2, i1); at odd depth by (i1, i2).
std::vector<int> interface_order(int64_t n, int l, const int64_t* g, int cnt)
{
    std::vector<int> o(cnt);
    std::iota(o.begin(), o.end(), 0);
    const bool even = (l % 2) == 0;
    auto key = [&](int i) {
        const int64_t i1 = g[i] % n, i2 = g[i] / n;
        return even ? std::make_pair(i2, i1) : std::make_pair(i1, i2);
    };
    std::sort(o.begin(), o.end(), [&](int a, int b) { return key(a) < key(b); });
    return o;
}

// ------------------------------------------------------------------ compression

namespace {

template <class V>
int upload_vec(DevMem& d, const std::vector<V>& h, cudaStream_t st)
{
    RS_CUDA(d.alloc(sizeof(V) * (h.empty() ? 1 : h.size())));
    if (!h.empty()) RS_CUDA(cudaMemcpyAsync(d.p, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice, st));
    return RS_OK;
}

int check_ctx(const IdCtx& ctx, cudaStream_t st)
{
    RS_CUDA(cudaStreamSynchronize(st));
    int s = 0;
    RS_CUDA(cudaMemcpy(&s, ctx.status, sizeof(int), cudaMemcpyDeviceToHost));
    if (s & DEV_TIMEOUT) return fail(RS_E_TIMEOUT, "a device-side wait exceeded spin_limit");
    if (s & DEV_SINGULAR) return fail(RS_E_SINGULAR, "pivot below 1e3 unit roundoff times the largest earlier pivot");
    if (s & DEV_BADSIZE) return fail(RS_E_CUDA, "a kernel found an out-of-range index and stopped");
    return RS_OK;
}

int hss_depth(int n, int leaf)
{
    int t = 0;
    while (((int64_t)n + ((int64_t)1 << t) - 1) >> t > leaf) ++t;
    return t;
}

constexpr int MAX_GRID_Y = 65535;

// One ID of a batch: node q of form f; r rows; mode 0 = HSS1D node, 1 = low-rank block.
struct IdJob {
    CForm* f;
    CNode* q;
    int r, mode;
    std::vector<int> out;
};

}  // namespace

template <class T>
int compress_forms(const IdCtx& ctx, cudaStream_t st, std::vector<CForm*>& forms, double eps, int leaf, DevMem& store,
                   int64_t& store_n)
{
    if (leaf < 1) return fail(RS_E_INVALID, "HSS1D leaf size must be at least 1");
    int maxT = 0;
    for (CForm* f : forms) {
        f->lev.clear();
        f->b12.clear(); f->b21.clear(); f->d_off.clear();
        if (f->hss) {
            if (f->rows != f->cols || (int)f->order.size() != f->rows) return fail(RS_E_INVALID, "bad HSS1D form");
            const int n = f->rows, t = hss_depth(n, leaf);
            f->depth = t;
            f->lev.assign(t + 1, {});
            if (t == 0) {
                CNode q;
                q.lo = 0; q.hi = n; q.a = n; q.k = 0;
                q.act = f->order;
                q.perm.resize(n);
                std::iota(q.perm.begin(), q.perm.end(), 0);
                f->lev[0].push_back(std::move(q));
            }
            for (int l = 1; l <= t; ++l) {
                f->lev[l].resize((size_t)1 << l);
                for (int j = 0; j < (1 << l); ++j) {
                    f->lev[l][j].lo = (int)(((int64_t)j * n) >> l);
                    f->lev[l][j].hi = (int)(((int64_t)(j + 1) * n) >> l);
                }
            }
            maxT = std::max(maxT, t);
        } else {
            f->depth = 0;
            f->lev.assign(1, std::vector<CNode>(1));
            CNode& q = f->lev[0][0];
            q.a = f->cols;
            q.act.resize(f->cols);
            std::iota(q.act.begin(), q.act.end(), 0);
        }
    }
    std::vector<DevMem> tbufs;
    int64_t t_total = 0;
    for (int h = 0; h < std::max(maxT, 1); ++h) {
        std::vector<IdJob> jobs;
        for (CForm* f : forms) {
            if (f->hss) {
                if (f->depth == 0 || f->depth - h < 1) continue;
                const int l = f->depth - h;
                for (int j = 0; j < (1 << l); ++j) {
                    CNode& q = f->lev[l][j];
                    q.act.clear();
                    if (l == f->depth) {
                        q.act.assign(f->order.begin() + q.lo, f->order.begin() + q.hi);
                    } else {
                        for (int c = 0; c < 2; ++c) {
                            const CNode& ch = f->lev[l + 1][2 * j + c];
                            for (int i = 0; i < ch.k; ++i) q.act.push_back(ch.act[ch.perm[i]]);
                        }
                    }
                    q.a = (int)q.act.size();
                    IdJob jb{f, &q, 0, 0, {}};
                    for (int p = 0; p < f->rows; ++p)
                        if (p < q.lo || p >= q.hi) jb.out.push_back(f->order[p]);
                    jb.r = 2 * (int)jb.out.size();
                    jobs.push_back(std::move(jb));
                }
            } else if (h == 0) {
                jobs.push_back(IdJob{f, &f->lev[0][0], f->rows, 1, {}});
            }
        }
        std::vector<IdJob*> run;
        for (IdJob& jb : jobs) {
            if (jb.q->a == 0 || jb.r == 0) {
                jb.q->k = 0;
                jb.q->perm.resize(jb.q->a);
                std::iota(jb.q->perm.begin(), jb.q->perm.end(), 0);
                jb.q->t_off = 0;
            } else {
                run.push_back(&jb);
            }
        }
        if (run.empty()) continue;
        const int nb = (int)run.size();
        std::vector<int32_t> lists, nn(nb);
        std::vector<ZProb> zp(nb);
        std::vector<int64_t> act_off(nb + 1, 0), y_off(nb + 1, 0);
        int max_r = 0, max_m = 0;
        int64_t max_el = 0;
        for (int b = 0; b < nb; ++b) {
            const IdJob& jb = *run[b];
            ZProb& z = zp[b];
            z.M = jb.f->M;
            z.ld = jb.f->ld;
            z.a = jb.q->a;
            z.mode = jb.mode;
            z.nout = jb.mode == 0 ? (int)jb.out.size() : jb.r;
            z.act_off = (int64_t)lists.size();
            lists.insert(lists.end(), jb.q->act.begin(), jb.q->act.end());
            z.out_off = (int64_t)lists.size();
            lists.insert(lists.end(), jb.out.begin(), jb.out.end());
            z.y_off = y_off[b];
            nn[b] = jb.r;
            act_off[b + 1] = act_off[b] + jb.q->a;
            y_off[b + 1] = y_off[b] + (int64_t)jb.r * jb.q->a;
            max_r = std::max(max_r, jb.r);
            max_m = std::max(max_m, jb.q->a);
            max_el = std::max<int64_t>(max_el, (int64_t)jb.r * jb.q->a);
        }
        DevMem d_lists, d_zp, d_act_off, d_y_off, d_nn, Y, piv, diag, kk, keys, norms;
        int rc;
        if ((rc = upload_vec(d_lists, lists, st))) return rc;
        if ((rc = upload_vec(d_zp, zp, st))) return rc;
        if ((rc = upload_vec(d_act_off, act_off, st))) return rc;
        if ((rc = upload_vec(d_y_off, y_off, st))) return rc;
        if ((rc = upload_vec(d_nn, nn, st))) return rc;
        RS_CUDA(Y.alloc(sizeof(T) * (size_t)(y_off[nb] + 1)));
        for (int b0 = 0; b0 < nb; b0 += MAX_GRID_Y)
            RS_CUDA(launch_zgather<T>(st, d_zp.as<ZProb>() + b0, std::min(MAX_GRID_Y, nb - b0), d_lists.as<int32_t>(),
                                      Y.as<T>(), max_el));
        const int64_t sum_a = act_off[nb];
        RS_CUDA(piv.alloc(sizeof(int32_t) * (size_t)(sum_a + 1)));
        RS_CUDA(diag.alloc(sizeof(T) * (size_t)(sum_a + 1)));
        RS_CUDA(kk.alloc(sizeof(int32_t) * (size_t)nb));
        RS_CUDA(ctx.bar->alloc(sizeof(unsigned int) * (size_t)nb));
        RS_CUDA(cudaMemsetAsync(ctx.bar->p, 0, sizeof(unsigned int) * (size_t)nb, st));
        const int G = choose_group(nb, max_m, [&](int g) { return cpqr_max_ctas<T>(max_r, max_m, g); });
        RS_CUDA(keys.alloc(sizeof(unsigned long long) * 2 * (size_t)nb * G));
        RS_CUDA(norms.alloc(sizeof(double) * 2 * (size_t)(sum_a + 1)));
        RS_CUDA(launch_cpqr<T>(st, nb, G, nullptr, 0, 0, d_act_off.as<int64_t>(), d_nn.as<int32_t>(), 0, d_y_off.as<int64_t>(),
                               Y.as<T>(), eps, kk.as<int32_t>(), piv.as<int32_t>(), diag.as<T>(),
                               ctx.bar->as<unsigned int>(), keys.as<unsigned long long>(), ctx.status, ctx.spin,
                               max_r, max_m, norms.as<double>(), norms.as<double>() + sum_a + 1));
        if ((rc = check_ctx(ctx, st))) return rc;
        std::vector<int32_t> k32(nb), ph((size_t)sum_a);
        RS_CUDA(cudaMemcpy(k32.data(), kk.p, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost));
        RS_CUDA(cudaMemcpy(ph.data(), piv.p, sizeof(int32_t) * (size_t)sum_a, cudaMemcpyDeviceToHost));
        std::vector<int32_t> skpos((size_t)sum_a + 1, 0), rscol((size_t)sum_a + 1, 0);
        std::vector<int64_t> t_off(nb + 1, 0);
        int max_res = 0, max_k = 0;
        for (int b = 0; b < nb; ++b) {
            CNode& q = *run[b]->q;
            const int64_t a0 = act_off[b];
            const int a = q.a, k = k32[b];
            if (k < 0 || k > a) return fail(RS_E_CUDA, "bad rank from the ID kernel");
            std::vector<int> ord(k);
            std::iota(ord.begin(), ord.end(), 0);
            std::sort(ord.begin(), ord.end(), [&](int x, int y) { return ph[a0 + x] < ph[a0 + y]; });
            std::vector<char> is_sk(a, 0);
            q.k = k;
            q.perm.assign(a, 0);
            for (int s = 0; s < k; ++s) {
                const int loc = ph[a0 + ord[s]];
                if (loc < 0 || loc >= a || is_sk[loc]) return fail(RS_E_CUDA, "bad pivot from the ID kernel");
                is_sk[loc] = 1;
                skpos[a0 + ord[s]] = s;
                q.perm[s] = loc;
            }
            int c = 0;
            for (int loc = 0; loc < a; ++loc)
                if (!is_sk[loc]) { rscol[a0 + c] = loc; q.perm[k + c] = loc; ++c; }
            t_off[b + 1] = t_off[b] + (int64_t)k * (a - k);
            q.t_off = t_total + t_off[b];
            max_res = std::max(max_res, a - k);
            max_k = std::max(max_k, k);
        }
        DevMem d_skpos, d_rscol, d_toff, Tb;
        if ((rc = upload_vec(d_skpos, skpos, st))) return rc;
        if ((rc = upload_vec(d_rscol, rscol, st))) return rc;
        if ((rc = upload_vec(d_toff, t_off, st))) return rc;
        RS_CUDA(Tb.alloc(sizeof(T) * (size_t)(t_off[nb] + 1)));
        RS_CUDA(launch_id_T<T>(st, nb, d_act_off.as<int64_t>(), kk.as<int32_t>(), d_nn.as<int32_t>(), 0,
                               d_y_off.as<int64_t>(), Y.as<T>(), piv.as<int32_t>(), diag.as<T>(),
                               d_skpos.as<int32_t>(), d_rscol.as<int32_t>(), d_toff.as<int64_t>(), Tb.as<T>(), max_res,
                               max_k));
        if ((rc = check_ctx(ctx, st))) return rc;
        t_total += t_off[nb];
        tbufs.push_back(std::move(Tb));
    }
    // store: T blocks (in the order above), then sibling, leaf and skeleton-column blocks
    int64_t off = t_total;
    std::vector<SubProb> sp;
    std::vector<int32_t> lists;
    auto add_sub = [&](const CForm* f, const std::vector<int>* rows, int nrow, const std::vector<int>& cols,
                       int64_t dst) {
        SubProb s{};
        s.M = f->M; s.ld = f->ld; s.rows = nrow; s.cols = (int)cols.size(); s.dst_off = dst;
        if (rows) { s.row_off = (int64_t)lists.size(); lists.insert(lists.end(), rows->begin(), rows->end()); }
        else s.row_off = -1;
        s.col_off = (int64_t)lists.size();
        lists.insert(lists.end(), cols.begin(), cols.end());
        if (s.rows > 0 && s.cols > 0) sp.push_back(s);
    };
    auto skel_rows = [](const CNode& q) {
        std::vector<int> v(q.k);
        for (int i = 0; i < q.k; ++i) v[i] = q.act[q.perm[i]];
        return v;
    };
    for (CForm* f : forms) {
        if (f->hss) {
            const int t = f->depth;
            const int nint = t == 0 ? 0 : (1 << t) - 1;
            f->b12.assign(nint, 0);
            f->b21.assign(nint, 0);
            for (int l = 0; l < t; ++l)
                for (int j = 0; j < (1 << l); ++j) {
                    const CNode& c1 = f->lev[l + 1][2 * j];
                    const CNode& c2 = f->lev[l + 1][2 * j + 1];
                    const std::vector<int> s1 = skel_rows(c1), s2 = skel_rows(c2);
                    const int hi = (1 << l) - 1 + j;
                    f->b12[hi] = off;
                    add_sub(f, &s1, c1.k, s2, off);
                    off += (int64_t)c1.k * c2.k;
                    f->b21[hi] = off;
                    add_sub(f, &s2, c2.k, s1, off);
                    off += (int64_t)c2.k * c1.k;
                }
            std::vector<CNode>& leaves = f->lev[t];
            f->d_off.assign(leaves.size(), 0);
            for (size_t j = 0; j < leaves.size(); ++j) {
                const CNode& q = leaves[j];
                std::vector<int> pa(q.a);
                for (int i = 0; i < q.a; ++i) pa[i] = q.act[q.perm[i]];
                f->d_off[j] = off;
                add_sub(f, &pa, q.a, pa, off);
                off += (int64_t)q.a * q.a;
            }
        } else {
            const CNode& q = f->lev[0][0];
            std::vector<int> sk(q.perm.begin(), q.perm.begin() + q.k);
            f->c_off = off;
            add_sub(f, nullptr, f->rows, sk, off);
            off += (int64_t)f->rows * q.k;
        }
    }
    store_n = off;
    RS_CUDA(store.alloc(sizeof(T) * (size_t)(off + 1)));
    int64_t pos = 0;
    for (DevMem& tb : tbufs) {
        const size_t bytes = tb.bytes - sizeof(T);   // allocated with one spare element
        if (bytes) RS_CUDA(cudaMemcpyAsync(store.as<T>() + pos, tb.p, bytes, cudaMemcpyDeviceToDevice, st));
        pos += (int64_t)(bytes / sizeof(T));
    }
    if (pos != t_total) return fail(RS_E_CUDA, "compressed store: T blocks do not add up");
    if (!sp.empty()) {
        DevMem d_sp, d_lists;
        int rc;
        if ((rc = upload_vec(d_sp, sp, st))) return rc;
        if ((rc = upload_vec(d_lists, lists, st))) return rc;
        int64_t max_el = 0;
        for (const SubProb& s : sp) max_el = std::max<int64_t>(max_el, (int64_t)s.rows * s.cols);
        for (size_t b0 = 0; b0 < sp.size(); b0 += MAX_GRID_Y)
            RS_CUDA(launch_subgather<T>(st, d_sp.as<SubProb>() + b0, (int)std::min<size_t>(MAX_GRID_Y, sp.size() - b0),
                                        d_lists.as<int32_t>(), store.as<T>(), max_el));
        RS_CUDA(cudaStreamSynchronize(st));
    }
    for (CForm* f : forms) {
        int64_t e = 0;
        for (const std::vector<CNode>& lv : f->lev)
            for (const CNode& q : lv) e += (int64_t)q.k * (q.a - q.k);
        if (f->hss) {
            const int t = f->depth;
            for (int l = 0; l < t; ++l)
                for (int j = 0; j < (1 << l); ++j) e += 2 * (int64_t)f->lev[l + 1][2 * j].k * f->lev[l + 1][2 * j + 1].k;
            for (const CNode& q : f->lev[t]) e += (int64_t)q.a * q.a;
        } else {
            e += (int64_t)f->rows * f->lev[0][0].k;
        }
        f->entries = e;
        f->M = nullptr;
    }
    return RS_OK;
}

template int compress_forms<double>(const IdCtx&, cudaStream_t, std::vector<CForm*>&, double, int, DevMem&, int64_t&);
template int compress_forms<float>(const IdCtx&, cudaStream_t, std::vector<CForm*>&, double, int, DevMem&, int64_t&);
template int compress_forms<cplx<double>>(const IdCtx&, cudaStream_t, std::vector<CForm*>&, double, int, DevMem&,
                                          int64_t&);
template int compress_forms<cplx<float>>(const IdCtx&, cudaStream_t, std::vector<CForm*>&, double, int, DevMem&,
                                         int64_t&);

// ------------------------------------------------------------------ apply programs
//
// A form is applied to the rows in_rows[] of an input buffer (nrhs columns, point-major) and
// written (or added) to the rows out_rows[] of an output buffer, through scratch rows Z.
// HSS1D (Eq. 2.9), for each node q with active set act_q in pivot order (skeleton, residual):
//   up    (leaves first)  X_q = x(act_q) [leaf] or the children's XH [internal];
//                         XH_q = X_q[sk] + T_q X_q[rs]   (in place above the leaves)
//   root                  YH_c1 = B12 XH_c2,  YH_c2 = B21 XH_c1  (children of the root)
//   down                  Y_q[rs] = T_q^T YH_q; at a leaf Y_q += D_q X_q, else the children's
//                         YH take their rows of Y_q and add the sibling terms B XH
//   final                 y(act_q) = Y_q at the leaves.
// Low rank X ~ C [I T] Pi^T:  XH = v[sk] + T v[rs], y = C XH; transposed: YH = C^T v,
// y[sk] = YH, y[rs] = T^T YH.
// Every step of every form is filed under a slot key (phase, level, step, buffers); the slots
// become the launches, in key order, so that one launch serves the same step of all forms.

namespace {

constexpr int MAXL = 1000;
enum { BUF_IN = 0, BUF_OUT = 1, BUF_Z = 2 };

struct SlotKey {
    int phase, lvl, sub, kind, src, dst, add;
    bool operator<(const SlotKey& o) const
    {
        return std::tie(phase, lvl, sub, kind, src, dst, add) <
               std::tie(o.phase, o.lvl, o.sub, o.kind, o.src, o.dst, o.add);
    }
};
struct Slot {
    std::vector<int64_t> s, d;
    std::vector<MatvecProb> mv;
};

struct Builder {
    std::map<SlotKey, Slot> slots;
    int64_t z = 0;
    int64_t zalloc(int64_t rows) { const int64_t r = z; z += rows; return r; }
    void copy(int phase, int lvl, int sub, int src, int dst, int add, int64_t s, int64_t d)
    {
        Slot& sl = slots[SlotKey{phase, lvl, sub, 0, src, dst, add}];
        sl.s.push_back(s);
        sl.d.push_back(d);
    }
    void mv(int phase, int lvl, int sub, int rows, int cols, int ld, int trans, int64_t a_off, int64_t x_off,
            int64_t y_off, double beta)
    {
        const int out_n = trans ? cols : rows;
        if (out_n <= 0) return;
        MatvecProb p{};
        p.rows = rows; p.cols = cols; p.ld = std::max(ld, 1); p.trans = trans;
        p.a_off = a_off; p.x_off = x_off; p.y_off = y_off; p.alpha = 1.0; p.beta = beta;
        slots[SlotKey{phase, lvl, sub, 1, BUF_Z, BUF_Z, 0}].mv.push_back(p);
    }
};

int up_key(int l) { return MAXL - l; }

void add_hss(Builder& B, const ProgItem& it)
{
    const CForm& f = *it.f;
    const int t = f.depth;
    const int l0 = t == 0 ? 0 : 1;
    // scratch rows per node: X (a rows), XH (k rows, leaves only), Y (a rows)
    std::vector<std::vector<int64_t>> zx(t + 1), zxh(t + 1), zy(t + 1);
    for (int l = l0; l <= t; ++l) {
        const size_t nn = f.lev[l].size();
        zx[l].resize(nn); zxh[l].resize(nn); zy[l].resize(nn);
        for (size_t j = 0; j < nn; ++j) {
            const CNode& q = f.lev[l][j];
            zx[l][j] = B.zalloc(q.a);
            zxh[l][j] = (l == t) ? B.zalloc(q.k) : zx[l][j];
            zy[l][j] = B.zalloc(q.a);
        }
    }
    const int fin = it.add ? 1 : 0;
    for (int l = t; l >= l0; --l)
        for (size_t j = 0; j < f.lev[l].size(); ++j) {
            const CNode& q = f.lev[l][j];
            if (l == t) {
                for (int i = 0; i < q.a; ++i) B.copy(0, up_key(l), 0, BUF_IN, BUF_Z, 0, it.in_rows[q.act[q.perm[i]]], zx[l][j] + i);
                for (int i = 0; i < q.k; ++i) B.copy(0, up_key(l), 0, BUF_IN, BUF_Z, 0, it.in_rows[q.act[q.perm[i]]], zxh[l][j] + i);
            } else {
                const int k1 = f.lev[l + 1][2 * j].k;
                for (int i = 0; i < q.a; ++i) {
                    const int loc = q.perm[i];
                    const int64_t src = loc < k1 ? zxh[l + 1][2 * j] + loc : zxh[l + 1][2 * j + 1] + (loc - k1);
                    B.copy(0, up_key(l), 1, BUF_Z, BUF_Z, 0, src, zx[l][j] + i);
                }
            }
            if (q.k > 0 && q.a > q.k)
                B.mv(0, up_key(l), 2, q.k, q.a - q.k, q.k, 0, q.t_off, zx[l][j] + q.k, zxh[l][j], 1.0);
        }
    if (t >= 1) {
        const CNode& c1 = f.lev[1][0];
        const CNode& c2 = f.lev[1][1];
        B.mv(1, 0, 0, c1.k, c2.k, c1.k, 0, f.b12[0], zxh[1][1], zy[1][0], 0.0);
        B.mv(1, 0, 0, c2.k, c1.k, c2.k, 0, f.b21[0], zxh[1][0], zy[1][1], 0.0);
    }
    for (int l = l0; l <= t; ++l)
        for (size_t j = 0; j < f.lev[l].size(); ++j) {
            const CNode& q = f.lev[l][j];
            B.mv(2, l, 0, q.k, q.a - q.k, q.k, 1, q.t_off, zy[l][j], zy[l][j] + q.k, 0.0);
            if (l == t) {
                B.mv(2, l, 1, q.a, q.a, q.a, 0, f.d_off[j], zx[l][j], zy[l][j], 1.0);
                for (int i = 0; i < q.a; ++i) B.copy(3, 0, fin, BUF_Z, BUF_OUT, it.add, zy[l][j] + i, it.out_rows[q.act[q.perm[i]]]);
            } else {
                std::vector<int> pinv(q.a);
                for (int i = 0; i < q.a; ++i) pinv[q.perm[i]] = i;
                const CNode& c1 = f.lev[l + 1][2 * j];
                const CNode& c2 = f.lev[l + 1][2 * j + 1];
                for (int i = 0; i < c1.k; ++i) B.copy(2, l, 2, BUF_Z, BUF_Z, 0, zy[l][j] + pinv[i], zy[l + 1][2 * j] + i);
                for (int i = 0; i < c2.k; ++i)
                    B.copy(2, l, 2, BUF_Z, BUF_Z, 0, zy[l][j] + pinv[c1.k + i], zy[l + 1][2 * j + 1] + i);
                const int hi = (1 << l) - 1 + (int)j;
                B.mv(2, l, 3, c1.k, c2.k, c1.k, 0, f.b12[hi], zxh[l + 1][2 * j + 1], zy[l + 1][2 * j], 1.0);
                B.mv(2, l, 3, c2.k, c1.k, c2.k, 0, f.b21[hi], zxh[l + 1][2 * j], zy[l + 1][2 * j + 1], 1.0);
            }
        }
}

void add_lr(Builder& B, const ProgItem& it, int tmax)
{
    const CForm& f = *it.f;
    const CNode& q = f.lev[0][0];
    const int p = f.rows, qn = f.cols, k = q.k;
    const int fin = it.add ? 1 : 0;
    const int u = up_key(tmax);
    if (!it.trans) {
        const int64_t zx = B.zalloc(qn), zy = B.zalloc(p);
        for (int i = 0; i < qn; ++i) B.copy(0, u, 0, BUF_IN, BUF_Z, 0, it.in_rows[q.perm[i]], zx + i);
        if (k > 0 && qn > k) B.mv(0, u, 2, k, qn - k, k, 0, q.t_off, zx + k, zx, 1.0);
        B.mv(1, 0, 0, p, k, p, 0, f.c_off, zx, zy, 0.0);
        for (int i = 0; i < p; ++i) B.copy(3, 0, fin, BUF_Z, BUF_OUT, it.add, zy + i, it.out_rows[i]);
    } else {
        const int64_t zx = B.zalloc(p), zy = B.zalloc(qn);
        for (int i = 0; i < p; ++i) B.copy(0, u, 0, BUF_IN, BUF_Z, 0, it.in_rows[i], zx + i);
        B.mv(0, u, 2, p, k, p, 1, f.c_off, zx, zy, 0.0);
        B.mv(1, 0, 0, k, qn - k, k, 1, q.t_off, zy, zy + k, 0.0);
        for (int i = 0; i < qn; ++i) B.copy(3, 0, fin, BUF_Z, BUF_OUT, it.add, zy + i, it.out_rows[q.perm[i]]);
    }
}

}  // namespace

int build_program(std::vector<ProgItem>& items, cudaStream_t st, Program& prog)
{
    prog = Program();
    Builder B;
    int tmax = 0;
    for (const ProgItem& it : items)
        if (it.f->hss) tmax = std::max(tmax, it.f->depth);
    for (const ProgItem& it : items) {
        const CForm& f = *it.f;
        if (f.rows == 0 || f.cols == 0) continue;
        const size_t nin = it.trans ? (size_t)f.rows : (size_t)f.cols;
        const size_t nout = it.trans ? (size_t)f.cols : (size_t)f.rows;
        if (it.in_rows.size() != nin || it.out_rows.size() != nout)
            return fail(RS_E_INVALID, "compressed apply: row maps do not match the form");
        if (f.hss) add_hss(B, it);
        else add_lr(B, it, tmax);
    }
    prog.z_rows = B.z;
    for (auto& kv : B.slots) {
        Slot& sl = kv.second;
        ProgStage s;
        s.kind = kv.first.kind;
        s.src = kv.first.src;
        s.dst = kv.first.dst;
        s.add = kv.first.add;
        int rc;
        if (s.kind == 0) {
            if (sl.s.empty()) continue;
            s.count = (int64_t)sl.s.size();
            if ((rc = upload_vec(s.a, sl.s, st))) return rc;
            if ((rc = upload_vec(s.b, sl.d, st))) return rc;
        } else {
            if (sl.mv.empty()) continue;
            // blocks of 16, 32 or 64 output rows: the HSS1D nodes are small (a few tens of
            // rows), and a block taller than its problem leaves most of its threads idle
            double outs = 0.0;
            for (const MatvecProb& p : sl.mv) outs += (double)(p.trans ? p.cols : p.rows);
            const double mean_out = outs / (double)sl.mv.size();
            s.rb = mean_out <= 24.0 ? 16 : mean_out <= 48.0 ? 32 : 64;
            std::vector<int64_t> blk(sl.mv.size());
            int64_t nblk = 0;
            for (size_t i = 0; i < sl.mv.size(); ++i) {
                const MatvecProb& p = sl.mv[i];
                blk[i] = nblk;
                nblk += ((p.trans ? p.cols : p.rows) + s.rb - 1) / s.rb;
                s.work += (double)p.rows * (double)p.cols;
            }
            s.count = nblk;
            s.np = (int)sl.mv.size();
            if ((rc = upload_vec(s.a, sl.mv, st))) return rc;
            if ((rc = upload_vec(s.b, blk, st))) return rc;
            prog.work += s.work;
        }
        prog.st.push_back(std::move(s));
    }
    RS_CUDA(cudaStreamSynchronize(st));
    return RS_OK;
}

template <class T>
int run_program(cudaStream_t st, const Program& prog, const T* store, const T* in, T* out, T* z, int nrhs)
{
    for (const ProgStage& s : prog.st) {
        if (s.kind == 0) {
            const T* src = s.src == BUF_IN ? in : s.src == BUF_Z ? z : out;
            T* dst = s.dst == BUF_Z ? z : out;
            RS_CUDA(launch_copy_rows<T>(st, s.count, s.a.as<int64_t>(), s.b.as<int64_t>(), src, dst, nrhs, s.add));
        } else {
            RS_CUDA(launch_matvec<T>(st, s.a.as<MatvecProb>(), s.b.as<int64_t>(), s.np, s.count, store, z, z, nrhs,
                                     s.rb));
        }
    }
    return RS_OK;
}
template int run_program<double>(cudaStream_t, const Program&, const double*, const double*, double*, double*, int);
template int run_program<float>(cudaStream_t, const Program&, const float*, const float*, float*, float*, int);
template int run_program<cplx<double>>(cudaStream_t, const Program&, const cplx<double>*, const cplx<double>*,
                                       cplx<double>*, cplx<double>*, int);
template int run_program<cplx<float>>(cudaStream_t, const Program&, const cplx<float>*, const cplx<float>*,
                                      cplx<float>*, cplx<float>*, int);

}  // namespace rs

// ------------------------------------------------------------------ the factorization's forms

namespace rs {

namespace {
using Clock = std::chrono::steady_clock;

// Grid indices of box b's skeleton (ascending g) and of its residual (ascending active
// position) on level L.
void box_points(const Level& L, int b, std::vector<int64_t>& sk, std::vector<int64_t>& rs)
{
    const int64_t a0 = L.act_off[b], k = L.k[b], m = L.m[b];
    sk.assign(L.skel.begin() + L.k_off[b], L.skel.begin() + L.k_off[b] + k);
    rs.resize((size_t)(m - k));
    for (int64_t c = 0; c < m - k; ++c) rs[(size_t)c] = L.act[a0 + L.perm[a0 + k + c]];
}
}  // namespace

template <class T>
int compress_levels(rs_op* op, cudaStream_t st)
{
    const int64_t kc = op->opts.k_cut;
    if (kc <= 0) return RS_OK;
    const auto t0 = Clock::now();
    std::vector<CForm*> all;
    for (int l = 1; l <= op->d; ++l) {
        Level& L = op->lev[l];
        L.cmp.assign(L.nb, 0);
        L.cbox.clear();
        for (int b = 0; b < L.nb; ++b)
            if (L.k[b] > kc) { L.cmp[b] = 1; L.cbox.push_back(b); }
        L.forms.assign(6 * L.cbox.size(), CForm());
        std::vector<int64_t> sk, rsg;
        for (size_t c = 0; c < L.cbox.size(); ++c) {
            const int b = L.cbox[c];
            const int64_t m = L.m[b], k = L.k[b], nr = m - k;
            box_points(L, b, sk, rsg);
            const std::vector<int> oc = cyclic_order(op->n, l, b, sk.data(), (int)k);
            const std::vector<int> oi = interface_order(op->n, l, rsg.data(), (int)nr);
            const T* Phi = L.d_Phi.as<T>() + L.phi_off[b];
            CForm* F = &L.forms[6 * c];
            F[0].hss = true;  F[0].rows = F[0].cols = (int)k;  F[0].order = oc; F[0].M = Phi;              F[0].ld = m;
            F[1].hss = true;  F[1].rows = F[1].cols = (int)nr; F[1].order = oi; F[1].M = Phi + k * m + k;  F[1].ld = m;
            F[2].hss = true;  F[2].rows = F[2].cols = (int)k;  F[2].order = oc;
            F[2].M = L.d_E.as<T>() + L.e_off[b]; F[2].ld = k;
            F[3].hss = false; F[3].rows = (int)k;  F[3].cols = (int)nr; F[3].M = Phi + k * m; F[3].ld = m;
            F[4].hss = false; F[4].rows = (int)nr; F[4].cols = (int)k;  F[4].M = Phi + k;     F[4].ld = m;
            F[5].hss = false; F[5].rows = (int)k;  F[5].cols = (int)nr;
            F[5].M = L.d_T.as<T>() + L.t_off[b]; F[5].ld = std::max<int64_t>(k, 1);
            for (int w = 0; w < 6; ++w)
                if (F[w].rows > 0 && F[w].cols > 0) all.push_back(&F[w]);
        }
    }
    if (all.empty()) return RS_OK;
    IdCtx ctx{op->d_status.as<int>(), &op->d_bar, (long long)op->opts.spin_limit};
    const double eps_c = op->opts.hss_eps > 0.0 ? op->opts.hss_eps : op->eps;
    int rc = compress_forms<T>(ctx, st, all, eps_c, op->opts.hss_leaf, op->d_cstore, op->cstore_n);
    if (rc) return rc;
    auto rows = [](int64_t base, int64_t n) {
        std::vector<int64_t> v((size_t)n);
        for (int64_t i = 0; i < n; ++i) v[(size_t)i] = base + i;
        return v;
    };
    for (int l = 1; l <= op->d; ++l) {
        Level& L = op->lev[l];
        if (L.cbox.empty()) continue;
        std::vector<ProgItem> iphi, iT, iE, iTt;
        for (size_t c = 0; c < L.cbox.size(); ++c) {
            const int b = L.cbox[c];
            const int64_t a0 = L.act_off[b], k = L.k[b], nr = L.m[b] - k, k0 = L.k_off[b];
            const CForm* F = &L.forms[6 * c];
            // Phi u: [phi_ss phi_sr; phi_rs phi_rr] on the box's rows of U (skeleton, residual)
            iphi.push_back({&F[0], false, rows(a0, k), rows(a0, k), false});
            iphi.push_back({&F[1], false, rows(a0 + k, nr), rows(a0 + k, nr), false});
            iphi.push_back({&F[3], false, rows(a0 + k, nr), rows(a0, k), true});
            iphi.push_back({&F[4], false, rows(a0, k), rows(a0 + k, nr), true});
            // t += T w[rs]; g = E t (and the same E in the downward pass); U[rs] = T^T t
            iT.push_back({&F[5], false, rows(a0 + k, nr), rows(k0, k), true});
            iE.push_back({&F[2], false, rows(k0, k), rows(k0, k), false});
            iTt.push_back({&F[5], true, rows(k0, k), rows(a0 + k, nr), false});
        }
        if ((rc = build_program(iphi, st, L.p_phi))) return rc;
        if ((rc = build_program(iT, st, L.p_T))) return rc;
        if ((rc = build_program(iE, st, L.p_E))) return rc;
        if ((rc = build_program(iTt, st, L.p_Tt))) return rc;
        if ((int)L.cbox.size() == L.nb) {
            L.d_Phi = DevMem();
            L.d_E = DevMem();
            L.d_T = DevMem();
            L.dense_freed = true;
        }
    }
    op->stats.ms_compress = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    return RS_OK;
}
template int compress_levels<double>(rs_op*, cudaStream_t);
template int compress_levels<float>(rs_op*, cudaStream_t);
template int compress_levels<cplx<double>>(rs_op*, cudaStream_t);
template int compress_levels<cplx<float>>(rs_op*, cudaStream_t);

}  // namespace rs

// ------------------------------------------------------------------ C API

using namespace rs;

struct rs_hss {
    int device = 0;
    int cplx = 0;
    int64_t n = 0;
    CForm form;
    DevMem store;
    int64_t store_n = 0;
    Program prog;
    DevMem d_status, d_bar, d_iota, xin, yout, z, hx, hy, m_dev;
};

namespace {

template <class T>
int hss_build_t(rs_hss* h, const void* Mdev, double eps, int leaf, cudaStream_t st)
{
    h->form.M = Mdev;
    h->form.ld = h->n;
    std::vector<CForm*> forms{&h->form};
    IdCtx ctx{h->d_status.as<int>(), &h->d_bar, (long long)1 << 26};
    int rc = compress_forms<T>(ctx, st, forms, eps, leaf, h->store, h->store_n);
    if (rc) return rc;
    std::vector<int64_t> iota((size_t)h->n);
    std::iota(iota.begin(), iota.end(), 0);
    std::vector<ProgItem> items{{&h->form, false, iota, iota, false}};
    return build_program(items, st, h->prog);
}

template <class T>
int hss_apply_t(rs_hss* h, const T* x, int64_t nrhs, T* y, cudaStream_t st)
{
    const int64_t n = h->n;
    const size_t e = sizeof(T);
    RS_CUDA(h->xin.alloc(e * (size_t)(n * nrhs)));
    RS_CUDA(h->yout.alloc(e * (size_t)(n * nrhs)));
    RS_CUDA(h->z.alloc(e * (size_t)(h->prog.z_rows * nrhs + 1)));
    RS_CUDA(launch_gather_cm<T, T>(st, n, h->d_iota.as<int64_t>(), x, n, h->xin.as<T>(), (int)nrhs));
    int rc = run_program<T>(st, h->prog, h->store.as<T>(), h->xin.as<T>(), h->yout.as<T>(), h->z.as<T>(), (int)nrhs);
    if (rc) return rc;
    RS_CUDA(launch_scatter_cm<T, T>(st, n, h->d_iota.as<int64_t>(), h->yout.as<T>(), n, y, (int)nrhs));
    return RS_OK;
}

const CNode* hss_node(const rs_hss* h, int level, int j)
{
    const CForm& f = h->form;
    if (f.depth == 0) return (level == 0 && j == 0) ? &f.lev[0][0] : nullptr;
    if (level < 1 || level > f.depth || j < 0 || j >= (1 << level)) return nullptr;
    return &f.lev[level][j];
}

}  // namespace

extern "C" {

int rs_hss1d_build(const void* M, int64_t n, int is_complex, const int64_t* order, int leaf, double eps, void* stream,
                   rs_hss** out)
{
    if (!M || !out || n < 1 || n > INT32_MAX / 4 || leaf < 1 || !(eps >= 0.0) || (is_complex != 0 && is_complex != 1))
        return fail(RS_E_INVALID, "bad argument");
    *out = nullptr;
    std::unique_ptr<rs_hss> h(new (std::nothrow) rs_hss());
    if (!h) return fail(RS_E_NOMEM, "host allocation");
    RS_CUDA(cudaGetDevice(&h->device));
    h->cplx = is_complex;
    h->n = n;
    h->form.hss = true;
    h->form.rows = h->form.cols = (int)n;
    h->form.order.resize((size_t)n);
    std::vector<char> seen((size_t)n, 0);
    for (int64_t p = 0; p < n; ++p) {
        const int64_t v = order ? order[p] : p;
        if (v < 0 || v >= n || seen[(size_t)v]) return fail(RS_E_INVALID, "order is not a permutation of 0..n-1");
        seen[(size_t)v] = 1;
        h->form.order[(size_t)p] = (int)v;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t esz = is_complex ? 2 * sizeof(double) : sizeof(double);
    const void* Md = M;
    if (on_other_device(M)) return fail(RS_E_INVALID, "M is device memory of another GPU than the current one");
    if (!is_device_ptr(M)) {
        RS_CUDA(h->m_dev.alloc(esz * (size_t)(n * n)));
        RS_CUDA(cudaMemcpyAsync(h->m_dev.p, M, esz * (size_t)(n * n), cudaMemcpyHostToDevice, st));
        Md = h->m_dev.p;
    }
    RS_CUDA(h->d_status.alloc(sizeof(int)));
    RS_CUDA(cudaMemsetAsync(h->d_status.p, 0, sizeof(int), st));
    std::vector<int64_t> iota((size_t)n);
    std::iota(iota.begin(), iota.end(), 0);
    RS_CUDA(h->d_iota.alloc(sizeof(int64_t) * (size_t)n));
    RS_CUDA(cudaMemcpyAsync(h->d_iota.p, iota.data(), sizeof(int64_t) * (size_t)n, cudaMemcpyHostToDevice, st));
    int rc = is_complex ? hss_build_t<cplx<double>>(h.get(), Md, eps, leaf, st)
                        : hss_build_t<double>(h.get(), Md, eps, leaf, st);
    if (rc) return rc;
    RS_CUDA(cudaStreamSynchronize(st));
    h->m_dev = DevMem();
    *out = h.release();
    return RS_OK;
}

int rs_hss1d_apply(rs_hss* h, const void* x, int64_t nrhs, void* y, void* stream)
{
    if (!h || !x || !y || nrhs < 1 || x == y) return fail(RS_E_INVALID, "bad argument");
    int dev = 0;
    RS_CUDA(cudaGetDevice(&dev));
    if (dev != h->device) return fail(RS_E_INVALID, "the current device is not the one the form was built on");
    if (on_other_device(x) || on_other_device(y))
        return fail(RS_E_INVALID, "x or y is device memory of another GPU than the form's");
    const bool dx = is_device_ptr(x), dy = is_device_ptr(y);
    if (dx != dy) return fail(RS_E_INVALID, "x and y must both be host or both be device pointers");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (h->cplx ? 2 : 1) * sizeof(double) * (size_t)(h->n * nrhs);
    const void* xi = x;
    void* yo = y;
    if (!dx) {
        RS_CUDA(h->hx.alloc(bytes));
        RS_CUDA(h->hy.alloc(bytes));
        RS_CUDA(cudaMemcpyAsync(h->hx.p, x, bytes, cudaMemcpyHostToDevice, st));
        xi = h->hx.p;
        yo = h->hy.p;
    }
    int rc = h->cplx ? hss_apply_t<cplx<double>>(h, (const cplx<double>*)xi, nrhs, (cplx<double>*)yo, st)
                     : hss_apply_t<double>(h, (const double*)xi, nrhs, (double*)yo, st);
    if (rc) return rc;
    if (!dx) {
        RS_CUDA(cudaMemcpyAsync(y, h->hy.p, bytes, cudaMemcpyDeviceToHost, st));
        RS_CUDA(cudaStreamSynchronize(st));
    }
    return RS_OK;
}

int rs_hss1d_info(const rs_hss* h, int* depth, int64_t* entries, int64_t* bytes)
{
    if (!h) return fail(RS_E_INVALID, "NULL form");
    if (depth) *depth = h->form.depth;
    if (entries) *entries = h->form.entries;
    if (bytes) *bytes = h->store_n * (h->cplx ? 2 : 1) * (int64_t)sizeof(double);
    return RS_OK;
}

int rs_hss1d_node(const rs_hss* h, int level, int node, int64_t* lo, int64_t* hi, int64_t* a, int64_t* k,
                  int64_t* skel_rows)
{
    if (!h) return fail(RS_E_INVALID, "NULL form");
    const CNode* q = hss_node(h, level, node);
    if (!q) return fail(RS_E_INVALID, "level/node out of range");
    if (lo) *lo = q->lo;
    if (hi) *hi = q->hi;
    if (a) *a = q->a;
    if (k) *k = q->k;
    if (skel_rows)
        for (int s = 0; s < q->k; ++s) skel_rows[s] = q->act[q->perm[s]];
    return RS_OK;
}

int rs_hss1d_free(rs_hss* h)
{
    delete h;
    return RS_OK;
}

int rs_op_box_order(const rs_op* op, int level, int box, int which, int64_t* out)
{
    if (!op || !out || level < 1 || level > op->d || box < 0 || box >= (1 << level) || (which != 0 && which != 1))
        return fail(RS_E_INVALID, "bad argument");
    const Level& L = op->lev[level];
    std::vector<int64_t> sk, rsg;
    box_points(L, box, sk, rsg);
    const std::vector<int> o = which == 0 ? cyclic_order(op->n, level, box, sk.data(), (int)sk.size())
                                          : interface_order(op->n, level, rsg.data(), (int)rsg.size());
    for (size_t i = 0; i < o.size(); ++i) out[i] = o[i];
    return RS_OK;
}

int rs_tree_box_order(const rs_tree* tree, int level, int box, int which, const int64_t* g, int64_t cnt, int64_t* out)
{
    if (!tree || level < 1 || level > tree->d || box < 0 || box >= (1 << level) || (which != 0 && which != 1) ||
        cnt < 0 || cnt > INT32_MAX || (cnt > 0 && (!g || !out)))
        return fail(RS_E_INVALID, "bad argument");
    const int64_t N = tree->n * tree->n;
    for (int64_t i = 0; i < cnt; ++i)
        if (g[i] < 0 || g[i] >= N) return fail(RS_E_INVALID, "grid index out of range");
    const std::vector<int> o = which == 0 ? cyclic_order(tree->n, level, box, g, (int)cnt)
                                          : interface_order(tree->n, level, g, (int)cnt);
    for (size_t i = 0; i < o.size(); ++i) out[i] = o[i];
    return RS_OK;
}

int rs_op_box_form(const rs_op* op, int level, int box, int which, int* depth, int64_t* entries, int64_t* nodes)
{
    if (!op || level < 1 || level > op->d || box < 0 || box >= (1 << level) || which < 0 || which > 5)
        return fail(RS_E_INVALID, "bad argument");
    const Level& L = op->lev[level];
    const auto it = std::find(L.cbox.begin(), L.cbox.end(), box);
    if (it == L.cbox.end()) return fail(RS_E_INVALID, "box is not compressed");
    const CForm& f = L.forms[6 * (it - L.cbox.begin()) + which];
    if (depth) *depth = f.hss ? f.depth : -1;
    if (entries) *entries = f.entries;
    if (nodes) {
        int64_t w = 0;
        if (f.lev.empty()) return RS_OK;
        const int l0 = (!f.hss || f.depth == 0) ? 0 : 1;
        const int l1 = f.hss ? f.depth : 0;
        for (int l = l0; l <= l1; ++l)
            for (const CNode& q : f.lev[l]) {
                nodes[w++] = f.hss ? q.lo : f.rows;
                nodes[w++] = f.hss ? q.hi : f.cols;
                nodes[w++] = q.a;
                nodes[w++] = q.k;
            }
    }
    return RS_OK;
}

}  // extern "C"
