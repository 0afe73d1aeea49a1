// rs_tree.cpp -- errors, options, the tree of Sec. 2.2 and its per-level index bookkeeping.
// Integer host code only; the floating-point work of the method runs in the CUDA kernels.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <string>
#include <vector>

#include "rs_host.h"

namespace rs {

static thread_local std::string g_err;
static std::atomic<int64_t> g_launches{0};

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_err = msg; }

int fail(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? RS_E_NOMEM : RS_E_CUDA;
}

// Box j of level l as integers: grid-cell origin (bx * wx, by * wy) and extents (wx, wy).
// The bit of j for depth t, most significant first, picks the lower (0) or upper (1) half of
// the split at that depth: x1 at even depth, x2 at odd depth.
BoxInt box_int(int64_t n, int l, int64_t j)
{
    BoxInt b{0, 0, n, n};
    int64_t x = 0, y = 0;
    for (int t = 0; t < l; ++t) {
        const int64_t bit = (j >> (l - 1 - t)) & 1;
        if ((t & 1) == 0) { x = 2 * x + bit; b.wx >>= 1; }
        else { y = 2 * y + bit; b.wy >>= 1; }
    }
    b.bx = x;
    b.by = y;
    return b;
}

int level_sets(int64_t n, int d, int l, const int64_t* child_k, const int64_t* child_skel, double rfac,
               std::vector<int64_t>& m, std::vector<int64_t>& act, std::vector<int64_t>& act_off,
               std::vector<int64_t>& nnear, std::vector<int64_t>& nearv, std::vector<int64_t>& near_off)
{
    if (l < 1 || l > d) return fail(RS_E_INVALID, "level out of range");
    const int64_t nb = int64_t(1) << l;
    m.assign(nb, 0);
    act_off.assign(nb + 1, 0);
    act.clear();
    if (l == d) {
        for (int64_t j = 0; j < nb; ++j) {
            const BoxInt b = box_int(n, l, j);
            for (int64_t i2 = b.by * b.wy; i2 < (b.by + 1) * b.wy; ++i2)
                for (int64_t i1 = b.bx * b.wx; i1 < (b.bx + 1) * b.wx; ++i1) act.push_back(i1 + n * i2);
            m[j] = b.wx * b.wy;
            act_off[j + 1] = (int64_t)act.size();
        }
    } else {
        if (!child_k || !child_skel) return fail(RS_E_INVALID, "child skeletons required above the leaf level");
        int64_t pos = 0;
        for (int64_t j = 0; j < nb; ++j) {
            const int64_t k1 = child_k[2 * j], k2 = child_k[2 * j + 1];
            if (k1 < 0 || k2 < 0) return fail(RS_E_INVALID, "negative skeleton size");
            act.insert(act.end(), child_skel + pos, child_skel + pos + k1 + k2);
            pos += k1 + k2;
            m[j] = k1 + k2;
            act_off[j + 1] = (int64_t)act.size();
        }
    }
    // near rows: touching same-level boxes (index distance <= 1 in both directions), their
    // active points strictly inside the proxy circle; all lengths in units of h/2
    nnear.assign(nb, 0);
    near_off.assign(nb + 1, 0);
    nearv.clear();
    // the level's boxes tile the grid: index them by position, so each box finds its (at most
    // eight) neighbours directly, then visits them in ascending box index
    std::vector<BoxInt> boxes(nb);
    int64_t nbx = 0, nby = 0;
    for (int64_t j = 0; j < nb; ++j) {
        boxes[j] = box_int(n, l, j);
        nbx = std::max(nbx, boxes[j].bx + 1);
        nby = std::max(nby, boxes[j].by + 1);
    }
    std::vector<int64_t> at((size_t)(nbx * nby), -1);
    for (int64_t j = 0; j < nb; ++j) at[(size_t)(boxes[j].bx + nbx * boxes[j].by)] = j;
    for (int64_t j = 0; j < nb; ++j) {
        const BoxInt b = boxes[j];
        const int64_t cx = (2 * b.bx + 1) * b.wx, cy = (2 * b.by + 1) * b.wy;
        const double R = rfac * (double)std::max(b.wx, b.wy);
        const double R2 = R * R;
        int64_t nbr[8];
        int cnt = 0;
        for (int64_t ey = -1; ey <= 1; ++ey)
            for (int64_t ex = -1; ex <= 1; ++ex) {
                const int64_t x = b.bx + ex, y = b.by + ey;
                if ((ex == 0 && ey == 0) || x < 0 || y < 0 || x >= nbx || y >= nby) continue;
                const int64_t q = at[(size_t)(x + nbx * y)];
                if (q >= 0) nbr[cnt++] = q;
            }
        std::sort(nbr, nbr + cnt);
        for (int c = 0; c < cnt; ++c) {
            const int64_t q = nbr[c];
            for (int64_t p = act_off[q]; p < act_off[q + 1]; ++p) {
                const int64_t g = act[p];
                const int64_t dx = 2 * (g % n) + 1 - cx, dy = 2 * (g / n) + 1 - cy;
                if ((double)(dx * dx + dy * dy) < R2) nearv.push_back(g);
            }
        }
        nnear[j] = (int64_t)nearv.size() - near_off[j];
        near_off[j + 1] = (int64_t)nearv.size();
    }
    return RS_OK;
}

}  // namespace rs

using namespace rs;

extern "C" {

void rs_opts_default(rs_opts* o)
{
    if (!o) return;
    o->proxy_points = 64;
    o->proxy_radius_factor = 1.5;
    o->precision = RS_FP64;
    o->refine_tol = 1e-10;
    o->refine_max_iter = 10;
    o->k_cut = 0;
    o->spin_limit = (int64_t)1 << 26;
    o->profile = 0;
    o->hss_leaf = 64;
    o->spd_inverse = 1;
    o->cpqr_variant = -1;
    o->translation_invariant = 0;
    o->sweep_panel = 0;
    o->forward_only = 0;
    o->gemm_form = 1;
    o->solve_graph = 1;
    o->per_box = 0;
    o->hss_eps = 0.0;
}

int64_t rs_launch_count(void) { return g_launches.load(); }

const char* rs_last_error(void) { return g_err.c_str(); }

int rs_build_tree(const double* points, int64_t N, int leaf_side, rs_tree** out)
{
    if (!out) return fail(RS_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!points || N < 4 || leaf_side < 1) return fail(RS_E_INVALID, "bad points, N or leaf_side");
    const int64_t n = (int64_t)llround(sqrt((double)N));
    if (n * n != N) return fail(RS_E_INVALID, "N is not a square");
    if (n % leaf_side) return fail(RS_E_INVALID, "n is not a multiple of leaf_side");
    int64_t q = n / leaf_side;
    int L = 0;
    while ((int64_t(1) << L) < q) ++L;
    if ((int64_t(1) << L) != q || L < 1) return fail(RS_E_INVALID, "n / leaf_side must be a power of two >= 2");
    if (2 * L > 40) return fail(RS_E_INVALID, "tree too deep");
    const double h = 1.0 / (double)n;
    rs_tree* t = new (std::nothrow) rs_tree();
    if (!t) return fail(RS_E_NOMEM, "host allocation");
    t->n = n;
    t->leaf = leaf_side;
    t->d = 2 * L;
    t->g_of_input.assign(N, -1);
    t->input_of_g.assign(N, -1);
    for (int64_t i = 0; i < N; ++i) {
        const double x = points[2 * i], y = points[2 * i + 1];
        const double fx = x / h - 0.5, fy = y / h - 0.5;
        const double rx = std::nearbyint(fx), ry = std::nearbyint(fy);
        if (!(std::fabs(fx - rx) <= 1e-9) || !(std::fabs(fy - ry) <= 1e-9) || rx < 0 || ry < 0 || rx >= n || ry >= n) {
            delete t;
            return fail(RS_E_NOT_GRID, "point " + std::to_string(i) + " is not a cell centre of the n x n grid");
        }
        const int64_t g = (int64_t)rx + n * (int64_t)ry;
        if (t->input_of_g[g] >= 0) {
            delete t;
            return fail(RS_E_NOT_GRID, "duplicate point " + std::to_string(i));
        }
        t->input_of_g[g] = i;
        t->g_of_input[i] = g;
    }
    *out = t;
    return RS_OK;
}

void rs_free_tree(rs_tree* t) { delete t; }

int rs_tree_info(const rs_tree* t, int64_t* n_side, int* depth, int64_t* grid_index_of_input)
{
    if (!t) return fail(RS_E_INVALID, "tree is NULL");
    if (n_side) *n_side = t->n;
    if (depth) *depth = t->d;
    if (grid_index_of_input) memcpy(grid_index_of_input, t->g_of_input.data(), sizeof(int64_t) * t->g_of_input.size());
    return RS_OK;
}

int rs_tree_level_sets(const rs_tree* t, int level, const int64_t* child_k, const int64_t* child_skel,
                       double proxy_radius_factor, int64_t* m, int64_t* act, int64_t* nnear, int64_t* near)
{
    if (!t || !m || !nnear) return fail(RS_E_INVALID, "NULL argument");
    std::vector<int64_t> mv, av, ao, nv, nr, no;
    const int rc = level_sets(t->n, t->d, level, child_k, child_skel, proxy_radius_factor, mv, av, ao, nv, nr, no);
    if (rc) return rc;
    memcpy(m, mv.data(), sizeof(int64_t) * mv.size());
    memcpy(nnear, nv.data(), sizeof(int64_t) * nv.size());
    if (act) memcpy(act, av.data(), sizeof(int64_t) * av.size());
    if (near) memcpy(near, nr.data(), sizeof(int64_t) * nr.size());
    return RS_OK;
}

}  // extern "C"
