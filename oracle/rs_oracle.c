/*
 * rs_oracle.c -- plain CPU oracle (FP64 / complex128) of the dense-block HSS inverse of
 * arXiv:1303.5466.  TEST INFRASTRUCTURE ONLY: see rs_oracle.h.  Built with
 * -ffp-contract=off so that its rounding does not depend on the host's FMA support.
 *
 * Readings of the paper taken here (the paper is silent or ambiguous on these):
 *   - grid: cell centres x_g = ((i1+1/2)h, (i2+1/2)h) of [0,1]^2, g = i1 + n i2;
 *   - tree: binary, depth t splits along x1 when t is even and x2 when t is odd; box j
 *     of level l has children 2j (lower half) and 2j+1 (upper half) (Sec. 2.2);
 *   - leaf points ascend in g; a parent's active set is sk(c1) then sk(c2), each
 *     ascending in g (Sec. 2.2, re-blocking: I_i = I_c1^sk u I_c2^sk);
 *   - neighbours: same-level boxes whose closed rectangles touch (edge or corner);
 *     near rows: neighbours' active points strictly inside the proxy circle, in
 *     (neighbour, active) order; proxy: P points c + R(cos 2 pi j/P, sin 2 pi j/P) with
 *     R = factor x the larger half-width (Sec. 2.2, equivalent densities);
 *   - E_i = (R_i F_i^{-1} L_i)^{-1} as in Algorithm 1 (the "E = R F^{-1} L" of
 *     Sec. 2.4 contradicts Algorithm 1 and the derivation of Eq. 2.11);
 *   - the Helmholtz kernel is +(i/4) H0 and the system is put in the symmetric form
 *     of Eq. (5.6) by the diagonal similarity S = diag(kappa sqrt(b)).
 */
#define _DEFAULT_SOURCE
#ifndef RO_PLANT
#define RO_PLANT 0
#endif
#include "rs_oracle.h"
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* HSS1D form (Sec. 3.2) of an explicit n x n matrix M on a one-dimensional ordering of
 * its indices: binary tree over runs of the ordering, node (l, j) covering positions
 * [floor(j n / 2^l), floor((j+1) n / 2^l)); the telescoping factorization of Eq. 2.9
 * with one ID per node serving its block row and block column. */
typedef struct {
    int lo, hi;        /* position range                                        */
    int a, k;          /* active size, skeleton size                            */
    int* act;          /* a row indices of M (leaf: positions lo..hi-1; above:
                          skeleton rows of child 1 then child 2)                */
    int* sk;           /* k local indices, ascending                            */
    int* rs;           /* a - k local indices, ascending                        */
    void* T;           /* k x (a-k) row-major scalars                           */
} ro_hnode;

struct ro_hss {
    int cplx, n, depth, leaf;
    int* order;        /* position -> row of M                                   */
    ro_hnode** node;   /* node[l][j], l = 1..depth                               */
    void** B12;        /* internal node (l, j), l < depth, heap index 2^l-1+j:
                          M(skeleton of child 1, skeleton of child 2)            */
    void** B21;        /* M(skeleton of child 2, skeleton of child 1)            */
    void** D;          /* leaf j: M(act, act), a x a row-major; depth 0: D[0] = M */
};

/* Low-rank form X ~ X(:, sk) [I T] (columns permuted back) of a p x q matrix, from a
 * column ID of X (Sec. 3.2, low-rank blocks). */
typedef struct {
    int p, q, k;
    int* sk;           /* k column indices, ascending      */
    int* rs;           /* q - k column indices, ascending  */
    void* C;           /* X(:, sk), p x k row-major         */
    void* T;           /* k x (q-k) row-major               */
} ro_lr;

typedef struct {
    int m, k, r, nnear;
    int64_t* active;   /* m globals                        */
    int64_t* near;     /* nnear globals                    */
    int64_t* skel;     /* k globals, ascending             */
    int* sk_local;     /* k local indices (skeleton order) */
    int* rs_local;     /* m-k local indices, ascending     */
    double* T;         /* k x (m-k) scalars                */
    double* Finv;      /* m x m scalars                    */
    double* E;         /* k x k scalars                    */
    /* extra compression of Sec. 3 (k > k_cut): the blocks of Phi = Pi^T F^{-1} Pi,
     * E and T in compressed form; the inverse apply then uses these */
    int hss;
    ro_hss* H_ss;      /* phi^{sk}, skeleton in cyclic order around the box      */
    ro_hss* H_rr;      /* phi^{rs}, residual in order along the interface        */
    ro_hss* H_E;       /* E, cyclic order                                        */
    ro_lr L_sr, L_rs;  /* phi^{s<-r}, phi^{r<-s}                                 */
    ro_lr L_T;         /* T                                                      */
} ro_box;

struct ro_op {
    int n, leaf, d;
    double h, eps;
    ro_opts opts;
    int nthreads;
    double* a;          /* N (diagonal coefficient a(x))            */
    double* s;          /* N (Helmholtz symmetric scaling kappa sqrt b) */
    double* b;          /* N (Helmholtz b) or NULL                  */
    double lap_c0;      /* -h^2/(4 pi): multiplies log r^2          */
    double lap_self;    /* -(1/2pi) C_h                             */
    double complex hz_self; /* (i/4) * integral of H0 over the cell */
    double* pcos;       /* proxy unit circle                        */
    double* psin;
    ro_box** lev;       /* lev[l][j], l = 1..d                      */
    int partial;        /* only the finest levels were factored (timing sample) */
    int m0;
    int64_t* active0;
    double* root_inv;
};

/* ------------------------------------------------------------------ geometry */

/* Integer description of box j at level l: x-index bx, y-index by, extents wx, wy in
 * grid cells.  The bit of j for depth t (MSB first) selects the half at that split. */
static void box_int(int n, int l, int j, int* bx, int* by, int* wx, int* wy)
{
    int x = 0, y = 0, nx = 0, ny = 0;
    for (int t = 0; t < l; ++t) {
        int bit = (j >> (l - 1 - t)) & 1;
        if ((t & 1) == 0) { x = 2 * x + bit; ++nx; } else { y = 2 * y + bit; ++ny; }
    }
    *bx = x; *by = y; *wx = n >> nx; *wy = n >> ny;
}

static void box_center_radius(const ro_op* op, int l, int j, double* cx, double* cy, double* R)
{
    int bx, by, wx, wy;
    box_int(op->n, l, j, &bx, &by, &wx, &wy);
    double hh = 0.5 * op->h;
    *cx = (double)((2 * bx + 1) * wx) * hh;
    *cy = (double)((2 * by + 1) * wy) * hh;
    int w = wx > wy ? wx : wy;
    *R = (op->opts.proxy_radius_factor * (double)w) * hh;
}

/* ------------------------------------------------------------------ quadrature */

double ro_laplace_cell_integral(double h)
{
    /* integral of log|y| over [-h/2,h/2]^2 = h^2 (log h - (1/2) log 2 - 3/2 + pi/4),
     * from the polar form over the eight triangles of the square */
#if RO_PLANT == 3
    return -h * h * (log(h) - 0.5 * log(2.0) - 1.5 + M_PI / 4.0);
#else
    return h * h * (log(h) - 0.5 * log(2.0) - 1.5 + M_PI / 4.0);
#endif
}

void ro_gauss_legendre(int n, double* x, double* w)
{
    /* roots of P_n by Newton's method from the Chebyshev-like initial guess; the weight is
     * 2 / ((1 - z^2) P_n'(z)^2), with P_n' from the three-term recurrence */
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-15) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1; p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

void ro_helmholtz_cell_integral(double h, double kappa, int nodes, double* re, double* im)
{
    /* integral over the cell of H0(kappa r) = 8 * int_0^{pi/4} int_0^{rho(th)} H0(kappa r) r dr dth,
     * rho = (h/2)/cos th, and int_0^rho r H0(kappa r) dr = (kappa rho H1(kappa rho) + 2i/pi)/kappa^2 */
    double* x = (double*)malloc(sizeof(double) * (size_t)nodes);
    double* w = (double*)malloc(sizeof(double) * (size_t)nodes);
    ro_gauss_legendre(nodes, x, w);
    double complex acc = 0.0;
    for (int i = 0; i < nodes; ++i) {
        double th = (M_PI / 8.0) * (1.0 + x[i]);
        double rho = 0.5 * h / cos(th);
        double z = kappa * rho;
        double complex H1 = j1(z) + I * y1(z);
        acc += (M_PI / 8.0) * w[i] * (z * H1 + 2.0 * I / M_PI) / (kappa * kappa);
    }
    acc *= 8.0;
    *re = creal(acc); *im = cimag(acc);
    free(x); free(w);
}

/* ------------------------------------------------------------------ matrix entries */

static inline void gxy(const ro_op* op, int64_t g, double* x, double* y)
{
    int64_t i1 = g % op->n, i2 = g / op->n;
    *x = ((double)i1 + 0.5) * op->h;
    *y = ((double)i2 + 0.5) * op->h;
}

/* Laplace, Sec. 5: A_gg' = -(1/2pi) h^2 log|x_g - x_g'|, A_gg = a_g - (1/2pi) C_h */
static double entry_d(const ro_op* op, int64_t g, int64_t gp)
{
    if (g == gp) return op->a[g] + op->lap_self;
    double x, y, xp, yp;
    gxy(op, g, &x, &y); gxy(op, gp, &xp, &yp);
    double dx = x - xp, dy = y - yp;
    return op->lap_c0 * log(dx * dx + dy * dy);
}

static double proxy_entry_d(const ro_op* op, double zx, double zy, int64_t g)
{
    double x, y;
    gxy(op, g, &x, &y);
    double dx = zx - x, dy = zy - y;
    return op->lap_c0 * log(dx * dx + dy * dy);
}

/* Helmholtz in the symmetric form of Eq. (5.6):
 * A_gg' = s_g (i/4) H0(kappa r) h^2 s_g',  A_gg = a_g + s_g^2 (i/4) int_cell H0 */
static double complex entry_z(const ro_op* op, int64_t g, int64_t gp)
{
    if (g == gp) return op->a[g] + op->s[g] * op->s[g] * op->hz_self;
    double x, y, xp, yp;
    gxy(op, g, &x, &y); gxy(op, gp, &xp, &yp);
    double dx = x - xp, dy = y - yp;
    double z = op->opts.kappa * sqrt(dx * dx + dy * dy);
    double complex k = 0.25 * I * (j0(z) + I * y0(z)) * (op->h * op->h);
    return op->s[g] * k * op->s[gp];
}

static double complex proxy_entry_z(const ro_op* op, double zx, double zy, int64_t g)
{
    double x, y;
    gxy(op, g, &x, &y);
    double dx = zx - x, dy = zy - y;
    double z = op->opts.kappa * sqrt(dx * dx + dy * dy);
    double complex k = 0.25 * I * (j0(z) + I * y0(z)) * (op->h * op->h);
    return k * op->s[g];
}

/* Translation-invariant mode: the entry between a lattice point outside the grid at (x, y)
 * (a translate of a grid point) and grid point g.  It is the off-diagonal formula; in the
 * Helmholtz form the outside point takes the constant scaling s of the grid. */
static double outside_entry_d(const ro_op* op, double x, double y, int64_t g)
{
    return proxy_entry_d(op, x, y, g);
}

static double complex outside_entry_z(const ro_op* op, double x, double y, int64_t g)
{
    return op->s[0] * proxy_entry_z(op, x, y, g);
}

/* Pivot key of the column-pivoted QR: the squared norm with its 40 low mantissa bits
 * cleared (a monotone map of non-negative doubles onto a grid of relative step 2^-12). */
static uint64_t pivot_key(double v)
{
    if (!(v > 0.0)) v = 0.0;
    uint64_t u;
    memcpy(&u, &v, sizeof u);
    return u & ~((UINT64_C(1) << 40) - 1);
}

/* ------------------------------------------------------------------ orders of Sec. 3.1 */

/* Skeleton points of box (l, j) ordered cyclically around the box: by angle about the box
 * centre, counter-clockwise from the positive x1 axis; points on one ray by distance, then
 * by grid index.  Decided on integer offsets in units of h/2 (exact). */
typedef struct { int64_t dx, dy, g; int idx; } cyc_key;

static int cyc_cmp(const void* pa, const void* pb)
{
    const cyc_key* a = (const cyc_key*)pa;
    const cyc_key* b = (const cyc_key*)pb;
    int ha = (a->dy < 0) || (a->dy == 0 && a->dx < 0);
    int hb = (b->dy < 0) || (b->dy == 0 && b->dx < 0);
    if (ha != hb) return ha - hb;
    int64_t cr = a->dx * b->dy - a->dy * b->dx;
    if (cr != 0) return cr > 0 ? -1 : 1;
    int64_t ra = a->dx * a->dx + a->dy * a->dy, rb = b->dx * b->dx + b->dy * b->dy;
    if (ra != rb) return ra < rb ? -1 : 1;
    return (a->g > b->g) - (a->g < b->g);
}

static void box_cyclic_order(const ro_op* op, int l, int j, const int64_t* pts, int cnt, int* order)
{
    int bx, by, wx, wy;
    box_int(op->n, l, j, &bx, &by, &wx, &wy);
    int64_t cx2 = (int64_t)(2 * bx + 1) * wx, cy2 = (int64_t)(2 * by + 1) * wy;
    cyc_key* key = (cyc_key*)malloc(sizeof(cyc_key) * (size_t)(cnt + 1));
    for (int i = 0; i < cnt; ++i) {
        int64_t g = pts[i];
        key[i].dx = 2 * (g % op->n) + 1 - cx2;
        key[i].dy = 2 * (g / op->n) + 1 - cy2;
        key[i].g = g;
        key[i].idx = i;
    }
    qsort(key, (size_t)cnt, sizeof(cyc_key), cyc_cmp);
    for (int i = 0; i < cnt; ++i) order[i] = key[i].idx;
    free(key);
}

/* Residual points of a box of level l ordered along the interface between its children:
 * a box at even depth is split along x1, so its interface runs along x2 and the points are
 * ordered by (i2, i1); at odd depth by (i1, i2). */
typedef struct { int64_t major, minor; int idx; } ifc_key;

static int ifc_cmp(const void* pa, const void* pb)
{
    const ifc_key* a = (const ifc_key*)pa;
    const ifc_key* b = (const ifc_key*)pb;
    if (a->major != b->major) return a->major < b->major ? -1 : 1;
    return (a->minor > b->minor) - (a->minor < b->minor);
}

static void box_interface_order(const ro_op* op, int l, const int64_t* pts, int cnt, int* order)
{
    ifc_key* key = (ifc_key*)malloc(sizeof(ifc_key) * (size_t)(cnt + 1));
    for (int i = 0; i < cnt; ++i) {
        int64_t i1 = pts[i] % op->n, i2 = pts[i] / op->n;
        key[i].major = (l % 2 == 0) ? i2 : i1;
        key[i].minor = (l % 2 == 0) ? i1 : i2;
        key[i].idx = i;
    }
    qsort(key, (size_t)cnt, sizeof(ifc_key), ifc_cmp);
    for (int i = 0; i < cnt; ++i) order[i] = key[i].idx;
    free(key);
}

/* ------------------------------------------------------------------ numeric core x2 */

#define SC double
#define FN(x) x##_d
#define ABS2(z) ((z) * (z))
#define ABSV(z) fabs(z)
#define CONJ(z) (z)
#define IS_CPLX 0
#include "ro_core.inc"
#undef SC
#undef FN
#undef ABS2
#undef ABSV
#undef CONJ
#undef IS_CPLX

#define SC double complex
#define FN(x) x##_z
#define ABS2(z) (creal(z) * creal(z) + cimag(z) * cimag(z))
#define ABSV(z) cabs(z)
#define CONJ(z) conj(z)
#define IS_CPLX 1
#include "ro_core.inc"
#undef SC
#undef FN
#undef ABS2
#undef ABSV
#undef CONJ
#undef IS_CPLX

/* ------------------------------------------------------------------ public API */

void ro_opts_default(ro_opts* o)
{
    o->kind = 0;
    o->kappa = 0.0;
    o->proxy_points = 64;
    o->proxy_radius_factor = 1.5;
    o->near_all = 0;
    o->threads = 0;
    o->max_levels = 0;
    o->k_cut = 0;
    o->hss_leaf = 64;
    o->hss_eps = 0.0;
    o->ti = 0;
}

int ro_id(int cplx, const double* Y, int r, int m, double eps, int* k_out, int* perm, double* T)
{
    if (r < 0 || m < 1 || !Y || !k_out || !perm || !T) return -1;
    if (cplx) return id_z((const double complex*)Y, r, m, eps, k_out, perm, (double complex*)T);
    return id_d(Y, r, m, eps, k_out, perm, T);
}

int ro_inverse(int cplx, const double* A, int m, double* Ainv)
{
    if (m < 1 || !A || !Ainv) return -1;
    if (cplx) return inverse_z((const double complex*)A, m, (double complex*)Ainv);
    return inverse_d(A, m, Ainv);
}

static int ilog2(int v) { int r = 0; while ((1 << r) < v) ++r; return ((1 << r) == v) ? r : -1; }

/* Active sets and near lists of level l, from the skeletons of level l+1 (or the grid). */
static void level_bookkeeping(ro_op* op, int l)
{
    int nb = 1 << l, n = op->n;
    for (int j = 0; j < nb; ++j) {
        ro_box* B = &op->lev[l][j];
        if (l == op->d) {
            int bx, by, wx, wy;
            box_int(n, l, j, &bx, &by, &wx, &wy);
            B->m = wx * wy;
            B->active = (int64_t*)malloc(sizeof(int64_t) * (size_t)B->m);
            int q = 0;
            for (int i2 = by * wy; i2 < (by + 1) * wy; ++i2)
                for (int i1 = bx * wx; i1 < (bx + 1) * wx; ++i1) B->active[q++] = (int64_t)i1 + (int64_t)n * i2;
        } else {
            ro_box* C1 = &op->lev[l + 1][2 * j];
            ro_box* C2 = &op->lev[l + 1][2 * j + 1];
            B->m = C1->k + C2->k;
            B->active = (int64_t*)malloc(sizeof(int64_t) * (size_t)(B->m + 1));
            memcpy(B->active, C1->skel, sizeof(int64_t) * (size_t)C1->k);
            memcpy(B->active + C1->k, C2->skel, sizeof(int64_t) * (size_t)C2->k);
        }
    }
    for (int j = 0; j < nb; ++j) {
        ro_box* B = &op->lev[l][j];
        int bx, by, wx, wy;
        box_int(n, l, j, &bx, &by, &wx, &wy);
        int64_t cx2 = (int64_t)(2 * bx + 1) * wx, cy2 = (int64_t)(2 * by + 1) * wy;
        int w = wx > wy ? wx : wy;
        double R2 = op->opts.proxy_radius_factor * (double)w;   /* in units of h/2 */
        double R2sq = R2 * R2;
        int cap = 0;
        for (int q = 0; q < nb; ++q) if (q != j) cap += op->lev[l][q].m;
        B->near = (int64_t*)malloc(sizeof(int64_t) * (size_t)(cap + 1));
        int cnt = 0;
        for (int q = 0; q < nb; ++q) {
            if (q == j) continue;
            int qx, qy, qwx, qwy;
            box_int(n, l, q, &qx, &qy, &qwx, &qwy);
            if (!op->opts.near_all && (abs(qx - bx) > 1 || abs(qy - by) > 1)) continue;
            const ro_box* Q = &op->lev[l][q];
            for (int p = 0; p < Q->m; ++p) {
                int64_t g = Q->active[p];
                if (!op->opts.near_all) {
                    int64_t i1 = g % n, i2 = g / n;
                    int64_t dx = 2 * i1 + 1 - cx2, dy = 2 * i2 + 1 - cy2;
                    if (!((double)(dx * dx + dy * dy) < R2sq)) continue;
                }
                B->near[cnt++] = g;
            }
        }
        B->nnear = cnt;
    }
}

int ro_factor(int n, int leaf_side, const double* a, const double* b, double eps,
              const ro_opts* opts, ro_op** out)
{
    if (!out || n < 2 || leaf_side < 1 || n % leaf_side) return -1;
    int L = ilog2(n / leaf_side);
    if (L < 1) return -1;
    ro_opts o;
    if (opts) o = *opts; else ro_opts_default(&o);
    if (o.kind != 0 && o.kind != 1) return -1;
    if (o.kind == 0 && b) return -1;
    if (o.proxy_points < 0) return -1;
    if (o.k_cut > 0 && (o.hss_leaf < 1 || !(o.hss_eps >= 0.0))) return -1;
    int64_t N = (int64_t)n * n;
    if (o.ti) {                  /* translation invariance needs constant a and b */
        if (o.k_cut > 0 || o.near_all) return -1;
        for (int64_t g = 1; g < N; ++g)
            if ((a && a[g] != a[0]) || (b && b[g] != b[0])) return -1;
    }
    ro_op* op = (ro_op*)calloc(1, sizeof(ro_op));
    op->n = n; op->leaf = leaf_side; op->d = 2 * L; op->h = 1.0 / n; op->eps = eps; op->opts = o;
#ifdef _OPENMP
    op->nthreads = o.threads > 0 ? o.threads : omp_get_max_threads();
#else
    op->nthreads = 1;
#endif
    op->a = (double*)malloc(sizeof(double) * (size_t)N);
    op->s = (double*)malloc(sizeof(double) * (size_t)N);
    for (int64_t g = 0; g < N; ++g) {
        op->a[g] = a ? a[g] : 1.0;
        double bg = b ? b[g] : 1.0;
        if (o.kind == 1 && !(bg > 0.0)) { ro_free(op); return -1; }
        op->s[g] = (o.kind == 1) ? o.kappa * sqrt(bg) : 1.0;
    }
    op->lap_c0 = -(op->h * op->h) / (4.0 * M_PI);
    op->lap_self = -ro_laplace_cell_integral(op->h) / (2.0 * M_PI);
    if (o.kind == 1) {
        double re, im;
        ro_helmholtz_cell_integral(op->h, o.kappa, 32, &re, &im);
        op->hz_self = 0.25 * I * (re + I * im);
    }
    int P = o.proxy_points;
    op->pcos = (double*)malloc(sizeof(double) * (size_t)(P + 1));
    op->psin = (double*)malloc(sizeof(double) * (size_t)(P + 1));
    for (int q = 0; q < P; ++q) {
        double ang = (2.0 * M_PI * (double)q) / (double)P;
        op->pcos[q] = cos(ang); op->psin[q] = sin(ang);
    }
    op->lev = (ro_box**)calloc((size_t)(op->d + 1), sizeof(ro_box*));
    for (int l = 1; l <= op->d; ++l) op->lev[l] = (ro_box*)calloc((size_t)1 << l, sizeof(ro_box));
    int rc = 0;
    const int lmin = (o.max_levels > 0 && o.max_levels < op->d) ? op->d - o.max_levels + 1 : 1;
    for (int l = op->d; l >= lmin && rc == 0; --l) {
        level_bookkeeping(op, l);
        int nb = 1 << l;
        int err = 0;
        if (o.ti) {
            rc = (o.kind == 0) ? factor_ti_level_d(op, l) : factor_ti_level_z(op, l);
            continue;
        }
        #pragma omp parallel for schedule(dynamic) num_threads(op->nthreads)
        for (int j = 0; j < nb; ++j) {
            int e = (o.kind == 0) ? factor_box_d(op, l, j) : factor_box_z(op, l, j);
            if (e) {
                #pragma omp critical
                err = e;
            }
        }
        rc = err;
    }
    if (rc == 0 && lmin == 1) rc = (o.kind == 0) ? factor_root_d(op) : factor_root_z(op);
    op->partial = (lmin > 1);
    if (rc) { ro_free(op); return rc; }
    *out = op;
    return 0;
}

int ro_fwd_apply(const ro_op* op, const double* x, int nrhs, double* y)
{
    if (!op || !x || !y || nrhs < 1 || op->partial || op->opts.k_cut > 0) return -1;
    if (op->opts.kind == 0) return fwd_sym_d(op, x, nrhs, y);
    int64_t N = (int64_t)op->n * op->n;
    const double complex* xz = (const double complex*)x;
    double complex* yz = (double complex*)y;
    double complex* xs = (double complex*)malloc(sizeof(double complex) * (size_t)N * nrhs);
    for (int c = 0; c < nrhs; ++c)
        for (int64_t g = 0; g < N; ++g) xs[(size_t)c * N + g] = xz[(size_t)c * N + g] / op->s[g];
    int rc = fwd_sym_z(op, xs, nrhs, yz);     /* A = S A_s S^{-1} (the symmetric form) */
    for (int c = 0; c < nrhs; ++c)
        for (int64_t g = 0; g < N; ++g) yz[(size_t)c * N + g] *= op->s[g];
    free(xs);
    return rc;
}

int ro_solve(const ro_op* op, const double* f, int nrhs, double* x)
{
    if (!op || !f || !x || nrhs < 1 || op->partial) return -1;
    if (op->opts.kind == 0) return solve_sym_d(op, f, nrhs, x);
    int64_t N = (int64_t)op->n * op->n;
    const double complex* fz = (const double complex*)f;
    double complex* xz = (double complex*)x;
    double complex* ft = (double complex*)malloc(sizeof(double complex) * (size_t)N * nrhs);
    for (int c = 0; c < nrhs; ++c)
        for (int64_t g = 0; g < N; ++g) ft[(size_t)c * N + g] = fz[(size_t)c * N + g] / op->s[g];
    int rc = solve_sym_z(op, ft, nrhs, xz);
    for (int c = 0; c < nrhs; ++c)
        for (int64_t g = 0; g < N; ++g) xz[(size_t)c * N + g] *= op->s[g];
    free(ft);
    return rc;
}

static void lr_free(ro_lr* L)
{
    free(L->sk); free(L->rs); free(L->C); free(L->T);
    memset(L, 0, sizeof *L);
}

void ro_free(ro_op* op)
{
    if (!op) return;
    if (op->lev) {
        for (int l = 1; l <= op->d; ++l) {
            if (!op->lev[l]) continue;
            for (int j = 0; j < (1 << l); ++j) {
                ro_box* B = &op->lev[l][j];
                free(B->active); free(B->near); free(B->skel); free(B->sk_local); free(B->rs_local);
                free(B->T); free(B->Finv); free(B->E);
                ro_hss1d_free(B->H_ss); ro_hss1d_free(B->H_rr); ro_hss1d_free(B->H_E);
                lr_free(&B->L_sr); lr_free(&B->L_rs); lr_free(&B->L_T);
            }
            free(op->lev[l]);
        }
        free(op->lev);
    }
    free(op->a); free(op->s); free(op->pcos); free(op->psin); free(op->active0); free(op->root_inv);
    free(op);
}

/* ------------------------------------------------------------------ inspection */

static const ro_box* getbox(const ro_op* op, int l, int j)
{
    if (!op || l < 1 || l > op->d || j < 0 || j >= (1 << l)) return NULL;
    return &op->lev[l][j];
}

int ro_depth(const ro_op* op) { return op ? op->d : -1; }

int ro_box_sizes(const ro_op* op, int l, int j, int* m, int* k, int* r, int* nnear)
{
    const ro_box* B = getbox(op, l, j);
    if (!B) return -1;
    if (m) *m = B->m;
    if (k) *k = B->k;
    if (r) *r = B->r;
    if (nnear) *nnear = B->nnear;
    return 0;
}

int ro_box_active(const ro_op* op, int l, int j, int64_t* out)
{
    const ro_box* B = getbox(op, l, j);
    if (!B) return -1;
    memcpy(out, B->active, sizeof(int64_t) * (size_t)B->m);
    return 0;
}

int ro_box_skel(const ro_op* op, int l, int j, int64_t* out)
{
    const ro_box* B = getbox(op, l, j);
    if (!B) return -1;
    memcpy(out, B->skel, sizeof(int64_t) * (size_t)B->k);
    return 0;
}

int ro_box_near(const ro_op* op, int l, int j, int64_t* out)
{
    const ro_box* B = getbox(op, l, j);
    if (!B || !B->near) return -1;           /* translation-invariant mode: no per-box list */
    memcpy(out, B->near, sizeof(int64_t) * (size_t)B->nnear);
    return 0;
}

static size_t esz(const ro_op* op) { return op->opts.kind == 1 ? 2 * sizeof(double) : sizeof(double); }

int ro_box_T(const ro_op* op, int l, int j, double* out)
{
    const ro_box* B = getbox(op, l, j);
    if (!B) return -1;
    memcpy(out, B->T, esz(op) * (size_t)B->k * (size_t)(B->m - B->k));
    return 0;
}

int ro_box_Finv(const ro_op* op, int l, int j, double* out)
{
    const ro_box* B = getbox(op, l, j);
    if (!B) return -1;
    memcpy(out, B->Finv, esz(op) * (size_t)B->m * (size_t)B->m);
    return 0;
}

int ro_box_E(const ro_op* op, int l, int j, double* out)
{
    const ro_box* B = getbox(op, l, j);
    if (!B) return -1;
    memcpy(out, B->E, esz(op) * (size_t)B->k * (size_t)B->k);
    return 0;
}

int ro_root_size(const ro_op* op) { return op ? op->m0 : -1; }

int ro_root_inv(const ro_op* op, double* out)
{
    if (!op) return -1;
    memcpy(out, op->root_inv, esz(op) * (size_t)op->m0 * (size_t)op->m0);
    return 0;
}

/* ------------------------------------------------------------------ brute force */

/* Entry of the system matrix as posed (not symmetrised): Laplace as in entry_d,
 * Helmholtz A_gg' = kappa^2 b_g (i/4) H0(kappa r) h^2, A_gg = a_g + kappa^2 b_g (i/4) int_cell H0. */
typedef struct { int n; double h, c0, lself; double complex hself; int kind; double kappa; } bf_ctx;

static void bf_init(bf_ctx* c, int n, int kind, double kappa)
{
    c->n = n; c->h = 1.0 / n; c->kind = kind; c->kappa = kappa;
    c->c0 = -(c->h * c->h) / (4.0 * M_PI);
    c->lself = -ro_laplace_cell_integral(c->h) / (2.0 * M_PI);
    c->hself = 0.0;
    if (kind == 1) {
        double re, im;
        ro_helmholtz_cell_integral(c->h, kappa, 32, &re, &im);
        c->hself = 0.25 * I * (re + I * im);
    }
}

static double complex bf_entry(const bf_ctx* c, const double* a, const double* b, int64_t g, int64_t gp)
{
    double ag = a ? a[g] : 1.0;
    if (c->kind == 0) {
        if (g == gp) return ag + c->lself;
        double x = ((double)(g % c->n) + 0.5) * c->h, y = ((double)(g / c->n) + 0.5) * c->h;
        double xp = ((double)(gp % c->n) + 0.5) * c->h, yp = ((double)(gp / c->n) + 0.5) * c->h;
        double dx = x - xp, dy = y - yp;
        return c->c0 * log(dx * dx + dy * dy);
    }
    double bg = b ? b[g] : 1.0;
    double kb = c->kappa * c->kappa * bg;
    if (g == gp) return ag + kb * c->hself;
    double x = ((double)(g % c->n) + 0.5) * c->h, y = ((double)(g / c->n) + 0.5) * c->h;
    double xp = ((double)(gp % c->n) + 0.5) * c->h, yp = ((double)(gp / c->n) + 0.5) * c->h;
    double dx = x - xp, dy = y - yp;
    double z = c->kappa * sqrt(dx * dx + dy * dy);
    return kb * 0.25 * I * (j0(z) + I * y0(z)) * (c->h * c->h);
}

void ro_entry(int n, int kind, double kappa, const double* a, const double* b, int64_t g,
              int64_t gp, double* re, double* im)
{
    bf_ctx c;
    bf_init(&c, n, kind, kappa);
    double complex v = bf_entry(&c, a, b, g, gp);
    *re = creal(v); *im = cimag(v);
}

int ro_matvec_rows(int n, int kind, double kappa, const double* a, const double* b,
                   const double* x, int nrhs, const int64_t* rows, int nrows, double* y)
{
    if (n < 1 || nrhs < 1 || !x || !y || (kind != 0 && kind != 1)) return -1;
    bf_ctx c;
    bf_init(&c, n, kind, kappa);
    int64_t N = (int64_t)n * n;
    #pragma omp parallel for schedule(dynamic)
    for (int q = 0; q < nrows; ++q) {
        int64_t g = rows[q];
        for (int col = 0; col < nrhs; ++col) {
            if (kind == 0) {
                double s = 0.0;
                for (int64_t gp = 0; gp < N; ++gp) s += creal(bf_entry(&c, a, b, g, gp)) * x[(size_t)col * N + gp];
                y[(size_t)col * nrows + q] = s;
            } else {
                const double complex* xz = (const double complex*)x;
                double complex s = 0.0;
                for (int64_t gp = 0; gp < N; ++gp) s += bf_entry(&c, a, b, g, gp) * xz[(size_t)col * N + gp];
                ((double complex*)y)[(size_t)col * nrows + q] = s;
            }
        }
    }
    return 0;
}

int ro_matvec(int n, int kind, double kappa, const double* a, const double* b, const double* x,
              int nrhs, double* y)
{
    int64_t N = (int64_t)n * n;
    int64_t* rows = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
    for (int64_t g = 0; g < N; ++g) rows[g] = g;
    int rc = ro_matvec_rows(n, kind, kappa, a, b, x, nrhs, rows, (int)N, y);
    free(rows);
    return rc;
}

/* ------------------------------------------------------------------ HSS1D (Sec. 3) */

int ro_hss1d_build(int cplx, const double* M, int n, const int* order, int leaf, double eps,
                   ro_hss** out)
{
    if (!M || !out || n < 1 || leaf < 1 || eps < 0.0) return -1;
    if (order) {
        char* seen = (char*)calloc((size_t)n, 1);
        for (int p = 0; p < n; ++p) {
            if (order[p] < 0 || order[p] >= n || seen[order[p]]) { free(seen); return -1; }
            seen[order[p]] = 1;
        }
        free(seen);
    }
    ro_hss* h = (ro_hss*)calloc(1, sizeof(ro_hss));
    int rc = cplx ? hss_build_z((const double complex*)M, n, order, leaf, eps, h)
                  : hss_build_d(M, n, order, leaf, eps, h);
    if (rc) { ro_hss1d_free(h); return rc; }
    *out = h;
    return 0;
}

int ro_hss1d_apply(const ro_hss* h, const double* x, int nrhs, double* y)
{
    if (!h || !x || !y || nrhs < 1) return -1;
    if (h->cplx) hss_apply_z(h, (const double complex*)x, nrhs, (double complex*)y);
    else hss_apply_d(h, x, nrhs, y);
    return 0;
}

int ro_hss1d_depth(const ro_hss* h) { return h ? h->depth : -1; }

int ro_hss1d_node(const ro_hss* h, int level, int j, int* lo, int* hi, int* a, int* k,
                  int* skel_rows, double* T)
{
    if (!h || level < 1 || level > h->depth || j < 0 || j >= (1 << level)) return -1;
    const ro_hnode* q = &h->node[level][j];
    if (lo) *lo = q->lo;
    if (hi) *hi = q->hi;
    if (a) *a = q->a;
    if (k) *k = q->k;
    if (skel_rows)
        for (int s = 0; s < q->k; ++s) skel_rows[s] = q->act[q->sk[s]];
    if (T) memcpy(T, q->T, (h->cplx ? 2 : 1) * sizeof(double) * (size_t)q->k * (size_t)(q->a - q->k));
    return 0;
}

int64_t ro_hss1d_entries(const ro_hss* h)
{
    if (!h) return -1;
    int t = h->depth;
    if (t == 0) return (int64_t)h->n * h->n;
    int64_t e = 0;
    for (int l = 1; l <= t; ++l)
        for (int j = 0; j < (1 << l); ++j) e += (int64_t)h->node[l][j].k * (h->node[l][j].a - h->node[l][j].k);
    for (int l = 0; l < t; ++l)
        for (int j = 0; j < (1 << l); ++j) e += 2 * (int64_t)h->node[l + 1][2 * j].k * h->node[l + 1][2 * j + 1].k;
    for (int j = 0; j < (1 << t); ++j) e += (int64_t)h->node[t][j].a * h->node[t][j].a;
    return e;
}

void ro_hss1d_free(ro_hss* h)
{
    if (!h) return;
    int t = h->depth;
    if (h->node)
        for (int l = 1; l <= t; ++l) {
            if (!h->node[l]) continue;
            for (int j = 0; j < (1 << l); ++j) {
                ro_hnode* q = &h->node[l][j];
                free(q->act); free(q->sk); free(q->rs); free(q->T);
            }
            free(h->node[l]);
        }
    int nint = (1 << t);
    if (h->B12) for (int i = 0; i < nint; ++i) free(h->B12[i]);
    if (h->B21) for (int i = 0; i < nint; ++i) free(h->B21[i]);
    if (h->D) for (int i = 0; i < nint; ++i) free(h->D[i]);
    free(h->node); free(h->B12); free(h->B21); free(h->D); free(h->order);
    free(h);
}

const ro_hss* ro_box_hss(const ro_op* op, int level, int j, int which)
{
    const ro_box* B = getbox(op, level, j);
    if (!B || !B->hss) return NULL;
    return which == 0 ? B->H_ss : which == 1 ? B->H_rr : which == 2 ? B->H_E : NULL;
}

int ro_box_lr_rank(const ro_op* op, int level, int j, int which)
{
    const ro_box* B = getbox(op, level, j);
    if (!B || !B->hss) return -1;
    return which == 0 ? B->L_sr.k : which == 1 ? B->L_rs.k : which == 2 ? B->L_T.k : -1;
}

int ro_box_order(const ro_op* op, int level, int j, int which, int* out)
{
    const ro_box* B = getbox(op, level, j);
    if (!B || !out || (which != 0 && which != 1)) return -1;
    if (which == 0) { box_cyclic_order(op, level, j, B->skel, B->k, out); return 0; }
    int nr = B->m - B->k;
    int64_t* rg = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nr + 1));
    for (int c = 0; c < nr; ++c) rg[c] = B->active[B->rs_local[c]];
    box_interface_order(op, level, rg, nr, out);
    free(rg);
    return 0;
}

static int64_t lr_entries(const ro_lr* L) { return (int64_t)L->p * L->k + (int64_t)L->k * (L->q - L->k); }

int64_t ro_compressed_entries(const ro_op* op, int64_t* dense_entries)
{
    if (!op) return -1;
    int64_t c = 0, d = 0;
    for (int l = 1; l <= op->d; ++l)
        for (int j = 0; j < (1 << l); ++j) {
            const ro_box* B = &op->lev[l][j];
            if (!B->hss) continue;
            int64_t m = B->m, k = B->k;
            d += m * m + k * k + k * (m - k);
            c += ro_hss1d_entries(B->H_ss) + ro_hss1d_entries(B->H_rr) + ro_hss1d_entries(B->H_E) +
                 lr_entries(&B->L_sr) + lr_entries(&B->L_rs) + lr_entries(&B->L_T);
        }
    if (dense_entries) *dense_entries = d;
    return c;
}
