/*
 * rs_oracle.h -- plain, slow CPU oracle of the dense-block recursive-skeletonization
 * inverse of Corona, Martinsson & Zorin, "An O(N) Direct Solver for Integral Equations
 * on the Plane" (arXiv:1303.5466).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library against the
 * paper.  Only tests, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (paper references are to sections, equations and algorithms):
 *   - Nystrom matrix on an n x n cell-centre grid of [0,1]^2 (Sec. 5, general formulation):
 *       Laplace:   A_gg' = -(1/2pi) h^2 log|x_g - x_g'|,  A_gg = a_g - (1/2pi) C_h
 *       Helmholtz: A_gg' = kappa^2 b_g (i/4) H0(kappa r) h^2,
 *                  A_gg  = a_g + kappa^2 b_g (i/4) * (integral of H0 over the h x h cell),
 *                  factored in the symmetric form of Eq. (5.6), S^{-1} A S with
 *                  S = diag(kappa sqrt(b)); ro_solve takes and returns the unscaled f, x
 *   - binary tree by alternating bisection (Sec. 2.2), proxy-accelerated IDs (Sec. 2.2,
 *     Eq. 2.1), the HSS inversion of Algorithm 1 with the E formula of Algorithm 2,
 *     and the inverse apply of Algorithm 6 restated from Eqs. (2.10)-(2.12).
 *
 * All arrays are host memory, caller-owned unless stated.  Complex values are interleaved
 * (re, im) doubles.  Functions return 0 on success and a negative value on bad input.
 */
#ifndef RS_ORACLE_H
#define RS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ro_op ro_op;

typedef struct {
    int kind;                    /* 0 = Laplace, 1 = Helmholtz (complex)                  */
    double kappa;                /* Helmholtz wavenumber                                   */
    int proxy_points;            /* P points on the proxy circle; 0 = no proxy rows        */
    double proxy_radius_factor;  /* R = factor * (larger box half-width)                   */
    int near_all;                /* 1: rows = every other box's active points (the full
                                    off-diagonal block row of Sec. 2.2, no acceleration)   */
    int threads;                 /* OpenMP threads over the boxes of a level (<=0: default) */
    int max_levels;              /* >0: factor only the max_levels finest levels and stop
                                    (a bounded sample for timing; ro_solve then refuses)   */
    int k_cut;                   /* >0: boxes with k > k_cut keep phi^{sk}, phi^{rs} and E
                                    in HSS1D form and phi^{s<-r}, phi^{r<-s}, T in low-rank
                                    form (Sec. 3), compressed at eps from the dense blocks;
                                    ro_solve uses these forms for those boxes              */
    int hss_leaf;                /* largest leaf run of the HSS1D trees                    */
    double hss_eps;              /* ID tolerance of that compression (0: eps)              */
    int ti;                      /* 1: translation-invariant mode (a and b constant): one
                                    ID and one set of blocks per level, taken on box 0
                                    with all eight neighbours present (Sec. 5, one set of
                                    matrices per level) and copied to every box           */
} ro_opts;

typedef struct ro_hss ro_hss;

void ro_opts_default(ro_opts* o);

/* Exact integral of log|y - x| over the h x h cell centred at x (Laplace diagonal). */
double ro_laplace_cell_integral(double h);
/* Integral of H0^(1)(kappa |y - x|) over the h x h cell centred at x (re, im out). */
void ro_helmholtz_cell_integral(double h, double kappa, int nodes, double* re, double* im);

/* Gauss-Legendre nodes/weights on [-1,1] (used by the Helmholtz cell integral). */
void ro_gauss_legendre(int n, double* x, double* w);

/* Column-pivoted Householder QR interpolative decomposition (Sec. 2.1, Eq. 2.1).
 * Pivots compare squared column norms with their 40 low mantissa bits cleared; ties go to
 * the lowest column index.
 * Y: r x m row-major (real: r*m doubles; complex: 2*r*m).  Outputs k, perm (m entries:
 * pivot order, first k = skeleton), T (k x (m-k) row-major, rows/cols in pivot order). */
int ro_id(int cplx, const double* Y, int r, int m, double eps, int* k_out, int* perm,
          double* T);

/* Inverse by LU with partial pivoting.  A, Ainv: m x m row-major. */
int ro_inverse(int cplx, const double* A, int m, double* Ainv);

/* Factor (Algorithm 1) for the n x n grid with leaf_side x leaf_side leaves.
 * a: N values (grid order g = i1 + n*i2) or NULL (= 1); b: N values of b(x) (Helmholtz)
 * or NULL (= 1). */
int ro_factor(int n, int leaf_side, const double* a, const double* b, double eps,
              const ro_opts* opts, ro_op** out);
/* y = A x through the HSS form of A that the factorization's IDs define (skeleton
 * interactions between siblings at every level, the IDs' T on both sides, dense leaf blocks):
 * the O(N) forward operator of the compressed matrix.  Its error against A x is of the order
 * of eps.  Refused for a partial factorization and with k_cut > 0.  x, y as for ro_solve. */
int ro_fwd_apply(const ro_op* op, const double* x, int nrhs, double* y);
/* Inverse apply (Algorithm 6).  f, x: N x nrhs column-major in grid order. */
int ro_solve(const ro_op* op, const double* f, int nrhs, double* x);
void ro_free(ro_op* op);

/* Inspection.  Levels are 0 (root) .. d (leaves); boxes 0 .. 2^l - 1. */
int ro_depth(const ro_op* op);
int ro_box_sizes(const ro_op* op, int level, int box, int* m, int* k, int* r, int* nnear);
int ro_box_active(const ro_op* op, int level, int box, int64_t* out);   /* m globals   */
int ro_box_skel(const ro_op* op, int level, int box, int64_t* out);     /* k globals,
                                                                           ascending   */
int ro_box_near(const ro_op* op, int level, int box, int64_t* out);     /* nnear       */
int ro_box_T(const ro_op* op, int level, int box, double* out);  /* k x (m-k), rows in
                                 skeleton (ascending global) order, columns in residual
                                 (ascending local) order                                 */
int ro_box_Finv(const ro_op* op, int level, int box, double* out);  /* m x m            */
int ro_box_E(const ro_op* op, int level, int box, double* out);     /* k x k            */
int ro_root_size(const ro_op* op);
int ro_root_inv(const ro_op* op, double* out);

/* HSS1D compression (Sec. 3.2) of an explicit n x n matrix M (row-major; complex:
 * interleaved) along the ordering order[position] = row (NULL: identity).  The tree halves
 * runs of positions until they hold at most `leaf`; node (l, j) covers positions
 * [floor(j n/2^l), floor((j+1) n/2^l)).  Each node's active columns (leaf: its positions;
 * above: the children's skeletons) get one ID at eps of [M(out, act); M(act, out)^T]
 * (out = every position outside the node), giving the telescoping form of Eq. 2.9. */
int ro_hss1d_build(int cplx, const double* M, int n, const int* order, int leaf, double eps,
                   ro_hss** out);
/* y = M x through the HSS1D form; x, y: n x nrhs row-major, indexed by row of M. */
int ro_hss1d_apply(const ro_hss* h, const double* x, int nrhs, double* y);
int ro_hss1d_depth(const ro_hss* h);
/* Node (level 1..depth, j): position range, active and skeleton sizes; skel_rows (k rows of
 * M, ascending local order) and T (k x (a-k) row-major) when non-NULL. */
int ro_hss1d_node(const ro_hss* h, int level, int j, int* lo, int* hi, int* a, int* k,
                  int* skel_rows, double* T);
/* Scalars stored by the form (T blocks, sibling blocks, leaf blocks). */
int64_t ro_hss1d_entries(const ro_hss* h);
void ro_hss1d_free(ro_hss* h);

/* Compressed blocks of box (level, j) when the factorization ran with k_cut (NULL / -1
 * otherwise): which = 0 phi^{sk}, 1 phi^{rs}, 2 E for the HSS1D forms; low-rank ranks
 * which = 0 phi^{s<-r}, 1 phi^{r<-s}, 2 T. */
const ro_hss* ro_box_hss(const ro_op* op, int level, int j, int which);
int ro_box_lr_rank(const ro_op* op, int level, int j, int which);
/* Orders of Sec. 3.1 for box (level, j): which = 0 skeleton cyclically around the box
 * (k entries: skeleton index at each position), 1 residual along the interface (m-k). */
int ro_box_order(const ro_op* op, int level, int j, int which, int* out);
/* Stored scalars of the compressed boxes' forms; *dense_entries (optional) receives what
 * the same blocks take densely (m^2 + k^2 + k(m-k) per box). */
int64_t ro_compressed_entries(const ro_op* op, int64_t* dense_entries);

/* Brute-force y = A x over all N x N entries (nrhs columns, grid order). */
int ro_matvec(int n, int kind, double kappa, const double* a, const double* b,
              const double* x, int nrhs, double* y);
/* Rows `rows[0..nrows)` of A x (nrhs columns): y is nrows x nrhs column-major. */
int ro_matvec_rows(int n, int kind, double kappa, const double* a, const double* b,
                   const double* x, int nrhs, const int64_t* rows, int nrows, double* y);
/* One dense entry A(g, g') (re, im). */
void ro_entry(int n, int kind, double kappa, const double* a, const double* b,
              int64_t g, int64_t gp, double* re, double* im);

#ifdef __cplusplus
}
#endif
#endif
