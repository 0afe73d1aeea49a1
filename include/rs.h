/*
 * rs.h -- C ABI of the GB300 (sm_103a) recursive-skeletonization direct solver for 2D
 * volume integral equations (Corona, Martinsson & Zorin, arXiv:1303.5466).
 *
 * The problem (Sec. 5, "General formulation"): on the n x n cell-centre grid
 * x_g = ((i1+1/2)h, (i2+1/2)h) of [0,1]^2, h = 1/n, solve A sigma = f with the Nystrom
 * matrix
 *   Laplace   (RS_LAPLACE):   A_gg' = -(1/2pi) h^2 log|x_g - x_g'|,
 *                             A_gg  = a_g - (1/2pi) int_cell log|y - x_g| dy;
 *   Helmholtz (RS_HELMHOLTZ): A_gg' = kappa^2 b_g (i/4) H0^(1)(kappa|x_g - x_g'|) h^2,
 *                             A_gg  = a_g + kappa^2 b_g (i/4) int_cell H0^(1)(kappa|y - x_g|) dy,
 *     factored in the symmetric form of Eq. (5.6) (diagonal similarity by kappa sqrt(b)).
 * The factorization is the dense-block HSS inverse of Algorithm 1 (with the E formula of
 * Algorithm 2), built level by level over a binary tree (Sec. 2.2) with proxy-accelerated
 * interpolative decompositions (Sec. 2.2, Eq. 2.1); the solve is the inverse apply of
 * Algorithm 6.  Every floating-point step runs in this library's CUDA kernels on the
 * current device; the host side does integer bookkeeping only.
 *
 * Conventions for every function below:
 *   - return 0 (RS_OK) on success or a negative RS_E_* code; nothing aborts, traps or exits;
 *     rs_last_error() gives a thread-local message for the last failure on this thread;
 *   - "host" pointers are ordinary CPU memory, "device" pointers are CUDA global memory of
 *     the current device; arrays are caller-owned and only read/written during the call
 *     unless stated otherwise;
 *   - rs_tree and rs_op objects are owned by the library until rs_free_tree / rs_free;
 *   - point order: the caller's order of `points` ("input order") is used for every
 *     per-point array (a, b, f, x); the library permutes internally;
 *   - grid index g = i1 + n*i2 identifies a point in the inspection functions;
 *   - complex values are interleaved (re, im) doubles.
 */
#ifndef RS_H
#define RS_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    RS_OK = 0,
    RS_E_INVALID = -1,        /* bad argument or size                                   */
    RS_E_NOT_GRID = -2,       /* points are not the cell centres of a uniform n x n grid */
    RS_E_NOMEM = -3,          /* host or device allocation failed                       */
    RS_E_SINGULAR = -4,       /* a pivot fell below 1e3 * unit roundoff * largest earlier */
    RS_E_NOT_CONVERGED = -5,  /* iterative refinement did not reach its tolerance        */
    RS_E_TIMEOUT = -6,        /* a bounded device-side wait expired                      */
    RS_E_CUDA = -7            /* a CUDA runtime call failed                              */
};

typedef enum { RS_LAPLACE = 0, RS_HELMHOLTZ = 1 } rs_kernel_kind;
typedef enum { RS_FP64 = 0, RS_MIXED_FP32 = 1, RS_C64_REFINED = 2, RS_C128 = 3 } rs_precision;

typedef struct rs_tree rs_tree;
typedef struct rs_op rs_op;
typedef struct rs_server rs_server;

/* Kernel of the integral operator.  b: host, N values of b(x) in input order, or NULL
 * (b = 1); must be > 0 everywhere for RS_HELMHOLTZ (the symmetric form divides by it). */
typedef struct {
    rs_kernel_kind kind;
    double kappa;
    const double* b;
} rs_kernel;

/* Factorization options; rs_opts_default() fills the values listed here. */
typedef struct {
    int proxy_points;            /* points on the proxy circle (Sec. 2.2)            [64]   */
    double proxy_radius_factor;  /* proxy radius / larger box half-width             [1.5]  */
    rs_precision precision;      /* arithmetic of the factorization                  [FP64] */
    double refine_tol;           /* target relative residual of the refined solve    [1e-10]*/
    int refine_max_iter;         /* refinement cap; past it RS_E_NOT_CONVERGED        [10]   */
    int64_t k_cut;               /* extra compression of Sec. 3: boxes whose skeleton has
                                    more than k_cut points keep phi^{sk}, phi^{rs} (the
                                    diagonal blocks of Pi^T F^{-1} Pi) and E in HSS1D form
                                    and phi^{s<-r}, phi^{r<-s} and T in low-rank form, each
                                    compressed at eps from its dense block after the
                                    factorization; the solve then applies those forms.
                                    0 = never                                        [0]    */
    int64_t spin_limit;          /* iteration cap of every device-side wait          [2^26] */
    int profile;                 /* 1: time every kernel launch with CUDA events on the
                                    launch stream (rs_op_profile)                     [0]    */
    int hss_leaf;                /* largest leaf run of the HSS1D trees (k_cut > 0)  [64]   */
    double hss_eps;              /* ID tolerance of that compression; 0 = eps         [0]    */
    int solve_graph;             /* 1: rs_solve of RS_FP64 / RS_C128 operators replays a CUDA
                                    graph of the whole inverse apply, captured once per nrhs
                                    (inputs staged through library buffers); 0: launch the
                                    kernels one by one                                [1]    */
    int per_box;                 /* 1: launch every factor and solve kernel for one box at a
                                    time (each box gets the whole GPU), the unbatched form
                                    that the per-level launches are measured against; same
                                    arithmetic up to rounding order                   [0]    */
    int spd_inverse;             /* 1: invert F, E and the root of a real symmetric kernel
                                    (RS_LAPLACE) by the symmetric sweep without pivoting
                                    (half the flops of Gauss-Jordan); when the pivots show
                                    a block that is not positive definite to working
                                    accuracy, the inversions are redone with pivoted
                                    Gauss-Jordan (all of them with the per-level launches,
                                    whose status is read once after the root; the failing
                                    level's in the per-box and translation-invariant modes;
                                    rs_stats.spd_fallbacks).  0: always pivoted GJ  [1]    */
    int cpqr_variant;            /* form of the column-pivoted QR (Eq. 2.1) on every level:
                                    0 = two passes over the open columns per step, 4 rows
                                    per lane in flight; 1 = the same with 8; 2 = look-ahead
                                    (one pass per step: the update of step s fused with the
                                    dot products of step s+1); 3 = 0 with the lists of open
                                    columns in global memory (taken by 0 and 1 by themselves
                                    for boxes whose lists do not fit shared memory); 4 =
                                    each box held in the shared memory of one thread-block
                                    cluster for the whole factorization (levels whose boxes
                                    fit 16 CTAs; the others take the default); 5 = 0 with
                                    eight columns per warp pass, their dot products summed
                                    by recursive halving across the lanes and the per-column
                                    bookkeeping done once per column; 6 = 0 with 2 rows per
                                    lane in flight and registers capped for five CTAs per SM;
                                    7 / 8 = blocked: the trailing updates deferred over
                                    panels of 16 / 8 steps, so a step reads each open column
                                    once (real scalars and boxes whose lists fit shared
                                    memory; the others take the default); -1 = the
                                    autotuner's table (rs_autotune), else 0 or 1 by
                                    occupancy. Same result up to rounding order       [-1]   */
    int translation_invariant;   /* a(x) (and b(x)) constant, so A depends only on the
                                    offset between grid points (Sec. 5: one set of matrix
                                    blocks per level).  1: each level's ID is taken once, on
                                    box 0 with all eight same-level neighbours present (also
                                    where they fall outside the unit square), and its T,
                                    F^{-1} and E are stored once and shared by every box of
                                    the level.  2: boxes whose active points, near points
                                    and children are translates of one another share one
                                    factored box (the per-box result, each distinct box
                                    factored once: ~13-24 per level at any grid size).
                                    Refused with varying a or b, with k_cut > 0, and for
                                    9 N > 2^31 - 1 (mode 1)                           [0]    */
    int sweep_panel;             /* panel width of the symmetric sweep (spd_inverse): 8 or
                                    16 columns per step (16: twice the FMAs per element
                                    loaded, half the steps); 0 = the autotuner's table,
                                    else 8                                            [0]    */
    int forward_only;            /* 1: the tree build alone (the IDs of every level, Sec. 2.2):
                                    the operator serves rs_fwd_apply (the compressed forward
                                    operator), rs_residual and rs_bicgstab's matvec, not
                                    rs_solve.  Not with translation_invariant, k_cut or
                                    per_box                                           [0]    */
    int gemm_form;               /* dense products of RS_FP64 operators (E of Algorithm 1,
                                    the inverses of F, E and the root in panels of 64, the
                                    block updates of T = R11^{-1} R12): 1 = exact products
                                    of 7-bit digit slices on the bf16 tensor cores, summed
                                    in integers (one rounding per entry; parts below 2^-56
                                    of the row and column maxima left out); 0 = FP64 FMA
                                    tiles and the element sweep                       [1]    */
} rs_opts;

void rs_opts_default(rs_opts* opts);
const char* rs_last_error(void);

/* Tree (Sec. 2.2): binary bisection of [0,1]^2, splitting x1 at even depth and x2 at odd
 * depth; box j of level l has children 2j (lower half) and 2j+1 (upper half); leaves are
 * leaf_side x leaf_side points at depth d = 2 log2(n / leaf_side).
 * points: host, N x 2 row-major (x1, x2), any order.  N must equal n^2 with
 * n = leaf_side * 2^L, L >= 1 (else RS_E_INVALID); points must be the cell centres of
 * [0,1]^2 up to 1e-9 h (else RS_E_NOT_GRID).  *out is owned by the caller until
 * rs_free_tree. */
int rs_build_tree(const double* points, int64_t N, int leaf_side, rs_tree** out);
void rs_free_tree(rs_tree* tree);
/* n (points per side), depth d, and (optional) grid index g of each input point. */
int rs_tree_info(const rs_tree* tree, int64_t* n_side, int* depth, int64_t* grid_index_of_input);

/* Host bookkeeping of one level, exposed for tests (no GPU needed).  Leaf level: the
 * boxes' points ascending in g.  Level l < d: box j's active set is the skeleton of child
 * 2j followed by that of child 2j+1, each ascending in g, given in child_k (2^(l+1)
 * counts) and child_skel (their concatenation).  Near rows of box j: active points of the
 * same-level boxes whose closed rectangles touch box j, strictly inside its proxy circle,
 * in (neighbour box, active) order.  Outputs: m[2^l], nnear[2^l]; when act / near are
 * non-NULL they receive the concatenations (caller sizes them from a first call). */
int rs_tree_level_sets(const rs_tree* tree, int level, const int64_t* child_k,
                       const int64_t* child_skel, double proxy_radius_factor,
                       int64_t* m, int64_t* act, int64_t* nnear, int64_t* near);

/* Factor (Algorithm 1; Algorithm 2 for E).  kernel: see rs_kernel.  a: host, N
 * values of a(x) in input order, or NULL (a = 1).  eps: ID tolerance; a CPQR step is kept
 * while |R_ss| > eps |R_00| (Eq. 2.1).  opts: NULL = defaults.  stream: cudaStream_t or
 * NULL (legacy default stream).  The factors stay resident on the current device until
 * rs_free.  The call is synchronous with respect to the host. */
int rs_factor(const rs_tree* tree, const rs_kernel* kernel, const double* a, double eps,
              const rs_opts* opts, void* stream, rs_op** out);

/* Inverse apply (Algorithm 6): x = A^{-1} f for nrhs right-hand sides.  f, x: N x nrhs
 * column-major in input order, double (Laplace) or interleaved complex128 (Helmholtz);
 * either both device pointers or both host pointers (detected per call; host buffers are
 * staged through device memory inside the call).  Device buffers must live on the
 * operator's GPU (memory of another GPU: RS_E_INVALID).  x may not alias f.  The call returns
 * after x is written (host) or after the work is enqueued on `stream` (device). */
int rs_solve(rs_op* op, const void* f, int64_t nrhs, void* x, void* stream);
/* Forward apply y = A x through the HSS form of A that the factorization's IDs define: the
 * off-diagonal blocks A(I_i, I_j) ~ L_i A(sk_i, sk_j) R_j (Sec. 2.2, the ID of Eq. 2.1 on both
 * sides), nested level by level (the telescoping form of Eq. 2.9), with the two children's
 * mutual blocks at every level and the leaves' diagonal blocks generated on the fly.  O(N) work
 * and no storage beyond the factor's T; its error against A x is of the order of eps (for
 * Helmholtz, in the symmetric form), and rs_solve inverts it to rounding.  x, y: as f, x of
 * rs_solve (y may not alias x).  RS_E_INVALID for operators with compressed boxes
 * (opts.k_cut > 0).  The call returns after y is written (host) or after the work is
 * enqueued on `stream` (device); it shares the operator's solve workspace, so it must not
 * run concurrently with rs_solve on the same operator. */
int rs_fwd_apply(rs_op* op, const void* x, int64_t nrhs, void* y, void* stream);
/* The preconditioned iterative solver of Sec. 5.4: BiCGstab on A x = f with the right
 * preconditioner M^{-1} (A M^{-1} y = f, x = M^{-1} y), one right-hand side.  A is applied
 * through its HSS form (rs_fwd_apply; a forward_only operator gives the tree build alone), M^{-1}
 * through rs_solve(M) -- e.g. A the Lippmann-Schwinger operator (Helmholtz, b varying) and M
 * the translation-invariant Helmholtz operator (b = 1).  f, x: device pointers, N values in
 * input order (double, or interleaved complex128 for Helmholtz); x may not alias f.  Stops when
 * the recursive residual |f - A x| / |f| (with A the HSS form) is at most tol; iters and
 * rel_res (host) report the iterations and that residual.  RS_E_NOT_CONVERGED after max_iter
 * iterations or on a breakdown (x then holds the last iterate).  Synchronous.  A and M must
 * share N and the kernel kind; M must be factored (not forward_only). */
int rs_bicgstab(rs_op* A, rs_op* M, const void* f, void* x, double tol, int max_iter, int* iters, double* rel_res,
                void* stream);
/* Check of the bounded device-side waits: one CTA enters the group barrier of the cooperative
 * kernels with a target that can never be reached.  The wait must end after `limit` polls and
 * the call returns RS_E_TIMEOUT (the expected outcome; RS_E_CUDA if the wait returned without
 * the timeout flag), with the CUDA context left usable.  stream: cudaStream_t or NULL.
 * Synchronous. */
int rs_wait_check(int64_t limit, void* stream);

/* Throughput probe of an FP64 pipe (no counterpart in the paper: it measures the roofline that
 * bounds the FP64 factorization of the work model of Sec. 4 on the present GPU).  kind:
 * RS_PROBE_DFMA, independent FP64 fused multiply-add chains on the CUDA cores; RS_PROBE_DMMA,
 * independent mma.sync m8n8k4 FP64 matrix instructions.  Each runs register-only chains on 16,
 * 32 and 64 warps per SM (DFMA: three chain layouts, eight chains sharing their operands or
 * four or two with their own); the best rate of three timed launches per shape (after one
 * warm-up, CUDA events on `stream`) gives *tflops_out (host).  Synchronous; allocates a few
 * KB of device memory.  RS_PROBE_BF16_MMA: mma.sync m16n8k16 bf16 products with FP32
 * accumulation, the pipe that the FP64 products of opts.gemm_form = 1 run on (flops of the bf16
 * products). */
enum { RS_PROBE_DFMA = 0, RS_PROBE_DMMA = 1, RS_PROBE_BF16_MMA = 2 };
int rs_fp64_probe(int kind, double* tflops_out, void* stream);
/* Release an operator.  Returns RS_E_INVALID, and frees nothing, while a server (or one of
 * its requests) still references it; NULL is accepted. */
int rs_free(rs_op* op);

/* Relative residuals |f_c - A x_c| / |f_c| of nrhs columns by an FP64 direct sum over all N^2
 * pairs (Laplace operators; the off-diagonal entries are tabulated over the (2n-1)^2 integer
 * offsets of the grid, one FMA per pair).  x, f: N x nrhs column-major FP64 in input order,
 * both device or both host.  rel_out: host, nrhs values.  Synchronous.  For RS_MIXED_FP32
 * operators rs_solve uses this residual for iterative refinement: x = 0, then repeatedly
 * x += A_eps^{-1} r, r = f - A x, until every column's relative residual is at most
 * opts.refine_tol (RS_E_NOT_CONVERGED after opts.refine_max_iter low-precision solves; x then
 * holds the last iterate). */
int rs_residual(rs_op* op, const void* x, const void* f, int64_t nrhs, double* rel_out, void* stream);

/* Inverse apply that allocates nothing.  This entry point has no counterpart in the paper; it
 * exists for callers that cannot allocate device memory while they serve solves: a process
 * whose device memory already belongs to another allocator or to fixed per-tenant budgets
 * (an extra cudaMalloc may fail or break the budget), or a latency-bound request path where a
 * cudaMalloc / cudaFree pair would synchronise the device.  rs_solve grows its workspace with
 * cudaMalloc on first use; rs_solve_noalloc computes the same x = A^{-1} f with its workspace
 * in one fixed device array of RS_NOALLOC_SCRATCH_DOUBLES doubles (32 MiB), which every GPU
 * that loads this library holds until the process exits, and calls no allocating routine.
 *   - f, x: device pointers on the operator's GPU only (host buffers, or memory of another
 *     GPU: RS_E_INVALID), N x nrhs column-major in input order; real FP64 operators only
 *     (RS_LAPLACE factored in RS_FP64);
 *   - the workspace grows linearly with nrhs (about 3 x N x nrhs doubles plus small terms);
 *     a request that does not fit (any nrhs above RS_NOALLOC_SCRATCH_DOUBLES / N among them,
 *     refused before any size arithmetic) returns RS_E_INVALID, names the size in
 *     rs_last_error(), and launches nothing;
 *   - the first call on a device looks up the array's device address (once per device, with
 *     that device current); make that first call before any stream capture;
 *   - all calls share the one array and each overwrites it: calls whose work overlaps on the
 *     GPU (different streams or threads) race and corrupt each other's results, so serialise
 *     them, e.g. on one stream;
 *   - returns once the work is enqueued on `stream`. */
#define RS_NOALLOC_SCRATCH_DOUBLES ((int64_t)4 << 20)
int rs_solve_noalloc(rs_op* op, const void* f, int64_t nrhs, void* x, void* stream);

/* Statistics of a factorization. */
typedef struct {
    int depth;
    int64_t n_side;
    int64_t root_m;
    int64_t bytes_factors;       /* device bytes of the stored factors (Phi, E, T, indices) */
    int64_t bytes_workspace;     /* device bytes of the solve workspace rs_solve has grown so
                                    far (0 until the first rs_solve; rs_solve_noalloc adds
                                    nothing)                                              */
    double flops_factor;         /* algorithmic flops of the factorization (the sum of the
                                    per-class formulas listed with RS_PROF_*)            */
    double flops_solve_per_rhs;  /* algorithmic flops of one inverse apply per RHS         */
    double bytes_solve;          /* factor bytes one inverse apply reads                   */
    double ms_tree;              /* wall time of the ID phase (Sec. 5 "tree build")        */
    double ms_inverse;           /* wall time of the inversion phase                       */
    int refine_iters;            /* RS_MIXED_FP32: low-precision solves of the last rs_solve */
    double refine_residual;      /* RS_MIXED_FP32: its final max relative FP64 residual     */
    int64_t compressed_boxes;    /* boxes in the compressed form of Sec. 3 (opts.k_cut)     */
    int64_t bytes_compressed;    /* device bytes of their compressed forms                 */
    int64_t bytes_dense_replaced;/* bytes the same blocks (Phi, E, T) take densely         */
    double ms_compress;          /* wall time of the compression                           */
    int spd_fallbacks;           /* inversions redone with pivoted Gauss-Jordan (opts.spd_inverse):
                                    with the per-level launches, a block found not SPD
                                    anywhere reruns every inversion of the factorization
                                    (2 x depth + 1); in the per-box and translation-invariant
                                    modes, those of the failing levels               */
    int refine_fp64_sums;        /* refined precisions: FP64 direct sums of the last rs_solve (the
                                    first residual, and each confirmation of the tolerance;
                                    the other corrections' products run in FP32)            */
} rs_stats;
int rs_op_stats(const rs_op* op, rs_stats* out);

/* Kernel classes timed when opts.profile is set.  Factor classes accumulate over rs_factor;
 * RS_PROF_SOLVE covers the kernels of the most recent rs_solve. */
enum {
    RS_PROF_ASSEMBLE_Y = 0,   /* Y = [K(near, I); K(proxy, I)] (work unit: entries)            */
    RS_PROF_CPQR = 1,         /* column-pivoted QR of Y (flops 4rmk - 2k^2(r+m) + 4k^3/3)       */
    RS_PROF_ID_T = 2,         /* T = R11^{-1} R12 (flops k^2 (m-k))                             */
    RS_PROF_ASSEMBLE_F = 3,   /* F (work unit: entries)                                         */
    RS_PROF_INV_F = 4,        /* F^{-1}: flops m^3 by the symmetric sweep, 2 m^3 by Gauss-Jordan  */
    RS_PROF_GEMM_E = 5,       /* W = F^{-1} L, E^{-1} = R W (flops 2m(m-k)k + 2k(m-k)k)          */
    RS_PROF_INV_E = 6,        /* E: flops k^3 by the sweep, 2 k^3 by Gauss-Jordan                 */
    RS_PROF_INV_ROOT = 7,     /* root F^{-1}: flops m^3 by the sweep, 2 m^3 by Gauss-Jordan       */
    RS_PROF_SOLVE = 8,        /* inverse apply (flops per RHS 2(2m^2 + 2k^2 + 2k(m-k)))         */
    RS_PROF_COUNT = 9
};
/* ms: summed event time; work: summed algorithmic flops (or entries); launches: count;
 * bytes: algorithmic bytes the class must move (solve: factor bytes read).  Any output may be
 * NULL.  Returns RS_E_INVALID for an unknown class. */
int rs_op_profile(const rs_op* op, int cls, double* ms, double* work, double* bytes, int64_t* launches);
/* ms: summed event time of the class's launches at tree level `level` (factor classes; the
 * root is level 0), 0 if none. */
int rs_op_profile_level(const rs_op* op, int cls, int level, double* ms);
/* Kernel launches made by this library in this process so far (all threads). */
int64_t rs_launch_count(void);

/* Autotuner (launch shapes; no counterpart in the paper).  Launch shapes -- the CTA-group size
 * of the CPQR and sweep kernels and the CPQR variant -- are chosen per level from the counts
 * of boxes and columns.  rs_autotune factors the given operator once with the current table
 * and once per candidate setting (each forced on every level, with per-level CUDA-event
 * timing), then records for every level's launch shape the fastest candidate of each kernel
 * in a process-wide table that later rs_factor calls consult; the table is written to `path`
 * as JSON unless path is NULL.  Choices never change what is computed: the CPQR variants
 * differ only in rounding order.  report may be NULL.  The table is shared by all threads;
 * while rs_autotune runs, its candidates apply to factorizations on the calling thread only.
 * rs_tune_load merges a file written by rs_tune_save into the table (RS_E_INVALID on any
 * malformed entry, leaving the table unchanged); rs_tune_clear empties it. */
typedef struct {
    int candidates;              /* settings timed                                         */
    int keys_set;                /* table entries written                                  */
    double default_factor_ms;    /* factor wall time with the table as it was              */
    double tuned_factor_ms;      /* factor wall time with the new table                    */
} rs_tune_report;
int rs_autotune(const rs_tree* tree, const rs_kernel* kernel, const double* a, double eps, const rs_opts* opts,
                void* stream, const char* path, rs_tune_report* report);
int rs_tune_save(const char* path);
int rs_tune_load(const char* path);
int rs_tune_clear(void);
int rs_tune_count(void);

/* Per-box inspection (copies from the device).  level 1..d, box 0..2^level-1.
 * sizes: m (active points), k (skeleton), r (ID rows), nnear (near rows). */
int rs_op_box_sizes(const rs_op* op, int level, int box, int64_t* m, int64_t* k, int64_t* r,
                    int64_t* nnear);
/* which: 0 = active set (m), 1 = near rows (nnear; refused in translation-invariant mode 1,
 * whose near rows belong to the level's template), 2 = skeleton ascending in g (k). */
int rs_op_box_indices(const rs_op* op, int level, int box, int which, int64_t* out);
/* Orders of Sec. 3.1 used by the extra compression (available for every box): which = 0,
 * the skeleton (k entries: index into the skeleton ascending in g) by angle about the box
 * centre, counter-clockwise from the +x1 direction, ties on one ray by distance then g;
 * which = 1, the residual points (m - k entries: index into the residual in ascending
 * active position) along the interface between the box's children, i.e. by (i2, i1) when
 * the level is even and by (i1, i2) when it is odd. */
int rs_op_box_order(const rs_op* op, int level, int box, int which, int64_t* out);
/* The same orders for caller-given points of box (level, box) of a tree (no GPU needed):
 * g: host, cnt grid indices; out: host, cnt entries, out[p] = index into g of the point at
 * position p.  which = 0 cyclic order, 1 interface order. */
int rs_tree_box_order(const rs_tree* tree, int level, int box, int which, const int64_t* g, int64_t cnt,
                      int64_t* out);
/* Compressed form of one block of a box compressed under opts.k_cut (RS_E_INVALID for other
 * boxes).  which: 0 phi^{sk}, 1 phi^{rs}, 2 E (HSS1D), 3 phi^{s<-r}, 4 phi^{r<-s}, 5 T (low
 * rank).  depth: HSS1D tree depth (-1 for a low-rank form); entries: stored scalars.  nodes
 * (optional; size 4 x (2^(depth+1) - 1), or 4 for a low-rank form): per node in level order
 * (levels 1..depth, or the single node of a depth-0 tree or a low-rank form) its position
 * range lo, hi, its active size a and its rank k. */
int rs_op_box_form(const rs_op* op, int level, int box, int which, int* depth, int64_t* entries,
                   int64_t* nodes);
/* which: 0 = T (k x (m-k), rows by skeleton ascending in g, columns by residual in active
 * order), 1 = F^{-1} (m x m, active order), 2 = E (k x k, skeleton order); row-major.
 * RS_E_INVALID for a level whose dense blocks were released after compression (k_cut). */
int rs_op_box_matrix(const rs_op* op, int level, int box, int which, double* out);
/* Root inverse F_root^{-1} (root_m x root_m, active order = skeletons of boxes (1,0) then
 * (1,1)), row-major. */
int rs_op_root_matrix(const rs_op* op, double* out);

/* ---------------------------------------------------------------------------------------
 * Serving: continuous batching of inverse applies over resident FP64 factorizations.  (The
 * paper notes that several right-hand sides vectorise, Sec. 5.1.3; the server extends that
 * to requests of different operators and sizes arriving over time.)
 * A scheduler thread admits requests in arrival order while fewer than max_inflight are in
 * flight and their solve workspace fits the device-memory budget, then advances every
 * in-flight request by one tree level per tick; each stage of a tick is one launch for all
 * requests in that phase, whatever their operator or nrhs.  A finished request frees its
 * memory at once and waiting requests join at the next tick.  Results equal rs_solve's.
 *   ops: RS_FP64 Laplace operators on one device, factored without k_cut; they stay owned by
 *   the caller but cannot be freed (rs_free returns RS_E_INVALID) until rs_server_free.
 *   mem_budget_bytes: device memory reserved for request workspace (allocated once).
 * --------------------------------------------------------------------------------------- */
int rs_server_create(rs_op* const* ops, int n_ops, size_t mem_budget_bytes, int max_inflight, rs_server** out);
/* Queue x = A_op^{-1} f.  f, x: device, N_op x nrhs column-major in the operator's input
 * order; caller-owned and untouched by the caller until the ticket completes.  Returns a
 * ticket; RS_E_NOMEM if the request could never fit the budget. */
int rs_server_submit(rs_server* s, int op_index, const void* f, int64_t nrhs, void* x, uint64_t* ticket);
/* Non-blocking: up to max completed tickets (completion order) into done_tickets. */
int rs_server_poll(rs_server* s, uint64_t* done_tickets, int max, int* n_done);
/* Block until every submitted request completed (RS_E_TIMEOUT after timeout_s seconds). */
int rs_server_drain(rs_server* s, double timeout_s);
/* Counters since creation (any output may be NULL). */
int rs_server_stats(rs_server* s, int64_t* submitted, int64_t* completed, int64_t* rhs_completed, int64_t* ticks,
                    int64_t* peak_inflight);
/* Latencies (ms, submission to observed completion) of completed requests in completion
 * order: up to max values into out_ms, the total count into *n. */
int rs_server_latencies(rs_server* s, double* out_ms, int64_t max, int64_t* n);
/* Finish the queued work, stop the scheduler and release the server. */
void rs_server_free(rs_server* s);

/* ---------------------------------------------------------------------------------------
 * HSS1D form of an explicit matrix (Sec. 3.2: the dense-block HSS compression that the extra
 * compression of rs_factor uses, exposed on its own).  Positions p = 0..n-1 of the ordering
 * order[p] (an index of M) are split into halving runs: node (l, j) covers positions
 * [floor(j n / 2^l), floor((j+1) n / 2^l)) and the tree stops at the first depth whose runs
 * hold at most `leaf` positions.  Each node's active indices (a leaf's positions; above, the
 * skeletons of its two children) get one interpolative decomposition at eps (a column-pivoted
 * QR step is kept while |R_ss| > eps |R_00|) of its block column stacked on its transposed
 * block row against every index outside the node, so that one skeleton serves both, and M is
 * held in the telescoping form of Eq. 2.9: interpolation blocks T per node, sibling blocks
 * between the skeletons of each node's two children, and dense leaf blocks.
 * --------------------------------------------------------------------------------------- */
typedef struct rs_hss rs_hss;
/* M: host or device, n x n column-major, double or (cplx = 1) interleaved complex128.
 * order: host, n entries forming a permutation of 0..n-1, or NULL (identity).  leaf >= 1,
 * eps >= 0.  The form lives on the current device until rs_hss1d_free.  Synchronous. */
int rs_hss1d_build(const void* M, int64_t n, int cplx, const int64_t* order, int leaf, double eps,
                   void* stream, rs_hss** out);
/* y = M x through the form; x, y: n x nrhs column-major, both host or both device, y may not
 * alias x.  Host buffers: returns when y is written; device buffers: when the work is
 * enqueued on `stream`. */
int rs_hss1d_apply(rs_hss* h, const void* x, int64_t nrhs, void* y, void* stream);
/* depth, stored scalars and device bytes of the form (any output may be NULL). */
int rs_hss1d_info(const rs_hss* h, int* depth, int64_t* entries, int64_t* bytes);
/* Node (level 1..depth, j < 2^level; a depth-0 tree has the single node (0, 0)): position
 * range, active size and rank; skel_rows (optional, k entries): the skeleton as indices of M,
 * ascending in active position. */
int rs_hss1d_node(const rs_hss* h, int level, int node, int64_t* lo, int64_t* hi, int64_t* a,
                  int64_t* k, int64_t* skel_rows);
int rs_hss1d_free(rs_hss* h);

#ifdef __cplusplus
}
#endif
#endif
