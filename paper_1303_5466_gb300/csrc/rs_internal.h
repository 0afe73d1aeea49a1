// rs_internal.h -- shared declarations of the library's host code and CUDA kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rs.h"
#include "k_scalar.cuh"

namespace rs {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define RS_CUDA(...)                                                 \
    do {                                                             \
        cudaError_t e__ = (__VA_ARGS__);                             \
        if (e__ != cudaSuccess) return cuda_fail(e__, #__VA_ARGS__); \
    } while (0)

// Kernel launches made by the library (rs_launch_count).
void count_launches(int n);

// Device status word bits written by kernels (never a trap): the host maps them to RS_E_*.
enum : int { DEV_OK = 0, DEV_SINGULAR = 1, DEV_TIMEOUT = 2, DEV_BADSIZE = 4, DEV_NOT_SPD = 8 };

// Pivot key of the column-pivoted QR: the squared column norm with its 40 low mantissa bits
// cleared (relative step 2^-12), and the low bits holding (2^40-1 - column index), so that the
// largest key picks the largest norm, and among norms equal in their leading bits the lowest
// column index.  The coarse step keeps CPU and GPU rounding differences from changing a pivot.
constexpr int KEY_BITS = 40;
constexpr unsigned long long KEY_MASK = (1ull << KEY_BITS) - 1ull;

// ------------------------------------------------------------------ grouped GEMM descriptor
// C = alpha * op(A) * op(B) + beta * C0 for one problem, all column-major (C0 may be C).
struct GemmProb {
    int M, N, K;
    int ta, tb;            // 1: use the transpose
    int lda, ldb, ldc, ldc0;
    int64_t a_off, b_off, c_off, c0_off;
    double alpha, beta;
    int tiles_m, tiles_n;
    int64_t tile0;         // first tile index of this problem in the launch
    int lower;             // 1: only the tiles on and below the diagonal (M = N; tiles_m (tiles_m + 1) / 2)
};

// FP64 grouped GEMM from exact products of 7-bit digit slices on the bf16 tensor cores
// (k_gemm_oz.cu): same descriptors and semantics as launch_gemm, T = double.  gemm_oz_plan
// re-tiles the descriptors (64 x 32 tiles; `lower` problems keep every tile that touches the lower
// triangle) and fills eoff (2 (np + 1) entries: each problem's first exponent line, then its first
// digit); the launch needs pl.lines ints (ex) and pl.digits bf16 values (digits) of device
// scratch, and eoff on the device.
struct OzPlan {
    int64_t tiles, lines, digits;
};
OzPlan gemm_oz_plan(std::vector<GemmProb>& probs, std::vector<int64_t>& eoff);
cudaError_t launch_gemm_oz(cudaStream_t st, const GemmProb* probs, int np, const OzPlan& pl, const int64_t* eoff,
                           int* ex, void* digits, const double* A, const double* B, double* C, const double* C0);

// Blocked symmetric sweep (k_sweep_bl.cu), FP64: sweep_bl_plan lays out the panel buffers (qoff:
// 64 m_b doubles per matrix, row-major; returns the total) and the two digit-GEMM lists of every step (gx:
// X = Q D^{-1}; gu: S <- S - X Q^T), off = the matrices' offsets; per step one panel launch,
// the two GEMMs, one write launch; launch_sweep_finish then negates and mirrors.
size_t sweep_bl_plan(int nb, const std::vector<int64_t>& sizes, int max_m, std::vector<int64_t>& qoff,
                     std::vector<std::vector<GemmProb>>& gx, std::vector<std::vector<GemmProb>>& gu,
                     const std::vector<int64_t>& off);
cudaError_t launch_sweep_bl_panel(cudaStream_t st, int nb, int k0, int max_m, const int32_t* m, const int64_t* off,
                                  const double* A, const int64_t* qoff, double* Q, double* D, double* maxp, int* status);
cudaError_t launch_sweep_bl_write(cudaStream_t st, int nb, int k0, int max_m, const int32_t* m, const int64_t* off,
                                  double* A, const int64_t* qoff, const double* X, const double* D);
template <class T>
cudaError_t launch_sweep_finish(cudaStream_t st, int nb, const int32_t* m, const int64_t* off, T* A, int max_m);

// T = R11^{-1} R12 by blocks of 64 rows with the updates on the digit-slice GEMM (k_idt_bl.cu,
// FP64): idt_bl_plan lays out the gathered [R11 | R12] blocks (rg_off, k m doubles per box,
// returns the total) and the GEMM list of every step; per step one solve launch and the GEMM.
size_t idt_bl_plan(int nb, const std::vector<int64_t>& m, const std::vector<int64_t>& k, int max_k,
                   std::vector<int64_t>& rg_off, std::vector<std::vector<GemmProb>>& gs);
cudaError_t launch_idt_gather(cudaStream_t st, int nb, int64_t max_km, const int64_t* act_off, const int32_t* kk,
                              const int32_t* nnear, int P, const int64_t* y_off, const double* Y, const int32_t* piv,
                              const double* diag, const int32_t* rscol, const int64_t* rg_off, double* Rg);
cudaError_t launch_idt_solve(cudaStream_t st, int nb, int q, int max_res, const int64_t* act_off, const int32_t* kk,
                             const int64_t* rg_off, double* Rg);
cudaError_t launch_idt_scatter(cudaStream_t st, int nb, int64_t max_kres, const int64_t* act_off, const int32_t* kk,
                               const int32_t* skpos, const int64_t* rg_off, const double* Rg, const int64_t* t_off,
                               double* Tout);

// Batched matrix-vector(s) descriptor: y = alpha * op(A) x + beta * y, A column-major
// (rows x cols, ld), x and y point-major (entry p of RHS c at p * nrhs + c); x_off and y_off
// count points (rows), so one descriptor serves every nrhs.
struct MatvecProb {
    int rows, cols, ld, trans;
    int64_t a_off, x_off, y_off;
    double alpha, beta;
};

// One block product of the forward apply: y(y_off + i) += sum_j A(pts[r_off + i], pts[c_off + j])
// x(x_off + j), i < rows, j < cols (vectors row-major with nrhs columns).
struct KbProb {
    int rows, cols;
    int64_t r_off, c_off, x_off, y_off;
};

// ------------------------------------------------------------------ launchers (kernels.cu)
// All launchers enqueue on `st`, return cudaError_t of the launch.

// Kernel constants.  Laplace: off-diagonal c0 log(|x - y|^2) (c0 = -h^2/(4 pi)), diagonal
// a_g + self.  Helmholtz, in the symmetric form of Eq. (5.6): off-diagonal
// s_g (i/4) H0(kappa r) h^2 s_g', diagonal a_g + s_g^2 (hs_re + i hs_im), s = kappa sqrt(b)
// (device array, grid order); the proxy rows are (i/4) H0(kappa |z - x|) h^2 s_g.
struct KernelK {
    double h, c0, self;
    int n;
    int kind;
    double kappa;
    double hs_re, hs_im;
    const double* s;        // Helmholtz s_g per grid point, or NULL: the constant s0
    double s0;
    // the off-diagonal entries on the grid depend only on the offset (d1, d2): when set, a
    // (2n-1)^2 table of K(d1 h, d2 h) in the factor's storage type (Helmholtz: without the
    // s_g s_g' scaling), read at (d1 + n - 1) + (2n - 1)(d2 + n - 1)
    const void* tab;
};

// All launchers below are instantiated for T = double (FP64 path), float (FP32 storage of the
// mixed-precision factor), cplx<double> (complex128) and cplx<float> (complex64).

// Y for every box of a level: rows = near points then P proxy points, columns = active
// points, column-major r x m at y_off[b].
template <class T>
cudaError_t launch_assemble_Y(cudaStream_t st, int nb, const int32_t* act, const int64_t* act_off,
                              const int32_t* near, const int64_t* near_off, const double* geo,
                              const double* ucirc, int P, const int64_t* y_off, T* Y, KernelK K,
                              int max_entries);

// Column-pivoted QR (Eq. 2.1) of every box's Y, G CTAs per box (cooperative when G > 1).
// Column norms and pivot choices are FP64 for every T; nrm and ref are FP64 work arrays of
// act_off[nb] entries each (the squared column norms, shared by the group's CTAs).  Outputs: kout[b],
// piv[act_off[b] + s] = physical column of pivot s (s < k), diag[act_off[b] + s] = R_ss.
// Y is overwritten by the factorisation (rows < k hold R).
// Group sizes: G CTAs for every box, or (cta_off != NULL, device, nb + 1 entries) box b takes
// CTAs cta_off[b] .. cta_off[b+1], ctas = cta_off[nb] in all.
// deep (the variant): 0 = four rows per lane in flight; 1 = eight (more registers; for
// launches with few CTAs per SM, where each warp must hide more memory latency by itself);
// 2 = the look-ahead form (k_cpqr_la.cu: one read and one write of each open column per step
// instead of two reads and a write), which needs wv, a work array of act_off[nb] entries;
// 3 = variant 0 with the open-column lists in global memory (gwork), which variants 0 and 1
// also take when shared memory cannot hold them: gwork then needs cpqr_gwork_ints() ints.
template <class T>
cudaError_t launch_cpqr(cudaStream_t st, int nb, int G, const int32_t* cta_off, int ctas, int deep,
                        const int64_t* act_off, const int32_t* nnear, int P,
                        const int64_t* y_off, T* Y, double eps, int32_t* kout, int32_t* piv, T* diag,
                        unsigned int* bar, unsigned long long* keys, int* status, long long spin_limit, int max_r,
                        int max_m, double* nrm, double* ref, T* wv = nullptr, int* gwork = nullptr);
// ints of global scratch a launch of `ctas` CTAs needs for its open-column lists (0: none)
template <class T>
size_t cpqr_gwork_ints(int max_r, int max_m, int deep, int ctas);
// Largest grid of the cpqr kernel (of the given variant) that can be co-resident for these sizes.
template <class T>
int cpqr_max_ctas(int max_r, int max_m, int G, int deep = 0);
template <class T>
cudaError_t launch_cpqr_la(cudaStream_t st, int nb, int G, const int32_t* cta_off, int ctas, const int64_t* act_off,
                           const int32_t* nnear, int P, const int64_t* y_off, T* Y, double eps, int32_t* kout,
                           int32_t* piv, T* diag, unsigned int* bar, unsigned long long* keys, int* status,
                           long long spin_limit, int max_r, int max_m, double* nrm, double* ref, T* wv);
template <class T>
int cpqr_la_max_ctas(int max_r, int max_m);
// Variant 4 (k_cpqr_cl.cu): one thread-block cluster of C CTAs per box, the box's Y held in the
// clusters' shared memory for the whole factorization (read once, R written back once).
// cpqr_cl_cluster: the cluster size for boxes up to max_r x max_m, 0 when they do not fit.
// Same outputs as launch_cpqr (kout, piv, diag, R in rows < k of Y); no barrier words, keys or
// norm arrays in global memory.
template <class T>
int cpqr_cl_cluster(int max_r, int max_m);
template <class T>
cudaError_t launch_cpqr_cl(cudaStream_t st, int nb, int C, const int64_t* act_off, const int32_t* nnear, int P,
                           const int64_t* y_off, T* Y, double eps, int32_t* kout, int32_t* piv, T* diag, int* status,
                           int max_r, int max_m);

// Variants 7 and 8 (k_cpqr_bl.cu): the trailing updates deferred over panels of nbp = 16 or 8
// steps; real scalars only.  Same arguments and outputs as launch_cpqr, plus sum_m (the level's
// act_off[nb] of all boxes, which F is indexed by) and scratch: cpqr_bl_bytes() bytes of
// device memory (V, F and the group partials).
template <class T>
bool cpqr_bl_fits(int max_r, int max_m);
template <class T>
int cpqr_bl_max_ctas(int max_r, int max_m, int nbp);
template <class T>
size_t cpqr_bl_bytes(int nb, int max_r, int64_t sum_m, int ctas, int nbp);
template <class T>
cudaError_t launch_cpqr_bl(cudaStream_t st, int nb, int G, const int32_t* cta_off, int ctas, int nbp,
                           const int64_t* act_off, const int32_t* nnear, int P, const int64_t* y_off, T* Y,
                           double eps, int32_t* kout, int32_t* piv, T* diag, unsigned int* bar,
                           unsigned long long* keys, int* status, long long spin_limit, int max_r, int max_m,
                           int64_t sum_m, double* nrm, double* ref, void* scratch);

// T = R11^{-1} R12 for every box, written column-major (k x (m-k)) at t_off[b], rows by
// sorted skeleton position (skpos[pivot position]) and columns by residual rank.
template <class T>
cudaError_t launch_id_T(cudaStream_t st, int nb, const int64_t* act_off, const int32_t* kk, const int32_t* nnear,
                        int P, const int64_t* y_off, const T* Y, const int32_t* piv, const T* diag,
                        const int32_t* skpos, const int32_t* rscol, const int64_t* t_off, T* Tout, int max_cols,
                        int max_k);

// F' = Pi^T F Pi for every box (sk-first order given by perm), column-major m x m at
// phi_off[b].  Leaf: kernel entries with diagonal a_g + self.  Non-leaf: E of the
// children on the diagonal blocks, kernel entries elsewhere.
template <class T>
cudaError_t launch_assemble_F(cudaStream_t st, int nb, bool leaf, const int32_t* act, const int64_t* act_off,
                              const int32_t* perm, const double* a, const int64_t* phi_off, T* Phi,
                              const int32_t* child_k, const int64_t* child_e_off, const T* childE, KernelK K,
                              int max_m);

// In-place blocked Gauss-Jordan inverse with partial pivoting of nb column-major matrices
// (sizes m[b], offsets off[b]), G CTAs per matrix (cooperative when G > 1).  ipiv: one int
// per row (ipiv_off[b]); pivbuf: 2 * gj_panel_width() ints per matrix; bar: one counter per
// matrix, zeroed before the launch.
template <class T>
cudaError_t launch_gj_inverse(cudaStream_t st, int nb, int G, const int32_t* m, const int64_t* off, T* A,
                              int32_t* ipiv, const int64_t* ipiv_off, int* pivbuf, unsigned int* bar, int* status,
                              long long spin_limit, int max_m);
// Deal `total` CTAs to nb groups in proportion to their work (at least one each, at most
// cap[b]); returns the prefix (nb + 1 entries).
std::vector<int32_t> proportional_groups(int total, const std::vector<double>& work, const std::vector<int>& cap);
// Co-resident CTAs of the GJ kernel for a launch of nb matrices of size <= max_m.
template <class T>
int gj_max_ctas(int max_m, int nb);
int gj_panel_width();

// In-place inverse of nb symmetric positive definite matrices (real T) by the symmetric sweep
// (k_sweep.cu), G CTAs per matrix (cooperative when G > 1), panels of nbw columns (8 =
// sweep_panel_width(), or 16): sizes m[b], offsets off[b]; Pb: 2 * nbw * m[b] elements per
// matrix at pb_off[b] (16-byte aligned); bar: one
// counter per matrix, zeroed before the launch.  Reads the lower triangle, writes the full
// inverse.  A matrix that is not SPD to working accuracy sets DEV_NOT_SPD and is left partly
// swept.
// Group sizes as for launch_cpqr: G per matrix, or the device prefix cta_off (ctas in all).
template <class T>
cudaError_t launch_sweep_inverse(cudaStream_t st, int nb, int G, const int32_t* cta_off, int ctas, const int32_t* m,
                                 const int64_t* off, T* A, T* Pb, const int64_t* pb_off, unsigned int* bar,
                                 int* status, long long spin_limit, int max_m, int nbw);
template <class T>
int sweep_max_ctas(int nbw);
int sweep_panel_width();

// Grouped GEMM over `np` problems (device descriptors), total tiles `tiles`.
template <class T>
cudaError_t launch_gemm(cudaStream_t st, const GemmProb* probs, int np, int64_t tiles, const T* A, const T* B, T* C,
                        const T* C0);

// Batched matvec(s) over `np` problems, blocks = sum over problems of ceil(out_rows / rb) with
// rb = 16, 32 or 64 output entries per block (blk0[p]: first block of problem p).
template <class T>
cudaError_t launch_matvec(cudaStream_t st, const MatvecProb* probs, const int64_t* blk0, int np, int64_t blocks,
                          const T* A, const T* x, T* y, int nrhs, int rb);
// Block size (rb) of a descriptor set whose problems give blocks64 blocks of 64 outputs.
int matvec_rows_per_block(int64_t blocks64);

// Point-major row gathers/scatters of the solve: out[p * nrhs + c] = in[idx[p] * nrhs + c]
// (gather) and the reverse (scatter), for p < count.
template <class T>
cudaError_t launch_gather_rows(cudaStream_t st, int64_t count, const int64_t* idx, const T* in, T* out, int nrhs);
template <class T>
cudaError_t launch_scatter_rows(cudaStream_t st, int64_t count, const int64_t* idx, const T* in, T* out, int nrhs);
// Column-major N x nrhs FP64 (input order) <-> point-major rows of type T at idx.
template <class Ti, class To>
cudaError_t launch_gather_cm(cudaStream_t st, int64_t count, const int64_t* idx, const Ti* in, int64_t N, To* out,
                             int nrhs);
template <class Ti, class To>
cudaError_t launch_scatter_cm(cudaStream_t st, int64_t count, const int64_t* idx, const Ti* in, int64_t N, To* out,
                              int nrhs);
// y[i] = a * x[i] + b * y[i]
template <class T>
cudaError_t launch_axpby(cudaStream_t st, int64_t n, T a, const T* x, T b, T* y);
// y[c N + i] = s[i]^pw x[c N + i], pw = +1 or -1 (instantiated for cplx<double>)
// Block products of the forward apply (k_forward.cu): problem p owns blocks blk0[p] ..
// of kblock_rows_per_block() rows each, nblk in all; entries from K (diagonal a_g + self where
// a row and a column are the same point).
template <class T>
cudaError_t launch_kblock_mv(cudaStream_t st, const KbProb* probs, const int64_t* blk0, int np, int64_t nblk,
                             const int32_t* pts, const T* x, T* y, int nrhs, const KernelK& K, const double* a);
int kblock_rows_per_block();

// One CTA waiting at a group barrier that can never complete (k_wait.cu): the bounded wait
// must end after `limit` polls with DEV_TIMEOUT in *status.  ctr: one zeroed counter.
cudaError_t launch_wait_check(cudaStream_t st, unsigned int* ctr, int* status, long long limit);

// Vector kernels of BiCGstab (k_krylov.cu), T = double or cplx<double>: *out = sum conj(a_i) b_i
// (part: dot_partials() scratch entries; fixed summation order), y = c0 x0 + c1 x1 + c2 x2.
template <class T>
cudaError_t launch_dot(cudaStream_t st, int64_t n, const T* a, const T* b, T* part, T* out);
int dot_partials();
template <class T>
cudaError_t launch_lincomb(cudaStream_t st, int64_t n, T c0, const T* x0, T c1, const T* x1, T c2, const T* x2,
                           T* y);

template <class T>
cudaError_t launch_scale_cm(cudaStream_t st, int64_t N, int nrhs, const double* sc, int pw, const T* x, T* y);

// Serving job lists (k_serve.cu).  MvJob: one request's descriptor set of one stage
// (blocks blk_start .. blk_start + nblk of the launch).  CopyJob: a gather, scatter or axpby
// over elements e_start .. e_start + count * nrhs (axpby: count elements, nrhs 1).
struct MvJob {
    const MatvecProb* probs;
    const int64_t* blk0;
    int np, nrhs, rb;
    int64_t blk_start;
    const double* A;
    const double* x;
    double* y;
};
enum { COPY_GATHER_ROWS = 0, COPY_SCATTER_ROWS = 1, COPY_GATHER_CM = 2, COPY_SCATTER_CM = 3, COPY_AXPBY = 4 };
struct CopyJob {
    int64_t e_start;
    int mode, nrhs;
    int64_t count, N;
    const int64_t* idx;
    const double* in;
    double* out;
    double a, b;
};
cudaError_t launch_mv_jobs(cudaStream_t st, const MvJob* jobs, int nj, int64_t blocks);
cudaError_t launch_copy_jobs(cudaStream_t st, const CopyJob* jobs, int nj, int64_t total);

// Extra compression of Sec. 3 (k_hss1d.cu).
// ZProb: ID input of one node, column-major r x a at y_off.  mode 0 (HSS1D node):
// r = 2 nout, rows i < nout are M(out[i], act[:]) and rows nout + i are M(act[:], out[i]);
// mode 1 (low-rank block): r = nout, rows are M(i, act[:]).  M column-major with ld; act and
// out are int32 lists at act_off / out_off of the launch's list array.
struct ZProb {
    const void* M;
    int64_t ld;
    int a, nout, mode;
    int64_t act_off, out_off, y_off;
};
// SubProb: dst[dst_off + i + j rows] = M(row[i], col[j]) (row_off < 0: row[i] = i).
struct SubProb {
    const void* M;
    int64_t ld;
    int rows, cols;
    int64_t row_off, col_off, dst_off;
};
template <class T>
cudaError_t launch_zgather(cudaStream_t st, const ZProb* probs, int np, const int32_t* lists, T* Y, int64_t max_el);
template <class T>
cudaError_t launch_subgather(cudaStream_t st, const SubProb* probs, int np, const int32_t* lists, T* dst,
                             int64_t max_el);
// out[dst[p] * nrhs + c] = in[src[p] * nrhs + c] (add != 0: +=), p < count.
template <class T>
cudaError_t launch_copy_rows(cudaStream_t st, int64_t count, const int64_t* src, const int64_t* dst, const T* in, T* out,
                             int nrhs, int add);

// FP64 direct-sum residual (k_residual.cu): Kt is the (2n-1)^2 offset table of the Laplace
// kernel; r = f - A x with x, f, r N x nrhs column-major in input order (ing[g] = input index
// of grid point g), xg, yg grid-order scratch, norms[2c] = |r_c|^2, norms[2c+1] = |f_c|^2.
// Helmholtz: Kt holds (i/4) H0(kappa |d| h) h^2 (complex), dg = a + kappa^2 b (i/4) int_cell H0 and
// the off-diagonal sum is scaled per row by rs = kappa^2 b (Laplace: rs = NULL).
cudaError_t launch_laplace_table(cudaStream_t st, int n, double h, double c0, double* Kt);
cudaError_t launch_helmholtz_table(cudaStream_t st, int n, double h, double kappa, cplx<double>* Kt);
template <class S>
cudaError_t launch_residual(cudaStream_t st, int n, int nrhs, const S* Kt, const S* dg, const double* rs,
                            const int64_t* ing, const S* x, const S* f, S* xg, S* yg, S* r, double* norms);
// out = (L) in, n entries (L = float or cplx<float> copies of the table and diagonal)
template <class S, class L>
cudaError_t launch_narrow(cudaStream_t st, int64_t n, const S* in, L* out);
// r <- r - A dx with the products of A dx in L, each 256-term tile sum added in S (table Kt
// and diagonal dg in L; dx, r in S, N x nrhs column-major in input order; xg (L) and yg (S)
// grid-order scratch); norms[2c] = norms[2c + 1] = |r_c|^2.
template <class S, class L>
cudaError_t launch_residual_update(cudaStream_t st, int n, int nrhs, const L* Kt, const L* dg, const double* rs,
                                   const int64_t* ing, const S* dx, S* r, L* xg, S* yg, double* norms);

}  // namespace rs
