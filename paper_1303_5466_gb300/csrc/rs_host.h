// rs_host.h -- host-side structures of the library (tree, per-level factor data, operator).
#pragma once
#include <stdint.h>

#include <atomic>
#include <functional>
#include <vector>

#include "rs_internal.h"

struct rs_tree {
    int64_t n = 0;          // points per side
    int leaf = 0;           // leaf side
    int d = 0;              // depth of the leaves
    std::vector<int64_t> g_of_input;   // grid index of input point i
    std::vector<int64_t> input_of_g;   // input index of grid point g
};

namespace rs {

struct BoxInt {
    int64_t bx, by, wx, wy;
};
BoxInt box_int(int64_t n, int l, int64_t j);

// Index sets of level l (see rs_tree_level_sets in rs.h).
int level_sets(int64_t n, int d, int l, const int64_t* child_k, const int64_t* child_skel, double rfac,
               std::vector<int64_t>& m, std::vector<int64_t>& act, std::vector<int64_t>& act_off,
               std::vector<int64_t>& nnear, std::vector<int64_t>& nearv, std::vector<int64_t>& near_off);

// Owned device allocation.
struct DevMem {
    void* p = nullptr;
    size_t bytes = 0, cap = 0;
    DevMem() = default;
    DevMem(const DevMem&) = delete;
    DevMem& operator=(const DevMem&) = delete;
    DevMem(DevMem&& o) noexcept : p(o.p), bytes(o.bytes), cap(o.cap) { o.p = nullptr; o.bytes = o.cap = 0; }
    DevMem& operator=(DevMem&& o) noexcept
    {
        if (this != &o) {
            if (p) cudaFree(p);
            p = o.p; bytes = o.bytes; cap = o.cap;
            o.p = nullptr; o.bytes = o.cap = 0;
        }
        return *this;
    }
    ~DevMem() { if (p) cudaFree(p); }
    // Grow-only; a growing buffer takes 1.25x the request (cap), so a sequence of slowly
    // growing requests (the levels of a factorization) reallocates -- and synchronises -- less
    // often.  `bytes` is the request of the last reallocation.
    cudaError_t alloc(size_t b)
    {
        if (b <= cap && p) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = cap = 0;
        const size_t want = bytes_hint(b);
        cudaError_t e = cudaMalloc(&p, want ? want : 16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            e = cudaMalloc(&p, b ? b : 16);          // without the headroom
            if (e == cudaSuccess) bytes = cap = b;
            return e;
        }
        bytes = b;
        cap = want;
        return e;
    }
    static size_t bytes_hint(size_t b) { return b < (size_t)1 << 20 ? b : b + b / 4; }
    template <class T> T* as() const { return (T*)p; }
};

// ------------------------------------------------------------------ extra compression (Sec. 3)
// One node of an HSS1D form, or the single node of a low-rank form.
struct CNode {
    int lo = 0, hi = 0;          // HSS1D: position range
    int a = 0, k = 0;            // active and skeleton sizes
    std::vector<int> act;        // a indices of the matrix, in active order
    std::vector<int> perm;       // a local indices: skeleton ascending, then residual ascending
    int64_t t_off = 0;           // T (k x (a-k), column-major, ld k) in the compressed store
};

// Compressed form of one block, built from the block's explicit dense form.
//   HSS1D (Sec. 3.2, the telescoping form of Eq. 2.9 on a 1D order): nodes lev[l][j] for
//     l = 1..depth (depth 0: a single dense node at lev[0][0]); sibling blocks b12/b21 of the
//     internal nodes (heap index 2^l - 1 + j, levels 0..depth-1) and permuted leaf blocks d_off.
//   Low rank: X ~ X(:, sk) [I T] Pi^T from a column ID of X: lev[0][0] (a = cols), c_off.
struct CForm {
    bool hss = true;
    int rows = 0, cols = 0, depth = 0;
    std::vector<int> order;                  // HSS1D: position -> index of the matrix
    std::vector<std::vector<CNode>> lev;
    std::vector<int64_t> b12, b21, d_off;
    int64_t c_off = 0;
    int64_t entries = 0;                     // stored scalars
    const void* M = nullptr;                 // dense source (during compression only)
    int64_t ld = 0;
};

// One launch of a compressed apply: a row copy between the apply's buffers (0 input,
// 1 output, 2 scratch), or a batched matvec on the scratch with the compressed store.
struct ProgStage {
    int kind = 0;                // 0 copy, 1 matvec
    int src = 0, dst = 0, add = 0;
    int64_t count = 0;           // copy: rows; matvec: blocks
    int np = 0;                  // matvec: problems
    int rb = 64;                 // matvec: output rows per block (16, 32 or 64, by problem size)
    DevMem a, b;                 // copy: source and destination rows; matvec: problems, first blocks
    double work = 0.0;           // matvec: sum of rows x cols
};
struct Program {
    std::vector<ProgStage> st;
    int64_t z_rows = 0;          // scratch rows the program uses
    double work = 0.0;           // sum of rows x cols of its matvecs
};

// Everything stored for one tree level (level 0 = root, factored without an ID).
struct Level {
    int l = 0;
    int nb = 0;
    // host copies
    std::vector<int64_t> m, k, r, nn;
    std::vector<int64_t> act, act_off, nearv, near_off;
    std::vector<int32_t> perm;        // per box: sorted skeleton locals, then residual locals
    std::vector<int64_t> skel;        // per box: skeleton grid indices, ascending (k entries)
    std::vector<int64_t> k_off;       // prefix sums of k
    std::vector<int64_t> t_off, phi_off, e_off, w_off;
    int max_m = 0, max_k = 0, max_r = 0;
    // device: bookkeeping
    DevMem d_act, d_act_off, d_perm, d_k, d_m;
    DevMem d_t_off, d_phi_off, d_e_off, d_ipiv_off, d_cb_off, d_k_off;
    // device: factors
    DevMem d_T, d_Phi, d_E;
    // device: solve index maps and descriptors
    DevMem d_idx_up;      // rows of the child-level vector buffer for each active position (l < d)
    DevMem d_idx_leaf;    // input index of each permuted leaf position (l == d)
    DevMem d_idx_sk;      // row act_off + a for each skeleton position a (k_off order)
    DevMem d_mv_phi, d_mv_phi_blk, d_mv_T, d_mv_T_blk, d_mv_E, d_mv_E_blk, d_mv_Tt, d_mv_Tt_blk;
    int n_mv_phi = 0, n_mv_T = 0, n_mv_E = 0, n_mv_Tt = 0;
    int rb_phi = 64, rb_T = 64, rb_E = 64, rb_Tt = 64;     // output entries per block
    std::vector<int64_t> h_blk_phi, h_blk_T, h_blk_E, h_blk_Tt;  // first block of each problem, then the total
    int64_t b_mv_phi = 0, b_mv_T = 0, b_mv_E = 0, b_mv_Tt = 0;
    int64_t sum_m = 0, sum_k = 0;
    double mvw_phi = 0, mvw_T = 0, mvw_E = 0, mvw_Tt = 0;   // sum of rows * cols per descriptor set
    // forward apply (rs_fwd_apply), built on first use: the mutual blocks of each box's two
    // children (points: the child level's skeletons, in k_off order) and, at the leaf level,
    // the diagonal blocks (points: the leaf points in the permuted order)
    DevMem d_fw_pts, d_fw_sib, d_fw_sib_blk, d_fw_leaf, d_fw_leaf_blk, d_fw_leaf_pts;
    int n_fw_sib = 0, n_fw_leaf = 0;
    int64_t b_fw_sib = 0, b_fw_leaf = 0;
    // translation-invariant modes: class of every box and the box factored for each class
    std::vector<int32_t> ti_cls;
    std::vector<int> ti_rep;
    // extra compression (Sec. 3): boxes with k > k_cut
    std::vector<char> cmp;                 // per box
    std::vector<int> cbox;                 // compressed boxes
    std::vector<CForm> forms;              // 6 per compressed box: phi_ss, phi_rr, E (HSS1D),
                                           // phi_sr, phi_rs, T (low rank)
    Program p_phi, p_T, p_E, p_Tt;         // compressed parts of the four solve applies
    bool dense_freed = false;
};

// Workspace layout of one inverse apply with nrhs columns (counts in storage elements).
struct SolveLayout {
    std::vector<int64_t> woff, goff;   // per-level row offsets of w and of g / phi
    int64_t max_m = 0, max_k = 0;
    int64_t n_w = 0, n_g = 0, n_u = 0, n_t = 0, n_z = 0;
    int64_t total() const { return n_w + 2 * n_g + 2 * n_u + n_t + n_z; }
};

// Workspace pointers of one inverse apply, in the factor's storage type: w (n_w), g and
// phi (n_g each), u and out (n_u each), t (n_t), z (n_z: scratch of the compressed applies).
struct SolveWork {
    void *w, *g, *phi, *u, *out, *t, *z;
};

struct ProfRec {
    int cls, level;
    cudaEvent_t e0, e1;
    double work, bytes;
};

// Autotuner table (rs_tune.cpp).  Keys: tune_key(kernel, scalar bytes, boxes, largest m, r).
std::string tune_key(const char* what, int esz, int nb, int64_t m, int64_t r);
double tune_get(const std::string& key, double dflt);
void tune_set(const std::string& key, double v);
int tune_count();
// Settings forced on every level by rs_autotune while it times one candidate (negative: none).
struct TuneTrial {
    double cpqr_gscale = -1.0;
    int cpqr_deep = -1;
    double sweep_gscale = -1.0;
    double cpqr_batch = -1.0;      // L2 batch budget of the CPQR launches, in units of 96 MB (0: none)
    int sweep_nb = -1;             // panel width of the sweep (8 or 16)
};
extern thread_local TuneTrial g_trial;

}  // namespace rs

struct rs_op;
namespace rs {
SolveLayout solve_layout(const rs_op* op, int64_t nrhs);
int solve_run(rs_op* op, const SolveLayout& Ls, const SolveWork& ws, const double* fd, double* xd, int64_t nrhs,
              cudaStream_t st, bool profile);
bool is_device_ptr(const void* p);
// True when p is device memory of a GPU other than the current one (kernels of the current
// device cannot read it without peer access, so the entry points refuse it).
bool on_other_device(const void* p);
int choose_group(int nb, int max_cols, const std::function<int(int)>& capacity);

// Extra compression (rs_hss1d.cpp).  Orders of Sec. 3.1 for box j of level l of an n x n grid:
// skeleton points (grid indices g) cyclically around the box, residual points along the
// interface between its children; both return the index of the point at each position.
std::vector<int> cyclic_order(int64_t n, int l, int64_t j, const int64_t* g, int cnt);
std::vector<int> interface_order(int64_t n, int l, const int64_t* g, int cnt);
// Device status and barrier words of the ID kernels, and their wait limit.
struct IdCtx {
    int* status;
    DevMem* bar;
    long long spin;
};
// Compress every form of `forms` (sources M/ld set; HSS1D forms with their order) at eps with
// HSS1D leaves of at most `leaf`, into a new store of T elements.
template <class T>
int compress_forms(const IdCtx& ctx, cudaStream_t st, std::vector<CForm*>& forms, double eps, int leaf, DevMem& store,
                   int64_t& store_n);
// Program builder input: form f applied (trans: X^T for a low-rank form) with input index i at
// row in_rows[i] of the input buffer and output index i to row out_rows[i] of the output buffer
// (add: accumulate).
struct ProgItem {
    const CForm* f;
    bool trans;
    std::vector<int64_t> in_rows, out_rows;
    bool add;
};
int build_program(std::vector<ProgItem>& items, cudaStream_t st, Program& prog);
template <class T>
int run_program(cudaStream_t st, const Program& prog, const T* store, const T* in, T* out, T* z, int nrhs);
}  // namespace rs
struct rs_op;
namespace rs {
// Compress the boxes of every level with k > opts.k_cut (after the dense factorization) and
// build the levels' apply programs; releases the dense blocks of fully compressed levels.
template <class T>
int compress_levels(rs_op* op, cudaStream_t st);
int apply_once(rs_op* op, const double* fd, double* xd, int64_t nrhs, cudaStream_t st);
int refine_solve(rs_op* op, const double* fd, double* xd, int64_t nrhs, cudaStream_t st);
int residual_apply(rs_op* op, const double* x, const double* f, int64_t nrhs, double* r, double* rel,
                   cudaStream_t st);
int kernel_tables(rs_op* op, cudaStream_t st);
void helmholtz_cell_integral(double h, double kappa, double* re, double* im);
}  // namespace rs

struct rs_op {
    int device = 0;
    int esz = 8;                      // bytes per stored factor entry (8 FP64, 4 mixed FP32)
    int64_t n = 0, N = 0;
    int d = 0;
    rs_kernel_kind kind = RS_LAPLACE;
    double kappa = 0.0;
    double eps = 0.0;
    rs_opts opts{};
    rs::KernelK K{};
    std::vector<int64_t> input_of_g;
    std::vector<rs::Level> lev;       // lev[0] = root, lev[l] for l = 1..d
    // translation-invariant mode (opts.translation_invariant): the one-box template of each
    // level (its ID on an extended lattice, then its F, F^{-1} and E), whose factors every box
    // of lev[l] shares
    std::vector<rs::Level> ti_lev;
    double ti_s0 = 1.0;               // the constant Helmholtz scaling s = kappa sqrt(b) there
    bool fw_built = false;            // forward-apply block lists uploaded
    bool defer_spd = false;           // sweeps of the inverse phase launch without a host check
                                      // of their status (checked once after the root)
    rs::DevMem d_a, d_ucirc, d_status, d_bar, d_ipiv, d_pivrow, d_pb;
    // factor-time scratch reused across levels, released with the op
    rs::DevMem t_ipoff, t_pboff, t_cta, t_W, t_p1, t_p2, t_k32, t_q1, t_q2, t_ck, t_ce;
    rs::DevMem t_oz1, t_oz2, t_ozo1, t_ozo2, t_ozx, t_ozd;   // digit-product GEMM: descriptors, offsets, exponents, digits
    rs::DevMem t_blq, t_blQ, t_blX, t_blD, t_blmp, t_blgx, t_blgu, t_blex, t_bleu;   // blocked sweep
    rs::DevMem t_idrg, t_idR, t_idg, t_ide;            // blocked id_T: offsets, [R11 | R12], GEMM lists
    rs::DevMem d_zero;                // one int64 zero: the first block of a one-problem launch
    // solve workspace (grown on demand)
    rs::DevMem s_u, s_w, s_g, s_phi, s_t, s_z, s_in, s_out, s_out2;
    int64_t s_nrhs = 0;
    // FP64 direct-sum residual (built on first use): offset table, diagonal, permutation,
    // and refinement workspace
    rs::DevMem d_ktab, d_diag, d_rs, d_ing, r_xg, r_yg, r_res, r_dx, r_x, r_norm;
    // FP32 (complex64) copies of the table and diagonal, and grid scratch, for the products of
    // the refinement's corrections
    rs::DevMem d_ktab_lo, d_diag_lo, r_xg_lo;
    // Helmholtz symmetric scaling s = kappa sqrt(b): grid order, input order; scaled RHS
    rs::DevMem d_s, d_s_in, s_fs;
    // compressed store of the Sec. 3 forms (opts.k_cut)
    rs::DevMem d_cstore;
    int64_t cstore_n = 0;
    rs_stats stats{};
    std::atomic<int> inflight{0};   // references held by servers and their requests
    // CUDA graphs of the inverse apply (opts.solve_graph), one per nrhs, captured on a private
    // stream with the staging buffers g_in / g_out; ws_gen counts workspace reallocations, and
    // a graph captured under an older workspace is dropped
    struct SolveGraph {
        int64_t nrhs;
        uint64_t gen;
        cudaGraphExec_t exec;
        int64_t launches;
    };
    std::vector<SolveGraph> graphs;
    cudaStream_t cap_stream = nullptr;
    uint64_t ws_gen = 0;
    const void* ws_ptrs[9] = {};
    rs::DevMem g_in, g_out;
    // profiling (opts.profile): pending event pairs and per-class sums
    std::vector<rs::ProfRec> pending;
    std::vector<cudaEvent_t> ev_pool, ev_all;
    double prof_ms[RS_PROF_COUNT] = {}, prof_work[RS_PROF_COUNT] = {}, prof_bytes[RS_PROF_COUNT] = {};
    std::vector<double> prof_level_ms[RS_PROF_COUNT];     // by tree level (factor classes)
    int64_t prof_n[RS_PROF_COUNT] = {};
    ~rs_op()
    {
        for (cudaEvent_t e : ev_all) cudaEventDestroy(e);
        for (SolveGraph& g : graphs) cudaGraphExecDestroy(g.exec);
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
};
