// rs_server.cpp -- continuous-batching server over resident factorizations.
//
// A scheduler thread owns one CUDA stream.  Each tick it
//   1. admits waiting requests in arrival order while the in-flight cap and the device-memory
//      budget allow (each request's solve workspace is carved from one arena);
//   2. advances every in-flight request by one step of the inverse apply (Algorithm 6): one
//      level of the upward pass, the root, or one level of the downward pass;
//   3. issues each stage of that step as a single launch whose job list holds every request
//      in that phase, across operators, levels and RHS counts;
//   4. waits for the previous tick (not this one) and retires the requests it finished
//      (freeing their memory at once).
// Two ticks are in flight at a time: the host builds and enqueues tick t+1 while the GPU runs
// tick t (the steps of a request are known in advance, and stream order keeps each request's
// stages in sequence), so the GPU does not idle while the host prepares job lists.  Job lists
// are staged through two buffers, one per tick in flight.  Requests that arrive while others
// run join at the next tick.  The per-request kernels do the same arithmetic as rs_solve, so
// results do not depend on the batch.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "rs_host.h"

namespace rs {
namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over [0, size) with 256-byte granules.
struct Arena {
    size_t size = 0;
    std::map<size_t, size_t> free_;   // offset -> length
    void init(size_t s)
    {
        size = s;
        free_.clear();
        free_[0] = s;
    }
    bool alloc(size_t bytes, size_t* off)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Req {
    uint64_t ticket = 0;
    int op = 0;
    int64_t nrhs = 0;
    const double* f = nullptr;
    double* x = nullptr;
    size_t off = 0, bytes = 0;
    SolveLayout Ls;
    int phase = 0;      // 0 up, 1 root, 2 down
    int level = 0;
    int64_t done_tick = -1;   // the tick that issues its last stage (retired once it completes)
    Clock::time_point t_submit;
    // workspace (device)
    double *w = nullptr, *g = nullptr, *phi = nullptr, *u = nullptr, *out = nullptr, *t = nullptr;
};

size_t round_up(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace
}  // namespace rs

struct rs_server {
    std::vector<rs_op*> ops;
    int device = 0;
    cudaStream_t st = nullptr;
    rs::DevMem pool;
    rs::Arena arena;
    int max_inflight = 64;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<rs::Req*> pending;
    std::vector<rs::Req*> inflight;
    std::deque<uint64_t> done_q;
    std::vector<double> lat_ms;
    uint64_t next_ticket = 1;
    int64_t submitted = 0, completed = 0, rhs_completed = 0, ticks = 0, peak_inflight = 0;
    bool stop = false;
    int error = RS_OK;
    std::string error_msg;
    std::thread worker;
    // job staging: one set per tick in flight
    rs::DevMem d_mv[2], d_cp[2];
    void* h_stage[2] = {nullptr, nullptr};
    size_t h_stage_bytes[2] = {0, 0};
    cudaEvent_t ev[2] = {nullptr, nullptr};
};

namespace rs {
namespace {

struct StageJobs {
    std::vector<MvJob> mv;
    std::vector<CopyJob> cp;
    int64_t mv_blocks = 0, cp_elems = 0;
    void add_mv(const Level& L, const DevMem& probs, const DevMem& blk0, int np, int64_t nblk, int rb,
                const double* A, const double* x, double* y, int64_t nrhs)
    {
        if (np <= 0 || nblk <= 0) return;
        MvJob j{probs.as<MatvecProb>(), blk0.as<int64_t>(), np, (int)nrhs, rb, mv_blocks, A, x, y};
        (void)L;
        mv.push_back(j);
        mv_blocks += nblk;
    }
    void add_cp(int mode, int64_t count, int64_t nrhs, int64_t N, const int64_t* idx, const double* in, double* out,
                double a = 0.0, double b = 0.0)
    {
        if (count <= 0) return;
        CopyJob j{cp_elems, mode, (int)nrhs, count, N, idx, in, out, a, b};
        cp.push_back(j);
        cp_elems += (mode == COPY_AXPBY) ? count : count * nrhs;
    }
};

// Stage order of one tick: up U1..U5, root, down D1..D7.
enum { U1, U2, U3, U4, U5, RT, D1, D2, D3, D4, D5, D6, D7, NSTAGE };

void build_jobs(rs_server* s, std::vector<StageJobs>& S)
{
    for (Req* r : s->inflight) {
        if (r->done_tick >= 0) continue;          // finished in a tick still in flight
        rs_op* op = s->ops[r->op];
        const int64_t nr = r->nrhs;
        const int d = op->d;
        if (r->phase == 1) {
            const Level& R = op->lev[0];
            S[RT].add_mv(R, R.d_mv_phi, R.d_mv_phi_blk, R.n_mv_phi, R.b_mv_phi, R.rb_phi, R.d_Phi.as<double>(),
                         r->g + r->Ls.goff[1] * nr, r->phi + r->Ls.goff[1] * nr, nr);
            continue;
        }
        const int l = r->level;
        const Level& L = op->lev[l];
        double* wl = r->w + r->Ls.woff[l] * nr;
        double* gl = r->g + r->Ls.goff[l] * nr;
        double* pl = r->phi + r->Ls.goff[l] * nr;
        if (r->phase == 0) {
            if (l == d) S[U1].add_cp(COPY_GATHER_CM, L.sum_m, nr, op->N, L.d_idx_leaf.as<int64_t>(), r->f, r->u);
            else S[U1].add_cp(COPY_GATHER_ROWS, L.sum_m, nr, 0, L.d_idx_up.as<int64_t>(), r->g + r->Ls.goff[l + 1] * nr, r->u);
            S[U2].add_mv(L, L.d_mv_phi, L.d_mv_phi_blk, L.n_mv_phi, L.b_mv_phi, L.rb_phi, L.d_Phi.as<double>(), r->u, wl, nr);
            S[U3].add_cp(COPY_GATHER_ROWS, L.sum_k, nr, 0, L.d_idx_sk.as<int64_t>(), wl, r->t);
            S[U4].add_mv(L, L.d_mv_T, L.d_mv_T_blk, L.n_mv_T, L.b_mv_T, L.rb_T, L.d_T.as<double>(), wl, r->t, nr);
            S[U5].add_mv(L, L.d_mv_E, L.d_mv_E_blk, L.n_mv_E, L.b_mv_E, L.rb_E, L.d_E.as<double>(), r->t, gl, nr);
        } else {
            S[D1].add_mv(L, L.d_mv_E, L.d_mv_E_blk, L.n_mv_E, L.b_mv_E, L.rb_E, L.d_E.as<double>(), pl, r->t, nr);
            S[D2].add_cp(COPY_AXPBY, L.sum_k * nr, 1, 0, nullptr, gl, r->t, -1.0, 1.0);
            S[D3].add_cp(COPY_SCATTER_ROWS, L.sum_k, nr, 0, L.d_idx_sk.as<int64_t>(), r->t, r->u);
            S[D4].add_mv(L, L.d_mv_Tt, L.d_mv_Tt_blk, L.n_mv_Tt, L.b_mv_Tt, L.rb_Tt, L.d_T.as<double>(), r->t, r->u, nr);
            S[D5].add_mv(L, L.d_mv_phi, L.d_mv_phi_blk, L.n_mv_phi, L.b_mv_phi, L.rb_phi, L.d_Phi.as<double>(), r->u, r->out, nr);
            S[D6].add_cp(COPY_AXPBY, L.sum_m * nr, 1, 0, nullptr, wl, r->out, 1.0, 1.0);
            if (l == d) S[D7].add_cp(COPY_SCATTER_CM, L.sum_m, nr, op->N, L.d_idx_leaf.as<int64_t>(), r->out, r->x);
            else S[D7].add_cp(COPY_SCATTER_ROWS, L.sum_m, nr, 0, L.d_idx_up.as<int64_t>(), r->out,
                              r->phi + r->Ls.goff[l + 1] * nr);
        }
    }
}

// Enqueue one tick through staging set `slot` (whose previous tick has completed) and record
// its completion event; no host synchronisation.
int run_tick(rs_server* s, int slot)
{
    std::vector<StageJobs> S(NSTAGE);
    build_jobs(s, S);
    size_t nmv = 0, ncp = 0;
    for (const StageJobs& j : S) { nmv += j.mv.size(); ncp += j.cp.size(); }
    const size_t bmv = nmv * sizeof(MvJob), bcp = ncp * sizeof(CopyJob);
    if (bmv + bcp > s->h_stage_bytes[slot]) {
        if (s->h_stage[slot]) cudaFreeHost(s->h_stage[slot]);
        s->h_stage[slot] = nullptr;
        s->h_stage_bytes[slot] = 0;
        RS_CUDA(cudaMallocHost(&s->h_stage[slot], 2 * (bmv + bcp) + 4096));
        s->h_stage_bytes[slot] = 2 * (bmv + bcp) + 4096;
    }
    DevMem& dmv = s->d_mv[slot];
    DevMem& dcp = s->d_cp[slot];
    RS_CUDA(dmv.alloc(bmv + 64));
    RS_CUDA(dcp.alloc(bcp + 64));
    MvJob* hm = (MvJob*)s->h_stage[slot];
    CopyJob* hc = (CopyJob*)((char*)s->h_stage[slot] + bmv);
    std::vector<size_t> mv_at(NSTAGE), cp_at(NSTAGE);
    size_t im = 0, ic = 0;
    for (int k = 0; k < NSTAGE; ++k) {
        mv_at[k] = im;
        cp_at[k] = ic;
        std::copy(S[k].mv.begin(), S[k].mv.end(), hm + im);
        std::copy(S[k].cp.begin(), S[k].cp.end(), hc + ic);
        im += S[k].mv.size();
        ic += S[k].cp.size();
    }
    if (bmv) RS_CUDA(cudaMemcpyAsync(dmv.p, hm, bmv, cudaMemcpyHostToDevice, s->st));
    if (bcp) RS_CUDA(cudaMemcpyAsync(dcp.p, hc, bcp, cudaMemcpyHostToDevice, s->st));
    for (int k = 0; k < NSTAGE; ++k) {
        RS_CUDA(launch_copy_jobs(s->st, dcp.as<CopyJob>() + cp_at[k], (int)S[k].cp.size(), S[k].cp_elems));
        RS_CUDA(launch_mv_jobs(s->st, dmv.as<MvJob>() + mv_at[k], (int)S[k].mv.size(), S[k].mv_blocks));
    }
    RS_CUDA(cudaEventRecord(s->ev[slot], s->st));
    return RS_OK;
}

void worker_main(rs_server* s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    int64_t enq = -1, waited = -1;       // last tick enqueued, last tick known complete
    auto fail_all = [&](int rc) {
        s->error = rc;
        s->error_msg = rs_last_error();
        for (Req* r : s->inflight) {
            s->ops[r->op]->inflight -= 1;
            delete r;
        }
        s->inflight.clear();
        s->cv_done.notify_all();
    };
    while (true) {
        // admission: arrival order, in-flight cap, memory budget
        while (!s->pending.empty() && (int)s->inflight.size() < s->max_inflight) {
            Req* r = s->pending.front();
            size_t off = 0;
            if (!s->arena.alloc(r->bytes, &off)) break;
            s->pending.pop_front();
            r->off = off;
            double* base = (double*)((char*)s->pool.p + off);
            r->w = base;
            r->g = r->w + r->Ls.n_w;
            r->phi = r->g + r->Ls.n_g;
            r->u = r->phi + r->Ls.n_g;
            r->out = r->u + r->Ls.n_u;
            r->t = r->out + r->Ls.n_u;
            r->phase = 0;
            r->level = s->ops[r->op]->d;
            s->inflight.push_back(r);
        }
        s->peak_inflight = std::max<int64_t>(s->peak_inflight, (int64_t)s->inflight.size());
        bool active = false;
        for (Req* r : s->inflight) active = active || r->done_tick < 0;
        if (!active && enq == waited) {
            if (s->stop) break;
            s->cv_work.wait(lk);
            continue;
        }
        if (active) {
            const int slot = (int)((enq + 1) & 1);       // its previous tick (enq - 1) has completed
            lk.unlock();
            const int rc = run_tick(s, slot);
            lk.lock();
            if (rc) {
                fail_all(rc);
                break;
            }
            ++enq;
            ++s->ticks;
            for (Req* r : s->inflight) {
                if (r->done_tick >= 0) continue;
                const int d = s->ops[r->op]->d;
                if (r->phase == 0) {
                    if (r->level == 1) r->phase = 1; else --r->level;
                } else if (r->phase == 1) {
                    r->phase = 2;
                    r->level = 1;
                } else if (r->level == d) {
                    r->done_tick = enq;
                } else {
                    ++r->level;
                }
            }
        }
        // wait for the older tick in flight (the newest one too when nothing new was issued)
        const int64_t target = active ? enq - 1 : enq;
        if (target > waited) {
            lk.unlock();
            const cudaError_t e = cudaEventSynchronize(s->ev[target & 1]);
            lk.lock();
            if (e != cudaSuccess) {
                fail_all(cuda_fail(e, "server tick"));
                break;
            }
            waited = target;
            const auto now = Clock::now();
            std::vector<Req*> keep;
            for (Req* r : s->inflight) {
                if (r->done_tick < 0 || r->done_tick > waited) {
                    keep.push_back(r);
                    continue;
                }
                s->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
                s->done_q.push_back(r->ticket);
                ++s->completed;
                s->rhs_completed += r->nrhs;
                s->arena.release(r->off, r->bytes);
                s->ops[r->op]->inflight -= 1;
                delete r;
            }
            s->inflight.swap(keep);
            s->cv_done.notify_all();
        }
    }
}

}  // namespace
}  // namespace rs

using namespace rs;

extern "C" {

int rs_server_create(rs_op* const* ops, int n_ops, size_t mem_budget_bytes, int max_inflight, rs_server** out)
{
    if (!out) return fail(RS_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!ops || n_ops < 1 || mem_budget_bytes < 4096 || max_inflight < 1)
        return fail(RS_E_INVALID, "need operators, a budget of at least 4 KiB and max_inflight >= 1");
    rs_server* s = new (std::nothrow) rs_server();
    if (!s) return fail(RS_E_NOMEM, "host allocation");
    for (int i = 0; i < n_ops; ++i) {
        if (!ops[i] || ops[i]->kind != RS_LAPLACE || ops[i]->opts.precision != RS_FP64 || ops[i]->opts.forward_only) {
            delete s;
            return fail(RS_E_INVALID, "the server batches real FP64 factored operators");
        }
        if (ops[i]->cstore_n > 0) {
            delete s;
            return fail(RS_E_INVALID, "the server batches dense-block operators (factored without k_cut)");
        }
        if (i && ops[i]->device != ops[0]->device) {
            delete s;
            return fail(RS_E_INVALID, "all operators must live on one device");
        }
        s->ops.push_back(ops[i]);
    }
    s->device = ops[0]->device;
    s->max_inflight = max_inflight;
    cudaError_t e = cudaSetDevice(s->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
    for (int q = 0; q < 2 && e == cudaSuccess; ++q) e = cudaEventCreateWithFlags(&s->ev[q], cudaEventDisableTiming);
    if (e == cudaSuccess) e = s->pool.alloc(mem_budget_bytes);
    if (e != cudaSuccess) {
        const int rc = cuda_fail(e, "server setup");
        for (int q = 0; q < 2; ++q)
            if (s->ev[q]) cudaEventDestroy(s->ev[q]);
        if (s->st) cudaStreamDestroy(s->st);
        delete s;
        return rc;
    }
    s->arena.init(mem_budget_bytes & ~(size_t)255);
    for (rs_op* op : s->ops) op->inflight += 1;      // the server holds a reference
    s->worker = std::thread(worker_main, s);
    *out = s;
    return RS_OK;
}

int rs_server_submit(rs_server* s, int op_index, const void* f, int64_t nrhs, void* x, uint64_t* ticket)
{
    if (!s || !f || !x || !ticket || nrhs < 1) return fail(RS_E_INVALID, "bad argument");
    if (op_index < 0 || op_index >= (int)s->ops.size()) return fail(RS_E_INVALID, "operator index out of range");
    if (f == x) return fail(RS_E_INVALID, "x may not alias f");
    if (!is_device_ptr(f) || !is_device_ptr(x)) return fail(RS_E_INVALID, "the server takes device buffers");
    rs_op* op = s->ops[op_index];
    {
        int dev = 0;
        RS_CUDA(cudaGetDevice(&dev));
        if (dev != op->device) return fail(RS_E_INVALID, "the current device is not the one the operator was factored on");
        if (on_other_device(f) || on_other_device(x))
            return fail(RS_E_INVALID, "f or x is device memory of another GPU than the operator's");
    }
    Req* r = new (std::nothrow) Req();
    if (!r) return fail(RS_E_NOMEM, "host allocation");
    r->op = op_index;
    r->nrhs = nrhs;
    r->f = (const double*)f;
    r->x = (double*)x;
    r->Ls = solve_layout(op, nrhs);
    r->bytes = round_up(sizeof(double) * (size_t)r->Ls.total());
    if (r->bytes > s->arena.size) {
        delete r;
        return fail(RS_E_NOMEM, "request workspace exceeds the server's memory budget");
    }
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->error) {
        delete r;
        return fail(s->error, "server stopped: " + s->error_msg);
    }
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    op->inflight += 1;
    s->pending.push_back(r);
    ++s->submitted;
    s->cv_work.notify_one();
    return RS_OK;
}

int rs_server_poll(rs_server* s, uint64_t* done_tickets, int max, int* n_done)
{
    if (!s || !n_done || max < 0 || (max > 0 && !done_tickets)) return fail(RS_E_INVALID, "bad argument");
    std::lock_guard<std::mutex> lk(s->mu);
    int n = 0;
    while (n < max && !s->done_q.empty()) {
        done_tickets[n++] = s->done_q.front();
        s->done_q.pop_front();
    }
    *n_done = n;
    return s->error;
}

int rs_server_drain(rs_server* s, double timeout_s)
{
    if (!s) return fail(RS_E_INVALID, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                        [&] { return s->error || s->completed == s->submitted; });
    if (s->error) return fail(s->error, "server stopped: " + s->error_msg);
    if (!ok) return fail(RS_E_TIMEOUT, "requests still in flight after the timeout");
    return RS_OK;
}

int rs_server_stats(rs_server* s, int64_t* submitted, int64_t* completed, int64_t* rhs_completed, int64_t* ticks,
                    int64_t* peak_inflight)
{
    if (!s) return fail(RS_E_INVALID, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    if (submitted) *submitted = s->submitted;
    if (completed) *completed = s->completed;
    if (rhs_completed) *rhs_completed = s->rhs_completed;
    if (ticks) *ticks = s->ticks;
    if (peak_inflight) *peak_inflight = s->peak_inflight;
    return RS_OK;
}

int rs_server_latencies(rs_server* s, double* out_ms, int64_t max, int64_t* n)
{
    if (!s || !n || max < 0 || (max > 0 && !out_ms)) return fail(RS_E_INVALID, "bad argument");
    std::lock_guard<std::mutex> lk(s->mu);
    const int64_t k = std::min<int64_t>(max, (int64_t)s->lat_ms.size());
    std::copy(s->lat_ms.begin(), s->lat_ms.begin() + k, out_ms);
    *n = (int64_t)s->lat_ms.size();
    return RS_OK;
}

void rs_server_free(rs_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (Req* r : s->pending) {
        s->ops[r->op]->inflight -= 1;
        delete r;
    }
    for (Req* r : s->inflight) {
        s->ops[r->op]->inflight -= 1;
        delete r;
    }
    for (rs_op* op : s->ops) op->inflight -= 1;
    if (s->st) {
        cudaStreamSynchronize(s->st);
        cudaStreamDestroy(s->st);
    }
    for (int q = 0; q < 2; ++q) {
        if (s->ev[q]) cudaEventDestroy(s->ev[q]);
        if (s->h_stage[q]) cudaFreeHost(s->h_stage[q]);
    }
    delete s;
}

}  // extern "C"
