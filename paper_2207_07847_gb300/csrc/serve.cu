// Serving: continuous batching of Laplacian solve requests.
//
// A server owns one worker thread.  Every graph (handle) with work in flight
// has a resident column batch (BatchWork, R columns) on its own CUDA stream;
// a request occupies a contiguous range of its graph's columns.  The worker
// loop, between two launches of `check_every` CG iterations of every batch:
//   1. admits queued requests into free columns of their graph's batch,
//      creating the batch if the HBM budget allows it (admission by memory
//      footprint);
//   2. starts the admitted columns (their CG state only; the other columns of
//      the batch keep their iterates) and launches the next iteration chunk of
//      every batch -- batches of different graphs overlap on the device;
//   3. reads the column flags, retires every request whose columns have all
//      stopped (true residuals, projection, results written back, callback),
//      and frees a batch once it is empty.
// On a LAP_MIXED handle the columns run the FP32 CG and each request is
// refined against its own FP64 true residual: when a request's inner solves
// have stopped, their corrections are added to its FP64 solution and the
// columns whose true residual misses the tolerance start the next inner solve
// from it.  On a LAP_FP64 handle the columns run in FP64 and restart from the
// true residual if their recurrence converged but the true residual did not.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <type_traits>
#include <unordered_map>

#include "batched_impl.cuh"

namespace lap {
namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { kQueued = 0, kActive = 1, kDone = 2 };

struct Request {
    uint64_t id = 0;
    lap_handle_s *h = nullptr;
    int nrhs = 0;
    const double *B = nullptr;
    double *X = nullptr;
    lap_done_cb cb = nullptr;
    void *user = nullptr;
    Clock::time_point arrival;
    int state = kQueued;
    bool cancel = false;
    bool started = false;
    int c0 = -1;
    int restarts = 0;                // true-residual restarts (FP64) or refinements (mixed)
    int iters = 0;                   // iterations of the finished inner solves (mixed)
    int64_t launches0 = 0;           // batch launch counter at admission
    lap_solve_info info{};
};

struct GraphBatch {
    lap_handle_s *h = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    std::unique_ptr<BatchWork> w;
    std::vector<Request *> owner;    // per column
    std::vector<BCol> cols;
    int64_t launches = 0;            // kernels launched for this batch
    bool launched = false;
    bool rejoin = false;             // restarted columns wait for their first direction
    bool mixed = false;              // FP32 columns refined in FP64
    ~GraphBatch()
    {
        if (s) cudaStreamSynchronize(s);
        w.reset();
        if (ev) cudaEventDestroy(ev);
        if (s) cudaStreamDestroy(s);
    }
};

constexpr int kServeRestarts = 4;     // true-residual restarts per request

int batch_width(const lap_server_options &o) { return std::min(256, pow2_at_least(o.max_slots)); }

int iterations_per_launch(const lap_server_options &o, const lap_handle_s &h)
{
    return o.check_every > 0 ? o.check_every : h.m.opt.check_every;
}

bool serve_mixed(const lap_handle_s &h) { return h.m.opt.precision == LAP_MIXED && h.L32.w != nullptr; }

// Upper estimate of make_batch's allocations for R columns (FP64 vectors, and
// FP32 ones for a mixed handle).
int64_t batch_bytes_estimate(const lap_handle_s &h, int R)
{
    const int64_t n = h.m.lev[0].n, nt = h.m.offset[h.m.levels];
    int64_t words = R * (8 * n + 2 * nt + std::max(h.L64.nchunks, 1)) + 2 * int64_t(kMaxRedBlocks) * R;
    if (serve_mixed(h)) words += R * (5 * n + 2 * nt + std::max(h.L32.nchunks, 1)) / 2;
    return 8 * words + (int64_t(1) << 20);
}

}  // namespace
}  // namespace lap

struct lap_server_s {
    lap_server_options opt{};
    int device = 0;
    int R = 8;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<lap::Request *> queue;                                   // under mu
    std::map<uint64_t, std::unique_ptr<lap::Request>> reqs;             // under mu
    std::unordered_map<lap_handle_s *, std::unique_ptr<lap::GraphBatch>> batches;   // worker only
    int64_t used_bytes = 0;                                             // worker only
    bool stop = false;                                                  // under mu
    uint64_t next_id = 1;                                               // under mu
};

namespace lap {
namespace {

// Finish request r (worker thread): record, wake waiters, call back.  r is
// not touched after its state becomes kDone (a waiter may free it).
void complete(lap_server_s &S, Request *r, lap_status st)
{
    r->info.status = st;
    r->info.seconds = std::chrono::duration<double>(Clock::now() - r->arrival).count();
    const lap_done_cb cb = r->cb;
    void *user = r->user;
    const uint64_t id = r->id;
    const lap_solve_info info = r->info;
    {
        std::lock_guard<std::mutex> g(S.mu);
        r->state = kDone;
    }
    S.cv_done.notify_all();
    if (cb) cb(user, id, &info);
}

lap_status create_batch(lap_server_s &S, lap_handle_s *h, GraphBatch *&out)
{
    auto gb = std::make_unique<GraphBatch>();
    gb->h = h;
    LAP_BCK(cudaStreamCreateWithFlags(&gb->s, cudaStreamNonBlocking));
    LAP_BCK(cudaEventCreateWithFlags(&gb->ev, cudaEventDisableTiming));
    gb->mixed = serve_mixed(*h);
    LAP_LTRY(make_batch(*h, S.R, gb->mixed, gb->s, gb->w));
    gb->owner.assign(static_cast<size_t>(S.R), nullptr);
    gb->cols.assign(static_cast<size_t>(S.R), BCol{});
    // every column starts stopped; a request's columns are started on join
    kb_set_flags<<<1, 256, 0, gb->s>>>(S.R, 0, S.R, gb->mixed ? gb->w->v32.col : gb->w->v64.col, kConverged);
    LAP_BCK(cudaGetLastError());
    gb->launches += 1;
    S.used_bytes += gb->w->bytes;
    out = gb.get();
    S.batches[h] = std::move(gb);
    return LAP_OK;
}

int free_range(const GraphBatch &gb, int k)
{
    const int R = static_cast<int>(gb.owner.size());
    for (int c0 = 0; c0 + k <= R; ++c0) {
        int c = c0;
        while (c < c0 + k && gb.owner[c] == nullptr) ++c;
        if (c == c0 + k) return c0;
        c0 = c;                       // skip past the occupied column
    }
    return -1;
}

// Admission: queued requests take free columns of their graph's batch; a
// graph without a batch gets one if the budget allows.  Requests that wait
// keep their place in the queue.
void admit(lap_server_s &S)
{
    std::vector<std::pair<Request *, lap_status>> finished;
    std::vector<Request *> pending;
    {
        std::lock_guard<std::mutex> g(S.mu);
        pending.assign(S.queue.begin(), S.queue.end());
    }
    std::vector<Request *> taken;
    for (Request *r : pending) {
        bool cancel;
        {
            std::lock_guard<std::mutex> g(S.mu);
            cancel = r->cancel;
        }
        if (cancel) {
            finished.push_back({r, LAP_ERR_CANCELLED});
            taken.push_back(r);
            continue;
        }
        auto bit = S.batches.find(r->h);
        GraphBatch *gb = bit == S.batches.end() ? nullptr : bit->second.get();
        if (!gb) {
            const int64_t est = batch_bytes_estimate(*r->h, S.R);
            if (!S.batches.empty() && S.used_bytes + est > S.opt.hbm_budget_bytes) continue;
            const lap_status st = create_batch(S, r->h, gb);
            if (st != LAP_OK) {
                S.batches.erase(r->h);
                finished.push_back({r, st});
                taken.push_back(r);
                continue;
            }
        }
        const int c0 = free_range(*gb, r->nrhs);
        if (c0 < 0) continue;
        for (int c = c0; c < c0 + r->nrhs; ++c) gb->owner[c] = r;
        r->c0 = c0;
        r->launches0 = gb->launches;
        taken.push_back(r);
        std::lock_guard<std::mutex> g(S.mu);
        r->state = kActive;
    }
    if (!taken.empty()) {
        std::lock_guard<std::mutex> g(S.mu);
        for (Request *r : taken)
            for (auto it = S.queue.begin(); it != S.queue.end(); ++it)
                if (*it == r) {
                    S.queue.erase(it);
                    break;
                }
    }
    for (auto &f : finished) complete(S, f.first, f.second);
}

// Start the newly admitted columns of gb, then launch one chunk of
// iterations and the copy of the column states.
template <typename V>
lap_status launch_t(lap_server_s &S, GraphBatch &gb)
{
    lap_handle_s &h = *gb.h;
    BatchWork &b = *gb.w;
    auto &v = vecs<V>(b);
    const bool mixed = std::is_same<V, float>::value;
    const int n = static_cast<int>(b.n), R = b.R, CT = b.CT;
    const lap_options &o = h.m.opt;
    const int64_t l0 = h.launches;
    // the first inner solve of a refined column: relative tolerance
    // max(refine_tol, 0.3 tol), at most 0.5
    const double tol0 = mixed ? std::min(0.5, std::max(o.refine_tol, 0.3 * o.tol)) : o.tol;
    bool joined = false;
    for (int c = 0; c < R; ++c) {
        Request *r = gb.owner[c];
        if (!r || r->started || c != r->c0) continue;
        kb_join_gather<<<bgrid(h, n, R, CT), kBThreads, 0, gb.s>>>(n, R, CT, r->c0, r->nrhs, h.perm1, r->B,
                                                                   b.Bs, v.col, b.part, b.ticket);
        kb_join_center<V><<<bgrid(h, n, R, CT), kBThreads, 0, gb.s>>>(
            n, R, CT, r->c0, r->nrhs, b.Bs, v.r, v.x, v.col, tol0, o.maxit, b.part, b.ticket,
            mixed ? b.x64 : nullptr);
        h.launches += 2;
        r->started = true;
        joined = true;
    }
    if (joined || gb.rejoin) {
        // z = B r for every column: the running columns recompute the z, rho
        // they already hold (same operands, same order: the same bits), and
        // only the joining (or restarted) columns take their first direction
        gb.rejoin = false;
        bprecond<V>(h, b, v, false, gb.s);
        kb_pupdate_join<V><<<bgrid(h, n, R, CT), kBThreads, 0, gb.s>>>(
            n, R, CT, o.prec == LAP_PREC_NONE ? v.r : v.z, v.p, v.col);
        kb_clear_join<<<1, 256, 0, gb.s>>>(R, v.col);
        h.launches += 2;
    }
    LAP_BCK(cudaGetLastError());
    LAP_LTRY(capture_iterations<V>(h, b, v, gb.s, iterations_per_launch(S.opt, h)));
    LAP_BCK(cudaGraphLaunch(v.g, gb.s));
    h.launches += v.nodes;
    LAP_BCK(cudaMemcpyAsync(b.hcol, v.col, sizeof(BCol) * R, cudaMemcpyDeviceToHost, gb.s));
    LAP_BCK(cudaEventRecord(gb.ev, gb.s));
    gb.launches += h.launches - l0;
    gb.launched = true;
    return LAP_OK;
}

lap_status launch(lap_server_s &S, GraphBatch &gb)
{
    return gb.mixed ? launch_t<float>(S, gb) : launch_t<double>(S, gb);
}

lap_status column_status(const BCol &c)
{
    switch (c.flag) {
    case kConverged: return LAP_OK;
    case kBreakdown: return LAP_ERR_BREAKDOWN;
    case kMaxit: return LAP_ERR_NO_CONVERGENCE;
    default: return LAP_ERR_NO_CONVERGENCE;
    }
}

// Retire the requests of gb whose columns have all stopped (or that were
// cancelled or timed out): refine or restart them, or write their solutions
// and complete them.
template <typename V>
lap_status retire_t(lap_server_s &S, GraphBatch &gb)
{
    lap_handle_s &h = *gb.h;
    BatchWork &b = *gb.w;
    auto &v = vecs<V>(b);
    const bool mixed = std::is_same<V, float>::value;
    const lap_options &o = h.m.opt;
    const int n = static_cast<int>(b.n), R = b.R, CT = b.CT;
    const int64_t l0 = h.launches;
    LAP_BCK(cudaEventSynchronize(gb.ev));
    gb.cols.assign(b.hcol, b.hcol + R);
    struct Done {
        Request *r;
        lap_status forced;               // LAP_OK: status from the columns
    };
    std::vector<Done> done;
    const auto now = Clock::now();
    for (int c = 0; c < R; ++c) {
        Request *r = gb.owner[c];
        // a request admitted after this chunk was launched has not started:
        // its columns still hold the stopped states of their previous owner
        if (!r || c != r->c0 || !r->started) continue;
        bool stopped = true;
        for (int j = r->c0; j < r->c0 + r->nrhs; ++j) stopped &= gb.cols[j].flag != kRun;
        bool cancel;
        {
            std::lock_guard<std::mutex> g(S.mu);
            cancel = r->cancel;
        }
        const double age = std::chrono::duration<double>(now - r->arrival).count();
        const bool late = o.timeout_s > 0.0 && age > o.timeout_s;
        lap_status forced = cancel ? LAP_ERR_CANCELLED : (late && !stopped) ? LAP_ERR_TIMEOUT : LAP_OK;
        if (!stopped && forced != LAP_OK) {
            kb_set_flags<<<1, 256, 0, gb.s>>>(R, r->c0, r->nrhs, v.col, kConverged);
            h.launches += 1;
            stopped = true;
        }
        if (stopped) done.push_back({r, forced});
    }
    if (done.empty()) return LAP_OK;
    double *xs = b.x64;                  // the FP64 solution
    if (mixed) {
        // the ended inner solves' corrections into the FP64 solutions
        for (const Done &d : done) {
            kb_add_cols<V><<<bgrid(h, n, R, CT), kBThreads, 0, gb.s>>>(n, R, CT, d.r->c0, d.r->nrhs, b.x64, v.x);
            h.launches += 1;
            int it = 0;
            for (int j = d.r->c0; j < d.r->c0 + d.r->nrhs; ++j) it = std::max(it, gb.cols[j].iter);
            d.r->iters += it;
        }
    } else {
        xs = reinterpret_cast<double *>(b.v64.x);
    }
    // true residuals of all columns (column states untouched) to r64 and tres
    bspmm<double, 3>(h, b, h.L64, xs, nullptr, b.r64, b.v64.chunk, v.col, gb.s);
    std::vector<double> tres(static_cast<size_t>(R));
    LAP_BCK(cudaMemcpyAsync(tres.data(), b.tres, sizeof(double) * R, cudaMemcpyDeviceToHost, gb.s));
    LAP_BCK(cudaStreamSynchronize(gb.s));
    // columns whose true residual misses the tolerance go on from it: the next
    // refinement step (mixed), or a restart of a converged recurrence (FP64)
    const double tol = o.tol;
    std::vector<Done> fin;
    for (const Done &d : done) {
        bool miss = false, again = false;
        for (int j = d.r->c0; j < d.r->c0 + d.r->nrhs; ++j) {
            miss |= !(tres[j] <= tol);
            again |= gb.cols[j].flag == kConverged && !(tres[j] <= tol);
        }
        const bool go = mixed ? (miss && d.r->restarts < o.max_refine && d.r->iters < o.maxit)
                              : (again && d.r->restarts < kServeRestarts);
        if (d.forced == LAP_OK && go) {
            d.r->restarts += 1;
            if (mixed) {
                kb_refine_copy<V><<<bgrid(h, n, R, CT), kBThreads, 0, gb.s>>>(
                    n, R, CT, d.r->c0, d.r->nrhs, b.r64, v.r, v.x, b.tres, tol);
                kb_refine_flags<<<1, 256, 0, gb.s>>>(R, d.r->c0, d.r->nrhs, v.col, b.tres, tol, o.refine_tol,
                                                     o.maxit);
            } else {
                kb_restart_copy<V><<<bgrid(h, n, R, CT), kBThreads, 0, gb.s>>>(
                    n, R, CT, d.r->c0, d.r->nrhs, b.r64, v.r, v.col, b.tres, tol);
                kb_restart_flags<<<1, 256, 0, gb.s>>>(R, d.r->c0, d.r->nrhs, v.col, b.tres, tol);
            }
            h.launches += 2;
            gb.rejoin = true;
        } else {
            fin.push_back(d);
        }
    }
    done.swap(fin);
    if (done.empty()) {
        gb.launches += h.launches - l0;
        return LAP_OK;
    }
    kb_mean<double><<<bgrid(h, n, R, CT), kBThreads, 0, gb.s>>>(n, R, CT, xs, b.means, b.part, b.ticket);
    h.launches += 1;
    for (const Done &d : done) {
        kb_scatter_range<double><<<bgrid(h, n, R, CT), kBThreads, 0, gb.s>>>(
            n, R, CT, d.r->c0, d.r->nrhs, h.perm1, xs, b.means, d.r->X);
        h.launches += 1;
    }
    LAP_BCK(cudaStreamSynchronize(gb.s));
    gb.launches += h.launches - l0;
    for (const Done &d : done) {
        Request *r = d.r;
        int it = 0;
        double rel = 0.0;
        lap_status st = LAP_OK;
        for (int j = r->c0; j < r->c0 + r->nrhs; ++j) {
            it = std::max(it, gb.cols[j].iter);
            rel = std::max(rel, tres[j]);
            const lap_status cs = column_status(gb.cols[j]);
            if (st == LAP_OK) st = cs;
            gb.owner[j] = nullptr;
        }
        // an inner solve that stops at its tolerance is converged; the outer
        // test is the true residual
        if (mixed && st == LAP_ERR_NO_CONVERGENCE && rel <= tol) st = LAP_OK;
        if (st == LAP_OK && !(rel <= tol)) st = LAP_ERR_NO_CONVERGENCE;
        if (d.forced != LAP_OK) st = d.forced;
        r->info.iterations = mixed ? r->iters : it;
        r->info.refinements = mixed ? r->restarts : 0;
        r->info.restarts = mixed ? 0 : r->restarts;
        r->info.relres = rel;
        r->info.relres_recurrence = 0.0;
        for (int j = r->c0; j < r->c0 + r->nrhs; ++j)
            r->info.relres_recurrence = std::max(r->info.relres_recurrence, gb.cols[j].relres);
        r->info.kernel_launches = static_cast<int32_t>(std::min<int64_t>(gb.launches - r->launches0, INT32_MAX));
        complete(S, r, st);
    }
    return LAP_OK;
}

lap_status retire(lap_server_s &S, GraphBatch &gb)
{
    return gb.mixed ? retire_t<float>(S, gb) : retire_t<double>(S, gb);
}

// A batch that failed on the device: complete its requests with `st` and drop it.
void fail_batch(lap_server_s &S, GraphBatch &gb, lap_status st)
{
    std::vector<Request *> rs;
    for (int c = 0; c < static_cast<int>(gb.owner.size()); ++c)
        if (gb.owner[c] && gb.owner[c]->c0 == c) rs.push_back(gb.owner[c]);
    std::fill(gb.owner.begin(), gb.owner.end(), nullptr);
    for (Request *r : rs) complete(S, r, st);
}

void worker_loop(lap_server_s &S)
{
    cudaSetDevice(S.device);
    for (;;) {
        admit(S);
        bool any_active = false;
        for (auto &kv : S.batches) {
            GraphBatch &gb = *kv.second;
            gb.launched = false;
            bool has = false;
            for (Request *r : gb.owner) has |= r != nullptr;
            if (!has) continue;
            const lap_status st = launch(S, gb);
            if (st != LAP_OK) fail_batch(S, gb, st);
            else any_active = true;
        }
        for (auto &kv : S.batches)
            if (kv.second->launched) {
                const lap_status st = retire(S, *kv.second);
                if (st != LAP_OK) fail_batch(S, *kv.second, st);
            }
        // free the batches with no request in them and none waiting for them
        {
            std::vector<lap_handle_s *> wanted;
            {
                std::lock_guard<std::mutex> g(S.mu);
                for (Request *q : S.queue) wanted.push_back(q->h);
            }
            for (auto it = S.batches.begin(); it != S.batches.end();) {
                bool empty = true;
                for (Request *r : it->second->owner) empty &= r == nullptr;
                const bool want = std::find(wanted.begin(), wanted.end(), it->first) != wanted.end();
                if (empty && !want) {
                    S.used_bytes -= it->second->w->bytes;
                    it = S.batches.erase(it);
                } else {
                    ++it;
                }
            }
        }
        if (!any_active) {
            std::unique_lock<std::mutex> lk(S.mu);
            if (S.stop && S.queue.empty()) break;
            S.cv_work.wait_for(lk, std::chrono::milliseconds(2));
        }
    }
    S.batches.clear();
}

}  // namespace
}  // namespace lap

using namespace lap;

extern "C" {

void lap_server_options_default(lap_server_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->hbm_budget_bytes = int64_t(32) << 30;
    o->max_slots = 16;
    o->check_every = 8;
}

lap_status lap_server_create(const lap_server_options *opts, lap_server *out)
{
    if (!out) return LAP_ERR_INVALID_ARG;
    *out = nullptr;
    auto S = std::make_unique<lap_server_s>();
    if (opts) S->opt = *opts;
    else lap_server_options_default(&S->opt);
    if (S->opt.max_slots < 1 || S->opt.max_slots > 256 || S->opt.hbm_budget_bytes <= 0)
        return LAP_ERR_INVALID_ARG;
    S->R = batch_width(S->opt);
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        (void)cudaGetLastError();
        return LAP_ERR_CUDA;
    }
    lap_server_s *raw = S.get();
    try {
        S->worker = std::thread([raw] { worker_loop(*raw); });
    } catch (...) {
        return LAP_ERR_OOM;
    }
    *out = S.release();
    return LAP_OK;
}

lap_status lap_serve_submit(lap_server s, lap_handle h, int32_t nrhs, const double *d_B, double *d_X,
                            lap_done_cb cb, void *user, uint64_t *req_id)
{
    if (!s || !h || h->host_only || nrhs < 1 || nrhs > s->R || !d_B || !d_X) return LAP_ERR_INVALID_ARG;
    if (h->m.opt.prec != LAP_PREC_MSP && h->m.opt.prec != LAP_PREC_NONE) return LAP_ERR_UNSUPPORTED;
    if (h->m.opt.prec == LAP_PREC_MSP && h->m.levels < 2) return LAP_ERR_UNSUPPORTED;
    if (batch_bytes_estimate(*h, s->R) > s->opt.hbm_budget_bytes) return LAP_ERR_BUSY;
    auto r = std::make_unique<Request>();
    r->h = h;
    r->nrhs = nrhs;
    r->B = d_B;
    r->X = d_X;
    r->cb = cb;
    r->user = user;
    r->arrival = Clock::now();
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->stop) return LAP_ERR_CANCELLED;
        r->id = s->next_id++;
        if (req_id) *req_id = r->id;
        s->queue.push_back(r.get());
        s->reqs[r->id] = std::move(r);
    }
    s->cv_work.notify_one();
    return LAP_OK;
}

lap_status lap_serve_wait(lap_server s, uint64_t req_id, double timeout_s, lap_solve_info *info)
{
    if (!s) return LAP_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return LAP_ERR_INVALID_ARG;
    Request *r = it->second.get();
    auto pred = [&] { return r->state == kDone; };
    if (timeout_s > 0) {
        if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) return LAP_ERR_TIMEOUT;
    } else {
        s->cv_done.wait(lk, pred);
    }
    const lap_solve_info res = r->info;
    s->reqs.erase(req_id);                 // the iterator may be stale after waiting
    if (info) *info = res;
    return static_cast<lap_status>(res.status);
}

lap_status lap_serve_cancel(lap_server s, uint64_t req_id)
{
    if (!s) return LAP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return LAP_ERR_INVALID_ARG;
    it->second->cancel = true;
    s->cv_work.notify_one();
    return LAP_OK;
}

void lap_server_destroy(lap_server s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        for (Request *r : s->queue) r->cancel = true;     // never admitted: cancelled
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    delete s;
}

}  // extern "C"
