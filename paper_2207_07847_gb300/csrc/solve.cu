// Host driver and C ABI of the GB300 graph-Laplacian solver.
//
// A handle owns the device copy of the setup (tree-ordered level-1 Laplacian,
// elimination data of T, top-level pseudo-inverse, optionally L_H), the
// workspaces of its solves and a private CUDA stream.  Each solve runs its CG
// iterations as CUDA graphs of `check_every` iterations; every scalar of the
// iteration (alpha, beta, rho, the convergence flag) lives on the device, so
// the host only reads a small status block between graph launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "device_model.cuh"
#include "kernels.cuh"
#include "lap_internal.h"
#include "solver.cuh"

// ---------------------------------------------------------------------------
// allocator
// ---------------------------------------------------------------------------
namespace {
std::mutex g_alloc_mu;
lap_alloc_fn g_alloc = nullptr;
lap_free_fn g_free = nullptr;
void *g_alloc_ctx = nullptr;
}  // namespace

namespace lap {
void *dev_alloc(size_t bytes, void *stream)
{
    lap_alloc_fn a;
    void *ctx;
    {
        std::lock_guard<std::mutex> g(g_alloc_mu);
        a = g_alloc;
        ctx = g_alloc_ctx;
    }
    if (a) return a(ctx, bytes, stream);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void *p, void *stream)
{
    lap_free_fn f;
    void *ctx;
    {
        std::lock_guard<std::mutex> g(g_alloc_mu);
        f = g_free;
        ctx = g_alloc_ctx;
    }
    if (!p) return;
    if (f) f(ctx, p, stream);
    else cudaFree(p);
}
}  // namespace lap

using namespace lap;

extern "C" {

void lap_options_default(lap_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->prec = LAP_PREC_MSP;
    o->precision = LAP_FP64;
    o->mu = 0.8;
    o->coarse_max = 32;
    o->max_levels = 0;
    o->seed = 0;
    o->order_random = 1;
    o->tol = 1e-8;
    o->maxit = 1000;
    o->inner_tol = 1e-2;
    o->inner_maxit = 200;
    o->refine_tol = 1e-4;
    o->max_refine = 20;
    o->check_every = 8;
    o->timeout_s = 0.0;
    o->spmv_tpr = 0;
    o->host_only = 0;
    o->stall_window = 1000;
    o->krylov = LAP_KRYLOV_CG;
    o->restart = 30;
}

const char *lap_status_string(int32_t s)
{
    switch (s) {
    case LAP_OK: return "ok";
    case LAP_ERR_INVALID_ARG: return "invalid argument";
    case LAP_ERR_NOT_SYMMETRIC: return "matrix not symmetric";
    case LAP_ERR_NOT_CONNECTED: return "graph not connected";
    case LAP_ERR_BAD_WEIGHT: return "edge weight not positive and finite";
    case LAP_ERR_OOM: return "out of memory";
    case LAP_ERR_CUDA: return "CUDA error";
    case LAP_ERR_NO_CONVERGENCE: return "no convergence within maxit";
    case LAP_ERR_BREAKDOWN: return "CG breakdown";
    case LAP_ERR_TIMEOUT: return "timeout";
    case LAP_ERR_CANCELLED: return "cancelled";
    case LAP_ERR_BUSY: return "busy";
    case LAP_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
    }
}

lap_status lap_set_allocator(lap_alloc_fn alloc, lap_free_fn release, void *ctx)
{
    if ((alloc == nullptr) != (release == nullptr)) return LAP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(g_alloc_mu);
    g_alloc = alloc;
    g_free = release;
    g_alloc_ctx = ctx;
    return LAP_OK;
}

lap_status lap_setup(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const double *w,
                     const lap_options *opts, void *stream, lap_handle *out)
{
    if (!out) return LAP_ERR_INVALID_ARG;
    *out = nullptr;
    lap_options o;
    if (opts) o = *opts;
    else lap_options_default(&o);
    if (o.prec < LAP_PREC_NONE || o.prec > LAP_PREC_PEGP_EXACT) return LAP_ERR_INVALID_ARG;
    if (o.precision != LAP_FP64 && o.precision != LAP_MIXED) return LAP_ERR_INVALID_ARG;
    if (!(o.tol > 0.0) || o.maxit < 1 || o.check_every < 1) return LAP_ERR_INVALID_ARG;
    if (o.krylov != LAP_KRYLOV_CG && o.krylov != LAP_KRYLOV_FGMRES) return LAP_ERR_INVALID_ARG;
    if (o.restart < 1 || o.restart > 128) return LAP_ERR_INVALID_ARG;
    if (o.matching != LAP_MATCH_GREEDY && o.matching != LAP_MATCH_HANDSHAKE) return LAP_ERR_INVALID_ARG;
    if (o.setup_device != 0 && o.setup_device != 1) return LAP_ERR_INVALID_ARG;
    std::string why;
    lap_status st = validate_csr(n, row_ptr, col_idx, w, &why);
    if (st != LAP_OK) return st;
    std::unique_ptr<lap_handle_s> h(new (std::nothrow) lap_handle_s());
    if (!h) return LAP_ERR_OOM;
    try {
        st = build_model(n, row_ptr, col_idx, w, o, h->m, stream);
    } catch (const std::bad_alloc &) {
        return LAP_ERR_OOM;
    }
    if (st != LAP_OK) return st;
    if (!o.host_only) {
        st = upload_model(*h, static_cast<cudaStream_t>(stream));
        if (st != LAP_OK) {
            destroy_handle(*h);
            return st;
        }
    }
    h->host_only = o.host_only != 0;
    *out = h.release();
    return LAP_OK;
}

void lap_destroy(lap_handle h)
{
    if (!h) return;
    destroy_handle(*h);
    delete h;
}

lap_status lap_update_options(lap_handle h, const lap_options *opts)
{
    if (!h || !opts) return LAP_ERR_INVALID_ARG;
    return update_options(*h, *opts);
}

lap_status lap_kernel_bench(lap_handle h, int32_t kernel, int32_t precision, int32_t reps,
                            double *ms_per_launch, double *bytes_per_launch)
{
    if (!h || h->host_only || !ms_per_launch || !bytes_per_launch || reps < 1) return LAP_ERR_INVALID_ARG;
    return kernel_bench(*h, kernel, precision, reps, ms_per_launch, bytes_per_launch);
}

lap_status lap_get_history(lap_handle h, double *h_out, int32_t cap, int32_t *count)
{
    if (!h || !count || h->host_only || (cap > 0 && !h_out)) return LAP_ERR_INVALID_ARG;
    int c = 0;
    lap_status st = get_history(*h, h_out, cap, &c);
    *count = c;
    return st;
}

lap_status lap_get_lanczos(lap_handle h, double *h_alpha, double *h_beta, int32_t cap, int32_t *count)
{
    if (!h || !count || h->host_only || (cap > 0 && !h_alpha && !h_beta)) return LAP_ERR_INVALID_ARG;
    int c = 0;
    lap_status st = get_lanczos(*h, h_alpha, h_beta, cap, &c);
    *count = c;
    return st;
}

lap_status lap_estimate_condition(lap_handle h, int32_t *steps, double *lambda_min, double *lambda_max)
{
    if (!h || h->host_only || !lambda_min || !lambda_max) return LAP_ERR_INVALID_ARG;
    if (h->m.opt.prec == LAP_PREC_PEGP_INNER) return LAP_ERR_UNSUPPORTED;
    int c = 0;
    lap_status st = get_lanczos(*h, nullptr, nullptr, 0, &c);
    if (st != LAP_OK) return st;
    if (c < 1) return LAP_ERR_INVALID_ARG;
    std::vector<double> al(static_cast<size_t>(c)), be(static_cast<size_t>(c));
    st = get_lanczos(*h, al.data(), be.data(), c, &c);
    if (st != LAP_OK) return st;
    std::vector<double> a, b;
    if (!lanczos_tridiagonal(al.data(), be.data(), c, a, b)) return LAP_ERR_BREAKDOWN;
    if (!tridiag_extremes(a, b, lambda_min, lambda_max)) return LAP_ERR_BREAKDOWN;
    if (steps) *steps = c;
    return LAP_OK;
}

lap_status lap_estimate_stretch(lap_handle h, int32_t samples, uint64_t seed, double *h_vals)
{
    if (!h || h->host_only || samples < 1 || !h_vals) return LAP_ERR_INVALID_ARG;
    return estimate_stretch(*h, samples, seed, h_vals);
}

lap_status lap_get_hierarchy_info(lap_handle h, lap_hierarchy_info *info)
{
    if (!h || !info) return LAP_ERR_INVALID_ARG;
    std::memset(info, 0, sizeof(*info));
    const HostModel &m = h->m;
    info->levels = m.levels;
    info->prec = m.opt.prec;
    info->n = m.lev[0].n;
    info->ntilde = m.offset[m.levels];
    info->nnz = m.lev[0].rp[m.lev[0].n];
    for (int k = 0; k < m.levels && k < LAP_MAX_LEVELS; ++k) info->level_size[k] = m.lev[k].n;
    info->nnz_H = m.has_LH ? m.LH.rp[m.LH.n] : 0;
    info->edges_T = m.edges_T;
    info->device_bytes = h->device_bytes;
    info->mu = m.mu;
    return LAP_OK;
}

lap_status lap_get_aggregates(lap_handle h, int32_t level, int32_t *agg_out, int32_t *pair_a,
                              int32_t *pair_b)
{
    if (!h || !agg_out) return LAP_ERR_INVALID_ARG;
    const HostModel &m = h->m;
    if (level < 1 || level >= m.levels) return LAP_ERR_INVALID_ARG;
    const HostLevel &L = m.lev[level - 1];
    std::copy(L.agg.begin(), L.agg.end(), agg_out);
    if (pair_a) std::copy(L.pa.begin(), L.pa.end(), pair_a);
    if (pair_b) std::copy(L.pb.begin(), L.pb.end(), pair_b);
    return LAP_OK;
}

lap_status lap_get_expanded_edges(lap_handle h, int32_t which, int64_t cap, int64_t *count,
                                  int64_t *i, int64_t *j, double *w)
{
    if (!h || !count || (which != 0 && which != 1)) return LAP_ERR_INVALID_ARG;
    if (which == 0 && !h->m.has_LH) return LAP_ERR_INVALID_ARG;
    std::vector<int64_t> I, J;
    std::vector<double> W;
    expanded_edges(h->m, which, I, J, W);
    *count = static_cast<int64_t>(I.size());
    if (!i) return LAP_OK;
    if (cap < *count || !j || !w) return LAP_ERR_INVALID_ARG;
    std::copy(I.begin(), I.end(), i);
    std::copy(J.begin(), J.end(), j);
    std::copy(W.begin(), W.end(), w);
    return LAP_OK;
}

lap_status lap_laplacian_apply(lap_handle h, const double *d_x, double *d_y, void *stream)
{
    if (!h || !d_x || !d_y || h->host_only) return LAP_ERR_INVALID_ARG;
    return block_laplacian(*h, d_x, d_y, static_cast<cudaStream_t>(stream));
}

lap_status lap_precond_apply(lap_handle h, const double *d_r, double *d_z, void *stream)
{
    if (!h || !d_r || !d_z || h->host_only) return LAP_ERR_INVALID_ARG;
    return block_precond(*h, d_r, d_z, static_cast<cudaStream_t>(stream));
}

lap_status lap_restrict_apply(lap_handle h, const double *d_r, double *d_rt, void *stream)
{
    if (!h || !d_r || !d_rt || h->host_only) return LAP_ERR_INVALID_ARG;
    return block_restrict(*h, d_r, d_rt, static_cast<cudaStream_t>(stream));
}

lap_status lap_prolong_apply(lap_handle h, const double *d_yt, double *d_z, void *stream)
{
    if (!h || !d_yt || !d_z || h->host_only) return LAP_ERR_INVALID_ARG;
    return block_prolong(*h, d_yt, d_z, static_cast<cudaStream_t>(stream));
}

lap_status lap_msp_solve(lap_handle h, const double *d_rt, double *d_yt, void *stream)
{
    if (!h || !d_rt || !d_yt || h->host_only) return LAP_ERR_INVALID_ARG;
    return block_msp_solve(*h, d_rt, d_yt, static_cast<cudaStream_t>(stream));
}

lap_status lap_pegp_apply(lap_handle h, const double *d_xt, double *d_yt, void *stream)
{
    if (!h || !d_xt || !d_yt || h->host_only) return LAP_ERR_INVALID_ARG;
    if (!h->m.has_LH) return LAP_ERR_INVALID_ARG;
    return block_pegp(*h, d_xt, d_yt, static_cast<cudaStream_t>(stream));
}

lap_status lap_pcg_solve(lap_handle h, const double *d_b, double *d_x, void *stream,
                         lap_solve_info *info)
{
    lap_solve_info local;
    lap_solve_info *inf = info ? info : &local;
    std::memset(inf, 0, sizeof(*inf));
    if (!h || !d_b || !d_x || d_b == d_x || h->host_only) return LAP_ERR_INVALID_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t l0 = h->launches;
    lap_status st = solve_device(*h, d_b, d_x, static_cast<cudaStream_t>(stream), *inf);
    inf->kernel_launches = static_cast<int32_t>(h->launches - l0);
    inf->status = st;
    inf->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

lap_status lap_pcg_solve_host(lap_handle h, const double *h_b, double *h_x, void *stream,
                              lap_solve_info *info)
{
    lap_solve_info local;
    lap_solve_info *inf = info ? info : &local;
    std::memset(inf, 0, sizeof(*inf));
    if (!h || !h_b || !h_x || h->host_only) return LAP_ERR_INVALID_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t l0 = h->launches;
    lap_status st = solve_host(*h, h_b, h_x, static_cast<cudaStream_t>(stream), *inf);
    inf->kernel_launches = static_cast<int32_t>(h->launches - l0);
    inf->status = st;
    inf->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

}  // extern "C"
