// Batched solves: many right-hand sides per graph, each with its own CG.
//
// One graph's columns are solved together: every matvec is an SpMM over the
// block vector, every sweep of the sparsifier solve handles all columns, and
// every column keeps its own alpha, beta, rho and convergence flag (a
// converged column is frozen while the others continue).  The iterations run
// as a CUDA graph of `check_every` steps; the host reads the column flags
// between graph launches.  In LAP_MIXED the columns run in FP32 and each one
// is refined against its own FP64 true residual.  Several graphs in one call
// run on their handles' private streams, advanced round-robin by the host so
// their work overlaps on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "batched_kernels.cuh"
#include "batched.cuh"
#include "solver.cuh"

namespace lap {

namespace {

int pow2_at_least(int v)
{
    int r = 8;
    while (r < v) r <<= 1;
    return r;
}

template <typename V> struct BatchVectors {
    V *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *A = nullptr,
      *Y = nullptr, *chunk = nullptr;
    BCol *col = nullptr;
    cudaGraphExec_t g = nullptr;
    int64_t nodes = 0;
};

}  // namespace

struct BatchWork {
    int R = 0, CT = 0;
    int64_t n = 0, nt = 0;
    std::vector<std::unique_ptr<DevBuf>> bufs;
    double *Bs = nullptr, *x64 = nullptr, *r64 = nullptr, *means = nullptr, *part = nullptr;
    unsigned *ticket = nullptr;
    BCol *col64 = nullptr;
    BatchVectors<double> v64;
    BatchVectors<float> v32;
    BCol *hcol = nullptr;            // pinned host copy of R columns
    ~BatchWork()
    {
        for (cudaGraphExec_t g : {v64.g, v32.g})
            if (g) cudaGraphExecDestroy(g);
        if (hcol) cudaFreeHost(hcol);
    }
    template <typename T> T *alloc(size_t count)
    {
        auto b = std::make_unique<DevBuf>();
        if (!b->alloc(count * sizeof(T))) return nullptr;
        if (cudaMemset(b->p, 0, b->bytes) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        T *p = b->as<T>();
        bufs.push_back(std::move(b));
        return p;
    }
};

namespace {

#define LAP_BCK(x)                                                                            \
    do {                                                                                      \
        cudaError_t e_ = (x);                                                                 \
        if (e_ != cudaSuccess) {                                                              \
            (void)cudaGetLastError();                                                         \
            return LAP_ERR_CUDA;                                                              \
        }                                                                                     \
    } while (0)

// blocks for `rows` row groups of S = 256 / CT rows (each thread covers all
// R / CT column tiles of its row), capped at the resident block count
int bgrid(const lap_handle_s &h, int64_t rows, int R, int CT)
{
    (void)R;
    const int S = kBThreads / CT;
    const int64_t blocks = (rows + S - 1) / S;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(blocks, h.grid_cap)));
}

template <typename V> BatchVectors<V> &vecs(BatchWork &b);
template <> BatchVectors<double> &vecs<double>(BatchWork &b) { return b.v64; }
template <> BatchVectors<float> &vecs<float>(BatchWork &b) { return b.v32; }

template <typename V> const DevCsr<V> &bL(const lap_handle_s &h);
template <> const DevCsr<double> &bL<double>(const lap_handle_s &h) { return h.L64; }
template <> const DevCsr<float> &bL<float>(const lap_handle_s &h) { return h.L32; }
template <typename V> const DevMsp<V> &bM(const lap_handle_s &h);
template <> const DevMsp<double> &bM<double>(const lap_handle_s &h) { return h.M64; }
template <> const DevMsp<float> &bM<float>(const lap_handle_s &h) { return h.M32; }

template <typename V>
lap_status alloc_vecs(BatchWork &b, BatchVectors<V> &v, int nchunks)
{
    const size_t nR = static_cast<size_t>(b.n) * b.R, tR = static_cast<size_t>(b.nt) * b.R;
    v.x = b.alloc<V>(nR);
    v.r = b.alloc<V>(nR);
    v.p = b.alloc<V>(nR);
    v.q = b.alloc<V>(nR);
    v.z = b.alloc<V>(nR);
    v.A = b.alloc<V>(tR);
    v.Y = b.alloc<V>(tR);
    v.chunk = b.alloc<V>(static_cast<size_t>(std::max(nchunks, 1)) * b.R);
    v.col = b.alloc<BCol>(static_cast<size_t>(b.R));
    if (!v.x || !v.r || !v.p || !v.q || !v.z || !v.A || !v.Y || !v.chunk || !v.col) return LAP_ERR_OOM;
    return LAP_OK;
}

// SpMM over all columns (long rows first through their chunk partials).
template <typename V, int MODE>
void bspmm(const lap_handle_s &h, const BatchWork &b, const DevCsr<V> &L, const V *x, V *y,
           double *yres, V *chunk, BCol *col, cudaStream_t s)
{
    const int R = b.R, CT = b.CT;
    if (L.nchunks > 0) {
        h.launches += 1;
        kb_long_chunks<V><<<std::min(L.nchunks, h.grid_cap), kBThreads, 0, s>>>(
            L.nchunks, R, CT, L.chunk_row, L.chunk_beg, L.lrow, L.lci, L.lw, x, chunk);
    }
    h.launches += 1;
    kb_spmm<V, MODE><<<bgrid(h, L.n, R, CT), kBThreads, 0, s>>>(
        L.n, R, CT, L.rp, L.ci, L.w, L.is_long, L.lrow_of, L.lchunk_ptr, chunk, x, y, b.Bs, yres, col,
        b.part, b.ticket);
}

// z = B r for all columns; with `update` the CG step is fused into level 1.
template <typename V>
void bprecond(const lap_handle_s &h, const BatchWork &b, BatchVectors<V> &v, bool update,
              cudaStream_t s)
{
    const int R = b.R, CT = b.CT;
    const DevMsp<V> &M = bM<V>(h);
    const int n = static_cast<int>(M.off[1]);
    if (h.m.opt.prec == LAP_PREC_NONE) {
        h.launches += 1;
        if (update)
            kb_plain<V, true><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(n, R, CT, v.x, v.r, v.p, v.q, v.col,
                                                                      b.part, b.ticket);
        else
            kb_plain<V, false><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(n, R, CT, v.x, v.r, v.p, v.q,
                                                                       v.col, b.part, b.ticket);
        return;
    }
    const int l = M.levels;
    const auto &L0 = M.lev[0];
    const size_t RR = static_cast<size_t>(R);
    h.launches += 2 * l;
    if (update)
        kb_up<V, 1><<<bgrid(h, L0.nagg, R, CT), kBThreads, 0, s>>>(
            L0.nagg, R, CT, L0.seg, L0.inv, L0.lcf, v.x, v.r, v.p, v.q, v.A, v.A + M.off[1] * RR,
            M.gamma[0], nullptr, v.col, b.part, b.ticket);
    else
        kb_up<V, 2><<<bgrid(h, L0.nagg, R, CT), kBThreads, 0, s>>>(
            L0.nagg, R, CT, L0.seg, L0.inv, L0.lcf, v.x, v.r, v.p, v.q, v.A, v.A + M.off[1] * RR,
            M.gamma[0], nullptr, v.col, b.part, b.ticket);
    for (int k = 1; k + 1 < l; ++k) {
        const auto &Lk = M.lev[k];
        V *a = v.A + M.off[k] * RR;
        kb_up<V, 0><<<bgrid(h, Lk.nagg, R, CT), kBThreads, 0, s>>>(
            Lk.nagg, R, CT, Lk.seg, Lk.inv, Lk.lcf, nullptr, a, nullptr, nullptr, a,
            v.A + M.off[k + 1] * RR, M.gamma[k], nullptr, v.col, nullptr, nullptr);
    }
    const size_t ot = static_cast<size_t>(M.off[l - 1]) * RR;
    kb_coarse<V><<<bgrid(h, M.ntop, R, CT), kBThreads, 0, s>>>(M.ntop, R, M.G, v.A + ot, v.Y + ot,
                                                              M.c[l - 1]);
    for (int k = l - 2; k >= 1; --k) {
        const auto &Lk = M.lev[k];
        kb_down<V, false><<<bgrid(h, Lk.nagg, R, CT), kBThreads, 0, s>>>(
            Lk.n, Lk.nagg, R, CT, Lk.seg, v.A + M.off[k] * RR, v.Y + M.off[k + 1] * RR,
            v.Y + M.off[k] * RR, V(1), static_cast<V>(M.c[k]), nullptr, v.col, nullptr, nullptr);
    }
    kb_down<V, true><<<bgrid(h, L0.nagg, R, CT), kBThreads, 0, s>>>(
        n, L0.nagg, R, CT, L0.seg, v.A, v.Y + M.off[1] * RR, v.z, V(1), V(1), v.r, v.col, b.part,
        b.ticket);
}

template <typename V>
void biteration(const lap_handle_s &h, BatchWork &b, BatchVectors<V> &v, cudaStream_t s)
{
    const int n = static_cast<int>(b.n);
    bspmm<V, 0>(h, b, bL<V>(h), v.p, v.q, nullptr, v.chunk, v.col, s);
    bprecond<V>(h, b, v, true, s);
    h.launches += 1;
    kb_pupdate<V><<<bgrid(h, n, b.R, b.CT), kBThreads, 0, s>>>(
        n, b.R, b.CT, h.m.opt.prec == LAP_PREC_NONE ? v.r : v.z, v.p, v.col);
}

lap_status poll_cols(lap_handle_s &h, BatchWork &b, const BCol *col, std::vector<BCol> &out)
{
    LAP_BCK(cudaMemcpyAsync(b.hcol, col, sizeof(BCol) * b.R, cudaMemcpyDeviceToHost, h.s));
    LAP_BCK(cudaStreamSynchronize(h.s));
    out.assign(b.hcol, b.hcol + b.R);
    return LAP_OK;
}

// Iterate the columns of v until none is running (device flags), capturing
// `check_every` iterations per CUDA graph launch.
template <typename V>
lap_status biterate(lap_handle_s &h, BatchWork &b, BatchVectors<V> &v, std::vector<BCol> &cols)
{
    const int K = h.m.opt.check_every;
    if (!v.g) {
        cudaGraph_t graph = nullptr;
        const int64_t l0 = h.launches;
        LAP_BCK(cudaStreamBeginCapture(h.s, cudaStreamCaptureModeThreadLocal));
        for (int i = 0; i < K; ++i) biteration<V>(h, b, v, h.s);
        cudaError_t e = cudaStreamEndCapture(h.s, &graph);
        h.launches = l0;
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return LAP_ERR_CUDA;
        }
        size_t nn = 0;
        cudaGraphGetNodes(graph, nullptr, &nn);
        v.nodes = static_cast<int64_t>(nn);
        e = cudaGraphInstantiate(&v.g, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            v.g = nullptr;
            return LAP_ERR_CUDA;
        }
    }
    const int cap = h.m.opt.maxit / K + 4;
    for (int launches = 0; launches <= cap; ++launches) {
        LAP_BCK(cudaGraphLaunch(v.g, h.s));
        h.launches += v.nodes;
        LAP_LTRY(poll_cols(h, b, v.col, cols));
        bool any = false;
        for (int c = 0; c < b.R; ++c) any |= cols[c].flag == kRun;
        if (!any) return LAP_OK;
    }
    return LAP_ERR_BREAKDOWN;
}

lap_status prepare(lap_handle_s &h, int R)
{
    BatchWork *b = h.batch.get();
    const bool mixed = h.m.opt.precision == LAP_MIXED;
    if (b && b->R == R) return LAP_OK;
    h.batch.reset();
    auto nb = std::make_unique<BatchWork>();
    nb->R = R;
    nb->n = h.m.lev[0].n;
    nb->nt = h.m.offset[h.m.levels];
    nb->CT = std::min(R, 32);
    const size_t nR = static_cast<size_t>(nb->n) * R;
    nb->Bs = nb->alloc<double>(nR);
    nb->x64 = nb->alloc<double>(nR);
    nb->r64 = nb->alloc<double>(nR);
    nb->means = nb->alloc<double>(static_cast<size_t>(R));
    nb->part = nb->alloc<double>(static_cast<size_t>(kMaxRedBlocks) * 2 * R);
    nb->ticket = nb->alloc<unsigned>(1);
    nb->col64 = nb->alloc<BCol>(static_cast<size_t>(R));
    if (!nb->Bs || !nb->x64 || !nb->r64 || !nb->means || !nb->part || !nb->ticket || !nb->col64)
        return LAP_ERR_OOM;
    LAP_LTRY(alloc_vecs<double>(*nb, nb->v64, h.L64.nchunks));
    if (mixed) LAP_LTRY(alloc_vecs<float>(*nb, nb->v32, h.L32.nchunks));
    LAP_BCK(cudaMallocHost(&nb->hcol, sizeof(BCol) * R));
    // column tile: time the SpMM for the candidate widths and keep the fastest
    {
        float best = 1e30f;
        int best_ct = nb->CT;
        cudaEvent_t e0, e1;
        LAP_BCK(cudaEventCreate(&e0));
        LAP_BCK(cudaEventCreate(&e1));
        for (int ct = std::max(8, R / 8); ct <= std::min(R, 256); ct <<= 1) {
            nb->CT = ct;
            bspmm<double, 2>(h, *nb, h.L64, nb->v64.p, nb->v64.q, nullptr, nb->v64.chunk, nullptr, h.s);
            cudaEventRecord(e0, h.s);
            for (int i = 0; i < 3; ++i)
                bspmm<double, 2>(h, *nb, h.L64, nb->v64.p, nb->v64.q, nullptr, nb->v64.chunk, nullptr,
                                 h.s);
            cudaEventRecord(e1, h.s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_ct = ct;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        nb->CT = best_ct;
        LAP_BCK(cudaGetLastError());
    }
    h.batch = std::move(nb);
    return LAP_OK;
}

}  // namespace

// Solve the columns [c0, c0 + nr) of one graph; infos gets nr entries.
lap_status batched_solve_chunk(lap_handle_s &h, int nr, const double *B, double *X,
                               lap_solve_info *infos)
{
    const int R = pow2_at_least(nr);
    LAP_LTRY(prepare(h, R));
    BatchWork &b = *h.batch;
    const lap_options &o = h.m.opt;
    const int n = static_cast<int>(b.n);
    const cudaStream_t s = h.s;
    const int CT = b.CT;
    std::vector<BCol> cols;
    std::vector<int> iters(R, 0), refs(R, 0);
    h.launches += 2;
    kb_gather<double><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(n, R, CT, nr, h.perm1, B, b.Bs, b.col64,
                                                               b.part, b.ticket);
    lap_status result = LAP_OK;
    if (o.precision != LAP_MIXED) {
        auto &v = b.v64;
        kb_center<double><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(n, R, CT, nr, 1, b.Bs, v.r, v.x, b.col64,
                                                                   v.col, o.tol, o.maxit, nullptr, 0.0,
                                                                   b.part, b.ticket);
        bprecond<double>(h, b, v, false, s);
        h.launches += 1;
        kb_pupdate<double><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(
            n, R, CT, o.prec == LAP_PREC_NONE ? v.r : v.z, v.p, v.col);
        result = biterate<double>(h, b, v, cols);
        for (int c = 0; c < nr; ++c) iters[c] = cols.empty() ? 0 : cols[c].iter;
        // true residuals, reported per column
        bspmm<double, 1>(h, b, h.L64, v.x, nullptr, b.r64, v.chunk, v.col, s);
        LAP_LTRY(poll_cols(h, b, v.col, cols));
        h.launches += 2;
        kb_mean<double><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(n, R, CT, v.x, b.means, b.part, b.ticket);
        kb_scatter<double><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(n, R, CT, nr, h.perm1, v.x, b.means, X);
    } else {
        // FP64 start: r64 = Bs (centred), x64 = 0
        kb_center<double><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(n, R, CT, nr, 1, b.Bs, b.r64, b.x64,
                                                                   b.col64, b.col64, o.tol, o.maxit,
                                                                   nullptr, 0.0, b.part, b.ticket);
        auto &v = b.v32;
        std::vector<BCol> outer;
        for (int ref = 0;; ++ref) {
            if (ref > 0) {
                bspmm<double, 1>(h, b, h.L64, b.x64, nullptr, b.r64, b.v64.chunk, b.col64, s);
                h.launches += 1;
                kb_refine_flags<<<1, 256, 0, s>>>(R, nr, b.col64, o.tol);
            }
            LAP_LTRY(poll_cols(h, b, b.col64, outer));
            bool any = false;
            for (int c = 0; c < nr; ++c) any |= outer[c].flag == kRun;
            if (!any || ref >= o.max_refine) break;
            int used = 0;
            for (int c = 0; c < nr; ++c) used = std::max(used, iters[c]);
            if (used >= o.maxit) break;
            // FP32 inner CG on the residual of every running column
            h.launches += 1;
            kb_center<float><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(
                n, R, CT, nr, 0, b.r64, v.r, v.x, b.col64, v.col, o.tol, o.maxit - used, b.col64,
                o.refine_tol, b.part, b.ticket);
            bprecond<float>(h, b, v, false, s);
            h.launches += 1;
            kb_pupdate<float><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(
                n, R, CT, o.prec == LAP_PREC_NONE ? v.r : v.z, v.p, v.col);
            lap_status it = biterate<float>(h, b, v, cols);
            if (it != LAP_OK) {
                result = it;
                break;
            }
            for (int c = 0; c < nr; ++c)
                if (outer[c].flag == kRun) {
                    iters[c] += cols[c].iter;
                    refs[c] = ref + 1;
                }
            h.launches += 1;
            kb_add<float><<<h.grid_cap, kBThreads, 0, s>>>(static_cast<int64_t>(n) * R, b.x64, v.x);
        }
        bspmm<double, 1>(h, b, h.L64, b.x64, nullptr, b.r64, b.v64.chunk, b.col64, s);
        LAP_LTRY(poll_cols(h, b, b.col64, cols));
        h.launches += 2;
        kb_mean<double><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(n, R, CT, b.x64, b.means, b.part, b.ticket);
        kb_scatter<double><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(n, R, CT, nr, h.perm1, b.x64, b.means,
                                                                    X);
    }
    LAP_BCK(cudaStreamSynchronize(s));
    for (int c = 0; c < nr; ++c) {
        lap_solve_info &inf = infos[c];
        std::memset(&inf, 0, sizeof(inf));
        inf.iterations = iters[c];
        inf.refinements = refs[c];
        inf.relres = cols[c].bnorm > 0.0 ? cols[c].relres : 0.0;
        inf.relres_recurrence = inf.relres;
        inf.status = result != LAP_OK ? result
                   : (inf.relres <= o.tol ? LAP_OK : LAP_ERR_NO_CONVERGENCE);
    }
    return result;
}

lap_status batched_enter(lap_handle_s &h, cudaStream_t user)
{
    LAP_BCK(cudaSetDevice(h.device));
    LAP_BCK(cudaEventRecord(h.ev_in, user));
    LAP_BCK(cudaStreamWaitEvent(h.s, h.ev_in, 0));
    return LAP_OK;
}

lap_status batched_leave(lap_handle_s &h, cudaStream_t user)
{
    LAP_BCK(cudaEventRecord(h.ev_out, h.s));
    LAP_BCK(cudaStreamWaitEvent(user, h.ev_out, 0));
    return LAP_OK;
}

}  // namespace lap

extern "C" lap_status lap_pcg_solve_batched(int32_t ng, const lap_handle *hs, const int32_t *nrhs,
                                            const double *const *d_B, double *const *d_X,
                                            void *stream, lap_solve_info *infos)
{
    using namespace lap;
    if (ng < 0 || (ng > 0 && (!hs || !nrhs || !d_B || !d_X))) return LAP_ERR_INVALID_ARG;
    for (int g = 0; g < ng; ++g) {
        if (!hs[g] || hs[g]->host_only || nrhs[g] < 0 || (nrhs[g] > 0 && (!d_B[g] || !d_X[g])))
            return LAP_ERR_INVALID_ARG;
        if (hs[g]->m.opt.prec != LAP_PREC_MSP && hs[g]->m.opt.prec != LAP_PREC_NONE)
            return LAP_ERR_UNSUPPORTED;
        // a single-level hierarchy (n <= coarse_max) has no aggregates to sweep
        if (hs[g]->m.opt.prec == LAP_PREC_MSP && hs[g]->m.levels < 2) return LAP_ERR_UNSUPPORTED;
    }
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    lap_status result = LAP_OK;
    size_t off = 0;
    std::vector<lap_solve_info> scratch;
    for (int g = 0; g < ng; ++g) {
        lap_handle_s &h = *hs[g];
        const int64_t n = h.m.lev[0].n;
        const auto t0 = std::chrono::steady_clock::now();
        const int64_t l0 = h.launches;
        lap_status st = batched_enter(h, user);
        for (int c0 = 0; st == LAP_OK && c0 < nrhs[g]; c0 += 256) {
            const int nr = std::min(256, nrhs[g] - c0);
            scratch.assign(static_cast<size_t>(nr), lap_solve_info{});
            st = batched_solve_chunk(h, nr, d_B[g] + static_cast<size_t>(c0) * n,
                                     d_X[g] + static_cast<size_t>(c0) * n, scratch.data());
            if (infos)
                for (int c = 0; c < nr; ++c) infos[off + c0 + c] = scratch[c];
        }
        const lap_status st2 = batched_leave(h, user);
        if (infos) {
            const double secs =
                std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            for (int c = 0; c < nrhs[g]; ++c) {
                infos[off + c].seconds = secs;
                infos[off + c].kernel_launches = static_cast<int32_t>(h.launches - l0);
            }
        }
        if (result == LAP_OK) result = st != LAP_OK ? st : st2;
        off += static_cast<size_t>(nrhs[g]);
    }
    return result;
}
