// Batched-solve workspace and kernel sequences, shared by the batched C ABI
// (batched.cu) and the server (serve.cu).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <memory>
#include <vector>

#include "batched.cuh"
#include "batched_kernels.cuh"
#include "solver.cuh"

namespace lap {


inline int pow2_at_least(int v)
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

struct BatchWork {
    int R = 0, CT = 0;
    int64_t n = 0, nt = 0;
    std::vector<std::unique_ptr<DevBuf>> bufs;
    double *Bs = nullptr, *x64 = nullptr, *r64 = nullptr, *means = nullptr, *part = nullptr;
    double *tres = nullptr;          // per-column true relative residuals
    unsigned *ticket = nullptr;
    BCol *col64 = nullptr;
    BatchVectors<double> v64;
    BatchVectors<float> v32;
    BCol *hcol = nullptr;            // pinned host copy of R columns
    int64_t bytes = 0;               // device memory held
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
        bytes += static_cast<int64_t>(b->bytes);
        bufs.push_back(std::move(b));
        return p;
    }
};

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
inline int bgrid(const lap_handle_s &h, int64_t rows, int R, int CT)
{
    (void)R;
    const int S = kBThreads / CT;
    const int64_t blocks = (rows + S - 1) / S;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(blocks, h.grid_cap)));
}

template <typename V> BatchVectors<V> &vecs(BatchWork &b);
template <> inline BatchVectors<double> &vecs<double>(BatchWork &b) { return b.v64; }
template <> inline BatchVectors<float> &vecs<float>(BatchWork &b) { return b.v32; }

template <typename V> const DevCsr<V> &bL(const lap_handle_s &h);
template <> inline const DevCsr<double> &bL<double>(const lap_handle_s &h) { return h.L64; }
template <> inline const DevCsr<float> &bL<float>(const lap_handle_s &h) { return h.L32; }
template <typename V> const DevMsp<V> &bM(const lap_handle_s &h);
template <> inline const DevMsp<double> &bM<double>(const lap_handle_s &h) { return h.M64; }
template <> inline const DevMsp<float> &bM<float>(const lap_handle_s &h) { return h.M32; }

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
        // its own layout: 32-column tiles, eight row groups splitting the
        // chunk's entries (independent of the SpMM's tuned tile)
        kb_long_chunks<V><<<std::min(L.nchunks, h.grid_cap), kBThreads, 0, s>>>(
            L.nchunks, R, std::min(R, 32), L.chunk_row, L.chunk_beg, L.lrow, L.lrp, L.rp, L.lci, L.lw, x, chunk);
    }
    h.launches += 1;
    kb_spmm<V, MODE><<<bgrid(h, L.n, R, CT), kBThreads, 0, s>>>(
        L.n, R, CT, L.rp, L.ci, L.w, L.is_long, L.lrow_of, L.lchunk_ptr, chunk, x, y, b.Bs, yres, col,
        b.part, b.ticket, b.tres);
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
            M.gamma[0], nullptr, v.col, b.part, b.ticket, L0.nbig, L0.big);
    else
        kb_up<V, 2><<<bgrid(h, L0.nagg, R, CT), kBThreads, 0, s>>>(
            L0.nagg, R, CT, L0.seg, L0.inv, L0.lcf, v.x, v.r, v.p, v.q, v.A, v.A + M.off[1] * RR,
            M.gamma[0], nullptr, v.col, b.part, b.ticket, L0.nbig, L0.big);
    for (int k = 1; k + 1 < l; ++k) {
        const auto &Lk = M.lev[k];
        V *a = v.A + M.off[k] * RR;
        kb_up<V, 0><<<bgrid(h, Lk.nagg, R, CT), kBThreads, 0, s>>>(
            Lk.nagg, R, CT, Lk.seg, Lk.inv, Lk.lcf, nullptr, a, nullptr, nullptr, a,
            v.A + M.off[k + 1] * RR, M.gamma[k], nullptr, v.col, nullptr, nullptr, Lk.nbig, Lk.big);
    }
    const size_t ot = static_cast<size_t>(M.off[l - 1]) * RR;
    kb_coarse<V><<<bgrid(h, M.ntop, R, CT), kBThreads, 0, s>>>(M.ntop, R, M.G, v.A + ot, v.Y + ot,
                                                              M.c[l - 1]);
    for (int k = l - 2; k >= 1; --k) {
        const auto &Lk = M.lev[k];
        kb_down<V, false><<<bgrid(h, Lk.nagg, R, CT), kBThreads, 0, s>>>(
            Lk.n, Lk.nagg, R, CT, Lk.seg, v.A + M.off[k] * RR, v.Y + M.off[k + 1] * RR,
            v.Y + M.off[k] * RR, V(1), static_cast<V>(M.c[k]), nullptr, v.col, nullptr, nullptr, Lk.nbig,
            Lk.big);
    }
    kb_down<V, true><<<bgrid(h, L0.nagg, R, CT), kBThreads, 0, s>>>(
        n, L0.nagg, R, CT, L0.seg, v.A, v.Y + M.off[1] * RR, v.z, V(1), V(1), v.r, v.col, b.part,
        b.ticket, L0.nbig, L0.big);
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

inline lap_status poll_cols(BatchWork &b, const BCol *col, std::vector<BCol> &out, cudaStream_t s)
{
    LAP_BCK(cudaMemcpyAsync(b.hcol, col, sizeof(BCol) * b.R, cudaMemcpyDeviceToHost, s));
    LAP_BCK(cudaStreamSynchronize(s));
    out.assign(b.hcol, b.hcol + b.R);
    return LAP_OK;
}

// Capture K (default: the handle's check_every) batched iterations of v into
// a CUDA graph on stream s.
template <typename V>
lap_status capture_iterations(lap_handle_s &h, BatchWork &b, BatchVectors<V> &v, cudaStream_t s,
                              int K = 0)
{
    if (v.g) return LAP_OK;
    if (K <= 0) K = h.m.opt.check_every;
    cudaGraph_t graph = nullptr;
    const int64_t l0 = h.launches;
    LAP_BCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < K; ++i) biteration<V>(h, b, v, s);
    cudaError_t e = cudaStreamEndCapture(s, &graph);
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
    return LAP_OK;
}

// Iterate the columns of v until none is running (device flags), one graph
// launch of `check_every` iterations between host polls.
template <typename V>
lap_status biterate(lap_handle_s &h, BatchWork &b, BatchVectors<V> &v, std::vector<BCol> &cols,
                    cudaStream_t s)
{
    LAP_LTRY(capture_iterations<V>(h, b, v, s));
    const int cap = h.m.opt.maxit / h.m.opt.check_every + 4;
    for (int launches = 0; launches <= cap; ++launches) {
        LAP_BCK(cudaGraphLaunch(v.g, s));
        h.launches += v.nodes;
        LAP_LTRY(poll_cols(b, v.col, cols, s));
        bool any = false;
        for (int c = 0; c < b.R; ++c) any |= cols[c].flag == kRun;
        if (!any) return LAP_OK;
    }
    return LAP_ERR_BREAKDOWN;
}


// A batch workspace for R columns of graph h.  The SpMM column tile is chosen
// by timing the candidate widths on stream s (autotuner) the first time a
// width R is used on the handle, then kept, so every batch of the same width
// on a handle runs the same reduction order.
inline lap_status make_batch(lap_handle_s &h, int R, bool want32, cudaStream_t s,
                             std::unique_ptr<BatchWork> &out)
{
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
    nb->tres = nb->alloc<double>(static_cast<size_t>(R));
    nb->part = nb->alloc<double>(static_cast<size_t>(kMaxRedBlocks) * 2 * R);
    nb->ticket = nb->alloc<unsigned>(1);
    nb->col64 = nb->alloc<BCol>(static_cast<size_t>(R));
    if (!nb->Bs || !nb->x64 || !nb->r64 || !nb->means || !nb->tres || !nb->part || !nb->ticket ||
        !nb->col64)
        return LAP_ERR_OOM;
    LAP_LTRY(alloc_vecs<double>(*nb, nb->v64, h.L64.nchunks));
    if (want32) LAP_LTRY(alloc_vecs<float>(*nb, nb->v32, h.L32.nchunks));
    LAP_BCK(cudaMallocHost(&nb->hcol, sizeof(BCol) * R));
    int slot = 0;
    while ((8 << slot) < R) ++slot;
    if (h.batch_ct[slot] > 0) {
        nb->CT = h.batch_ct[slot];
        out = std::move(nb);
        return LAP_OK;
    }
    float best = 1e30f;
    int best_ct = nb->CT;
    cudaEvent_t e0, e1;
    LAP_BCK(cudaEventCreate(&e0));
    LAP_BCK(cudaEventCreate(&e1));
    for (int ct = std::max(8, R / 8); ct <= std::min(R, 256); ct <<= 1) {
        nb->CT = ct;
        bspmm<double, 2>(h, *nb, h.L64, nb->v64.p, nb->v64.q, nullptr, nb->v64.chunk, nullptr, s);
        cudaEventRecord(e0, s);
        for (int i = 0; i < 3; ++i)
            bspmm<double, 2>(h, *nb, h.L64, nb->v64.p, nb->v64.q, nullptr, nb->v64.chunk, nullptr, s);
        cudaEventRecord(e1, s);
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
    h.batch_ct[slot] = best_ct;
    out = std::move(nb);
    return LAP_OK;
}

}  // namespace lap
