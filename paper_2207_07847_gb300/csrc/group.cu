// Solve groups: many graphs of uneven size solved together, one launch per
// PCG phase for all of them (group_kernels.cuh).
//
// lap_group_create merges the graphs' setups block-diagonally on the host:
//   * graphs ordered by decreasing hierarchy depth (stable), so that on every
//     level the graphs that have it form a prefix, and the graphs that
//     aggregate it further a prefix of those;
//   * merged level k = the level-k vertices (tree order) of those graphs, in
//     that order; the level-1 Laplacians concatenated with their columns
//     shifted; level k's segment array = the aggregating graphs' segments
//     shifted to merged indices; pair and leftover coefficients concatenated
//     (their offsets then match the merged indices, since leftovers of a
//     graph number n_k - 2 n_(k+1));
//   * each graph's top level keeps its own dense pseudo-inverse and scale
//     c_l (l its depth), applied for all graphs by one launch.
// The restriction factors and prolongation coefficients of level k depend
// only on mu and k, so the graphs of a group share mu.  lap_pcg_solve_group
// then runs the batched CG (every (graph, column) pair with its own scalars;
// FP64, or FP32 columns refined against their FP64 true residuals) with each
// phase launched once over the merged arrays, iterations captured in CUDA
// graphs of check_every steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <numeric>
#include <vector>

#include "batched_impl.cuh"
#include "group_kernels.cuh"

namespace lap {
namespace {

constexpr int kGroupMaxBlocks = 128;     // blocks per graph in the reducing kernels

template <typename V> struct GroupPrec {
    V *w = nullptr;                       // merged level-1 weights
    std::vector<V *> inv, lcf;            // per level below the deepest top
};

template <typename V> struct GroupVecs {
    V *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *A = nullptr, *Y = nullptr;
    BCol *col = nullptr;
    cudaGraphExec_t g = nullptr;
    int64_t nodes = 0;
};

}  // namespace
}  // namespace lap

struct lap_group_s {
    int G = 0, device = 0, R = 0, CT = 0, grid_cap = 0;
    cudaStream_t s = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<lap_handle_s *> hs;             // caller's order
    std::vector<int> order;                     // merged position -> caller's index
    lap_options opt{};                          // the first handle's solve options
    int kmax = 0;                               // deepest hierarchy (levels)
    int n_all = 0;
    int64_t nt_all = 0;
    std::vector<int64_t> off;                   // merged expanded offset of each level, kmax + 1
    std::vector<int> nlev, nagg;                // merged vertices per level, aggregates per level
    std::vector<double> gamma, cc;              // c_(k+1)/c_k and c_k per level
    std::vector<std::unique_ptr<lap::DevBuf>> bufs;
    int64_t bytes = 0;
    // device arrays
    int *rp = nullptr, *ci = nullptr, *perm = nullptr, *gid = nullptr, *nrhs = nullptr, *n_of = nullptr;
    int *top_row = nullptr, *ntop = nullptr;
    const double **Gs = nullptr;
    double *scale = nullptr;
    double **Bp = nullptr;                      // device tables of the caller's pointers
    double **Xp = nullptr;
    lap::GRange *rows = nullptr, *aggs0 = nullptr;
    std::vector<int *> seg;
    lap::GroupPrec<double> p64;
    lap::GroupPrec<float> p32;
    bool mixed = false, plain = false;
    // workspace for R columns
    double *Bs = nullptr, *x64 = nullptr, *r64 = nullptr, *means = nullptr, *part = nullptr;
    unsigned *ticket = nullptr;
    lap::BCol *col64 = nullptr, *hcol = nullptr;
    lap::GroupVecs<double> v64;
    lap::GroupVecs<float> v32;
    std::vector<std::unique_ptr<lap::DevBuf>> wbufs;
    int64_t launches = 0;

    template <typename T> T *alloc(std::vector<std::unique_ptr<lap::DevBuf>> &into, size_t count)
    {
        auto b = std::make_unique<lap::DevBuf>();
        if (!b->alloc(count * sizeof(T))) return nullptr;
        if (cudaMemset(b->p, 0, b->bytes) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        T *p = b->as<T>();
        bytes += static_cast<int64_t>(b->bytes);
        into.push_back(std::move(b));
        return p;
    }
    template <typename T> lap_status upload(T **dst, const std::vector<T> &src)
    {
        *dst = alloc<T>(bufs, std::max<size_t>(src.size(), 1));
        if (!*dst) return LAP_ERR_OOM;
        if (!src.empty() &&
            cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
            (void)cudaGetLastError();
            return LAP_ERR_CUDA;
        }
        return LAP_OK;
    }
    void drop_work()
    {
        for (cudaGraphExec_t *g : {&v64.g, &v32.g})
            if (*g) {
                cudaGraphExecDestroy(*g);
                *g = nullptr;
            }
        if (hcol) cudaFreeHost(hcol);
        hcol = nullptr;
        for (auto &b : wbufs) bytes -= static_cast<int64_t>(b->bytes);
        wbufs.clear();
        R = 0;
    }
    ~lap_group_s()
    {
        if (s) cudaStreamSynchronize(s);
        drop_work();
        bufs.clear();
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        if (s) cudaStreamDestroy(s);
    }
};

namespace lap {
namespace {

#define LAP_GCK(x)                        \
    do {                                  \
        cudaError_t e_ = (x);             \
        if (e_ != cudaSuccess) {          \
            (void)cudaGetLastError();     \
            return LAP_ERR_CUDA;          \
        }                                 \
    } while (0)

int nblocks(int items, int S) { return std::max(1, std::min(kGroupMaxBlocks, (items + S - 1) / S)); }

template <typename V>
lap_status upload_prec(lap_group_s &G, GroupPrec<V> &P, const std::vector<double> &w,
                       const std::vector<std::vector<double>> &inv, const std::vector<std::vector<double>> &lcf)
{
    auto conv = [](const std::vector<double> &a) {
        std::vector<V> o(a.size());
        for (size_t i = 0; i < a.size(); ++i) o[i] = static_cast<V>(a[i]);
        return o;
    };
    LAP_LTRY(G.upload(&P.w, conv(w)));
    P.inv.assign(inv.size(), nullptr);
    P.lcf.assign(lcf.size(), nullptr);
    for (size_t k = 0; k < inv.size(); ++k) {
        LAP_LTRY(G.upload(&P.inv[k], conv(inv[k])));
        LAP_LTRY(G.upload(&P.lcf[k], conv(lcf[k])));
    }
    return LAP_OK;
}

lap_status build_group(lap_group_s &G)
{
    const int ng = G.G;
    std::vector<int> ord(ng);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(),
                     [&](int a, int b) { return G.hs[a]->m.levels > G.hs[b]->m.levels; });
    G.order = ord;
    G.kmax = G.hs[ord[0]]->m.levels;
    const int K = G.kmax;
    // merged level sizes and each graph's base on each level
    std::vector<std::vector<int>> base(K, std::vector<int>(ng, -1));
    G.nlev.assign(K, 0);
    for (int k = 0; k < K; ++k)
        for (int t = 0; t < ng; ++t) {
            const HostModel &m = G.hs[ord[t]]->m;
            if (m.levels > k) {
                base[k][t] = G.nlev[k];
                G.nlev[k] += static_cast<int>(m.lev[k].n);
            }
        }
    G.off.assign(K + 1, 0);
    for (int k = 0; k < K; ++k) G.off[k + 1] = G.off[k] + G.nlev[k];
    G.n_all = G.nlev[0];
    G.nt_all = G.off[K];
    // level-1 CSR, permutation, graph ids
    std::vector<int> rp(1, 0), ci, perm, gid, n_of(ng);
    std::vector<double> w;
    for (int t = 0; t < ng; ++t) {
        const HostModel &m = G.hs[ord[t]]->m;
        const HostCsr &L = m.L1;
        const int b = base[0][t];
        n_of[t] = static_cast<int>(L.n);
        for (int64_t i = 0; i < L.n; ++i) {
            for (int64_t p = L.rp[i]; p < L.rp[i + 1]; ++p) {
                ci.push_back(b + L.ci[p]);
                w.push_back(L.w[p]);
            }
            rp.push_back(static_cast<int>(ci.size()));
            perm.push_back(m.lev[0].perm[i]);
            gid.push_back(t);
        }
    }
    if (ci.size() > static_cast<size_t>(INT32_MAX)) return LAP_ERR_UNSUPPORTED;
    // levels: segments (merged), coefficients (concatenated)
    const int nl = std::max(K - 1, 0);
    std::vector<std::vector<int>> segs(nl);
    std::vector<std::vector<double>> inv(nl), lcf(nl);
    G.nagg.assign(nl, 0);
    for (int k = 0; k < nl; ++k) {
        std::vector<int> &sg = segs[k];
        for (int t = 0; t < ng; ++t) {
            const HostModel &m = G.hs[ord[t]]->m;
            if (m.levels <= k + 1) continue;           // no aggregates on this level
            const HostMspLevel &S = m.msp[k];
            const int b = base[k][t];
            for (int64_t J = 0; J < S.nagg; ++J) sg.push_back(b + S.seg[J]);
            inv[k].insert(inv[k].end(), S.inv.begin(), S.inv.end());
            lcf[k].insert(lcf[k].end(), S.lcf.begin(), S.lcf.end());
            G.nagg[k] += static_cast<int>(S.nagg);
        }
        // end of the last aggregating graph's members
        int end = 0;
        for (int t = 0; t < ng; ++t) {
            const HostModel &m = G.hs[ord[t]]->m;
            if (m.levels > k + 1) end = base[k][t] + static_cast<int>(m.lev[k].n);
        }
        sg.push_back(end);
    }
    // per-level coefficients (shared mu)
    const HostModel &m0 = G.hs[ord[0]]->m;
    G.cc.assign(m0.c.begin(), m0.c.end());
    G.gamma.assign(nl, 0.0);
    for (int k = 0; k < nl; ++k) G.gamma[k] = m0.c[k + 1] / m0.c[k];
    // tops
    std::vector<int> top_row(ng), ntop(ng);
    std::vector<double> scale(ng);
    std::vector<const double *> Gs(ng);
    for (int t = 0; t < ng; ++t) {
        const lap_handle_s &h = *G.hs[ord[t]];
        const int l = h.m.levels;
        top_row[t] = static_cast<int>(G.off[l - 1]) + base[l - 1][t];
        ntop[t] = static_cast<int>(h.m.lev[l - 1].n);
        scale[t] = h.m.c[l - 1];
        Gs[t] = h.M64.G;                                 // the handle's own device copy
    }
    // block ranges
    G.CT = 8;
    const int S = kBThreads / G.CT;
    std::vector<GRange> rows(ng), aggs0(ng);
    for (int t = 0; t < ng; ++t) {
        const int n = n_of[t];
        rows[t] = GRange{base[0][t], base[0][t] + n, nblocks(n, S), 0};
        const HostModel &m = G.hs[ord[t]]->m;
        const int na = m.levels > 1 ? static_cast<int>(m.msp[0].nagg) : 0;
        const int a0 = m.levels > 1 ? base[1][t] : 0;
        aggs0[t] = GRange{a0, a0 + na, nblocks(std::max(na, 1), S), 0};
    }
    LAP_LTRY(G.upload(&G.rp, rp));
    LAP_LTRY(G.upload(&G.ci, ci));
    LAP_LTRY(G.upload(&G.perm, perm));
    LAP_LTRY(G.upload(&G.gid, gid));
    LAP_LTRY(G.upload(&G.n_of, n_of));
    LAP_LTRY(G.upload(&G.top_row, top_row));
    LAP_LTRY(G.upload(&G.ntop, ntop));
    LAP_LTRY(G.upload(&G.scale, scale));
    {
        std::vector<const double *> g2(Gs);
        const double **p = nullptr;
        LAP_LTRY(G.upload(&p, g2));
        G.Gs = p;
    }
    LAP_LTRY(G.upload(&G.rows, rows));
    LAP_LTRY(G.upload(&G.aggs0, aggs0));
    G.seg.assign(nl, nullptr);
    for (int k = 0; k < nl; ++k) LAP_LTRY(G.upload(&G.seg[k], segs[k]));
    LAP_LTRY(upload_prec<double>(G, G.p64, w, inv, lcf));
    if (G.mixed) LAP_LTRY(upload_prec<float>(G, G.p32, w, inv, lcf));
    G.nrhs = G.alloc<int>(G.bufs, static_cast<size_t>(ng));
    G.Bp = G.alloc<double *>(G.bufs, static_cast<size_t>(ng));
    G.Xp = G.alloc<double *>(G.bufs, static_cast<size_t>(ng));
    if (!G.nrhs || !G.Bp || !G.Xp) return LAP_ERR_OOM;
    return LAP_OK;
}

template <typename V> GroupVecs<V> &gvecs(lap_group_s &G);
template <> GroupVecs<double> &gvecs<double>(lap_group_s &G) { return G.v64; }
template <> GroupVecs<float> &gvecs<float>(lap_group_s &G) { return G.v32; }
template <typename V> GroupPrec<V> &gprec(lap_group_s &G);
template <> GroupPrec<double> &gprec<double>(lap_group_s &G) { return G.p64; }
template <> GroupPrec<float> &gprec<float>(lap_group_s &G) { return G.p32; }

template <typename V>
lap_status alloc_gvecs(lap_group_s &G, GroupVecs<V> &v)
{
    const size_t nR = static_cast<size_t>(G.n_all) * G.R, tR = static_cast<size_t>(G.nt_all) * G.R;
    v.x = G.alloc<V>(G.wbufs, nR);
    v.r = G.alloc<V>(G.wbufs, nR);
    v.p = G.alloc<V>(G.wbufs, nR);
    v.q = G.alloc<V>(G.wbufs, nR);
    v.z = G.alloc<V>(G.wbufs, nR);
    v.A = G.alloc<V>(G.wbufs, tR);
    v.Y = G.alloc<V>(G.wbufs, tR);
    v.col = G.alloc<BCol>(G.wbufs, static_cast<size_t>(G.G) * G.R);
    if (!v.x || !v.r || !v.p || !v.q || !v.z || !v.A || !v.Y || !v.col) return LAP_ERR_OOM;
    return LAP_OK;
}

lap_status prepare(lap_group_s &G, int R)
{
    if (G.R == R) return LAP_OK;
    G.drop_work();
    G.R = R;
    G.CT = std::min(R, 32);
    // the block ranges were cut for CT = 8; recut for this width
    const int S = kBThreads / G.CT;
    std::vector<GRange> rows(G.G), aggs0(G.G);
    LAP_GCK(cudaMemcpy(rows.data(), G.rows, sizeof(GRange) * G.G, cudaMemcpyDeviceToHost));
    LAP_GCK(cudaMemcpy(aggs0.data(), G.aggs0, sizeof(GRange) * G.G, cudaMemcpyDeviceToHost));
    for (int t = 0; t < G.G; ++t) {
        rows[t].nb = nblocks(rows[t].hi - rows[t].lo, S);
        aggs0[t].nb = nblocks(std::max(aggs0[t].hi - aggs0[t].lo, 1), S);
    }
    LAP_GCK(cudaMemcpy(G.rows, rows.data(), sizeof(GRange) * G.G, cudaMemcpyHostToDevice));
    LAP_GCK(cudaMemcpy(G.aggs0, aggs0.data(), sizeof(GRange) * G.G, cudaMemcpyHostToDevice));
    const size_t nR = static_cast<size_t>(G.n_all) * R;
    G.Bs = G.alloc<double>(G.wbufs, nR);
    G.x64 = G.alloc<double>(G.wbufs, nR);
    G.r64 = G.alloc<double>(G.wbufs, nR);
    G.means = G.alloc<double>(G.wbufs, static_cast<size_t>(G.G) * R);
    G.part = G.alloc<double>(G.wbufs, static_cast<size_t>(G.G) * kGroupMaxBlocks * 2 * R);
    G.ticket = G.alloc<unsigned>(G.wbufs, static_cast<size_t>(G.G));
    G.col64 = G.alloc<BCol>(G.wbufs, static_cast<size_t>(G.G) * R);
    if (!G.Bs || !G.x64 || !G.r64 || !G.means || !G.part || !G.ticket || !G.col64) return LAP_ERR_OOM;
    LAP_LTRY(alloc_gvecs<double>(G, G.v64));
    if (G.mixed) LAP_LTRY(alloc_gvecs<float>(G, G.v32));
    LAP_GCK(cudaMallocHost(&G.hcol, sizeof(BCol) * G.G * R));
    return LAP_OK;
}

dim3 ggrid(const lap_group_s &G) { return dim3(kGroupMaxBlocks, G.G); }

int egrid(const lap_group_s &G, int64_t rows)
{
    const int S = kBThreads / G.CT;
    const int64_t b = (rows + S - 1) / S;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(b, G.grid_cap)));
}

template <typename V, int MODE>
void gspmm(lap_group_s &G, const V *x, V *y, double *yres, BCol *col)
{
    G.launches += 1;
    kg_spmm<V, MODE><<<ggrid(G), kBThreads, 0, G.s>>>(G.R, G.CT, G.rows, G.rp, G.ci, gprec<V>(G).w, x, y, G.Bs,
                                                        yres, col, G.part, kGroupMaxBlocks, G.ticket);
}

// z = B r for every (graph, column); with update the CG step is fused into
// the finest level.
template <typename V>
void gprecond(lap_group_s &G, GroupVecs<V> &v, bool update)
{
    const int R = G.R, CT = G.CT;
    const size_t RR = static_cast<size_t>(R);
    const cudaStream_t s = G.s;
    if (G.plain) {
        G.launches += 1;
        if (update)
            kg_plain<V, true><<<ggrid(G), kBThreads, 0, s>>>(R, CT, G.rows, v.x, v.r, v.p, v.q, v.col, G.part,
                                                            kGroupMaxBlocks, G.ticket);
        else
            kg_plain<V, false><<<ggrid(G), kBThreads, 0, s>>>(R, CT, G.rows, v.x, v.r, v.p, v.q, v.col, G.part,
                                                             kGroupMaxBlocks, G.ticket);
        return;
    }
    GroupPrec<V> &P = gprec<V>(G);
    const int nl = G.kmax - 1;
    G.launches += 2 * nl + 1;
    if (update)
        kg_up<V, 1><<<ggrid(G), kBThreads, 0, s>>>(G.nagg[0], R, CT, G.aggs0, G.seg[0], P.inv[0], P.lcf[0], v.x,
                                                   v.r, v.p, v.q, v.A, v.A + G.off[1] * RR, (V)G.gamma[0], v.col,
                                                   G.part, kGroupMaxBlocks, G.ticket);
    else
        kg_up<V, 2><<<ggrid(G), kBThreads, 0, s>>>(G.nagg[0], R, CT, G.aggs0, G.seg[0], P.inv[0], P.lcf[0], v.x,
                                                   v.r, v.p, v.q, v.A, v.A + G.off[1] * RR, (V)G.gamma[0], v.col,
                                                   G.part, kGroupMaxBlocks, G.ticket);
    for (int k = 1; k < nl; ++k) {
        V *a = v.A + G.off[k] * RR;
        kg_up<V, 0><<<egrid(G, G.nagg[k]), kBThreads, 0, s>>>(G.nagg[k], R, CT, nullptr, G.seg[k], P.inv[k],
                                                               P.lcf[k], nullptr, a, nullptr, nullptr, a,
                                                               v.A + G.off[k + 1] * RR, (V)G.gamma[k], v.col,
                                                               nullptr, 0, nullptr);
    }
    kg_coarse<V><<<dim3(4, G.G), kBThreads, 0, s>>>(R, G.top_row, G.ntop, G.Gs, G.scale, v.A, v.Y);
    for (int k = nl - 1; k >= 1; --k)
        kg_down<V, false><<<egrid(G, G.nagg[k]), kBThreads, 0, s>>>(
            G.nagg[k], R, CT, nullptr, nullptr, G.seg[k], v.A + G.off[k] * RR, v.Y + G.off[k + 1] * RR,
            v.Y + G.off[k] * RR, V(1), static_cast<V>(G.cc[k]), nullptr, v.col, nullptr, 0, nullptr);
    kg_down<V, true><<<ggrid(G), kBThreads, 0, s>>>(G.nagg[0], R, CT, G.aggs0, G.n_of, G.seg[0], v.A,
                                                    v.Y + G.off[1] * RR, v.z, V(1), V(1), v.r, v.col, G.part,
                                                    kGroupMaxBlocks, G.ticket);
}

template <typename V>
void giteration(lap_group_s &G, GroupVecs<V> &v)
{
    gspmm<V, 0>(G, v.p, v.q, nullptr, v.col);
    gprecond<V>(G, v, true);
    G.launches += 1;
    kg_pupdate<V><<<egrid(G, G.n_all), kBThreads, 0, G.s>>>(G.n_all, G.R, G.CT, G.gid, G.plain ? v.r : v.z, v.p,
                                                             v.col);
}

lap_status gpoll(lap_group_s &G, const BCol *col, std::vector<BCol> &out)
{
    const size_t n = static_cast<size_t>(G.G) * G.R;
    LAP_GCK(cudaMemcpyAsync(G.hcol, col, sizeof(BCol) * n, cudaMemcpyDeviceToHost, G.s));
    LAP_GCK(cudaStreamSynchronize(G.s));
    out.assign(G.hcol, G.hcol + n);
    return LAP_OK;
}

template <typename V>
lap_status giterate(lap_group_s &G, GroupVecs<V> &v, std::vector<BCol> &cols)
{
    if (!v.g) {
        cudaGraph_t graph = nullptr;
        const int64_t l0 = G.launches;
        LAP_GCK(cudaStreamBeginCapture(G.s, cudaStreamCaptureModeThreadLocal));
        for (int i = 0; i < G.opt.check_every; ++i) giteration<V>(G, v);
        cudaError_t e = cudaStreamEndCapture(G.s, &graph);
        G.launches = l0;
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
    const int cap = G.opt.maxit / G.opt.check_every + 4;
    for (int launches = 0; launches <= cap; ++launches) {
        LAP_GCK(cudaGraphLaunch(v.g, G.s));
        G.launches += v.nodes;
        LAP_LTRY(gpoll(G, v.col, cols));
        bool any = false;
        for (const BCol &c : cols) any |= c.flag == kRun;
        if (!any) return LAP_OK;
    }
    return LAP_ERR_BREAKDOWN;
}

lap_status group_solve(lap_group_s &G, const int *nrhs, lap_solve_info *infos)
{
    int maxr = 1;
    for (int t = 0; t < G.G; ++t) maxr = std::max(maxr, nrhs[G.order[t]]);
    const int R = pow2_at_least(maxr);
    LAP_LTRY(prepare(G, R));
    const lap_options &o = G.opt;
    const cudaStream_t s = G.s;
    const int CT = G.CT, ng = G.G;
    std::vector<int> nr_m(ng);
    for (int t = 0; t < ng; ++t) nr_m[t] = nrhs[G.order[t]];
    LAP_GCK(cudaMemcpyAsync(G.nrhs, nr_m.data(), sizeof(int) * ng, cudaMemcpyHostToDevice, s));
    std::vector<BCol> cols;
    std::vector<int> iters(static_cast<size_t>(ng) * R, 0), refs(static_cast<size_t>(ng) * R, 0);
    G.launches += 2;
    kg_gather<<<ggrid(G), kBThreads, 0, s>>>(R, CT, G.rows, G.nrhs, G.perm, (const double *const *)G.Bp, G.Bs,
                                             G.col64, G.part,
                                             kGroupMaxBlocks, G.ticket);
    lap_status result = LAP_OK;
    const size_t NC = static_cast<size_t>(ng) * R;
    if (!G.mixed) {
        auto &v = G.v64;
        kg_center<double><<<ggrid(G), kBThreads, 0, s>>>(R, CT, G.rows, G.nrhs, 1, G.Bs, v.r, v.x, G.col64, v.col,
                                                         o.tol, o.maxit, nullptr, 0.0, G.part, kGroupMaxBlocks,
                                                         G.ticket);
        gprecond<double>(G, v, false);
        G.launches += 1;
        kg_pupdate<double><<<egrid(G, G.n_all), kBThreads, 0, s>>>(G.n_all, R, CT, G.gid, G.plain ? v.r : v.z,
                                                                    v.p, v.col);
        result = giterate<double>(G, v, cols);
        for (size_t c = 0; c < NC; ++c) iters[c] = cols.empty() ? 0 : cols[c].iter;
        gspmm<double, 1>(G, v.x, nullptr, G.r64, v.col);
        LAP_LTRY(gpoll(G, v.col, cols));
        G.launches += 2;
        kg_mean<double><<<ggrid(G), kBThreads, 0, s>>>(R, CT, G.rows, v.x, G.means, G.part, kGroupMaxBlocks,
                                                       G.ticket);
        kg_scatter<double><<<ggrid(G), kBThreads, 0, s>>>(R, CT, G.rows, G.nrhs, G.perm, v.x, G.means, G.Xp);
    } else {
        kg_center<double><<<ggrid(G), kBThreads, 0, s>>>(R, CT, G.rows, G.nrhs, 1, G.Bs, G.r64, G.x64, G.col64,
                                                         G.col64, o.tol, o.maxit, nullptr, 0.0, G.part,
                                                         kGroupMaxBlocks, G.ticket);
        auto &v = G.v32;
        std::vector<BCol> outer;
        for (int ref = 0;; ++ref) {
            if (ref > 0) {
                gspmm<double, 1>(G, G.x64, nullptr, G.r64, G.col64);
                G.launches += 1;
                kg_refine_flags<<<1, 256, 0, s>>>(ng, R, G.nrhs, G.col64, o.tol);
            }
            LAP_LTRY(gpoll(G, G.col64, outer));
            bool any = false;
            for (const BCol &c : outer) any |= c.flag == kRun;
            if (!any || ref >= o.max_refine) break;
            int used = 0;
            for (size_t c = 0; c < NC; ++c) used = std::max(used, iters[c]);
            if (used >= o.maxit) break;
            G.launches += 1;
            kg_center<float><<<ggrid(G), kBThreads, 0, s>>>(R, CT, G.rows, G.nrhs, 0, G.r64, v.r, v.x, G.col64,
                                                            v.col, o.tol, o.maxit - used, G.col64, o.refine_tol,
                                                            G.part, kGroupMaxBlocks, G.ticket);
            gprecond<float>(G, v, false);
            G.launches += 1;
            kg_pupdate<float><<<egrid(G, G.n_all), kBThreads, 0, s>>>(G.n_all, R, CT, G.gid,
                                                                      G.plain ? v.r : v.z, v.p, v.col);
            lap_status it = giterate<float>(G, v, cols);
            if (it != LAP_OK) {
                result = it;
                break;
            }
            for (size_t c = 0; c < NC; ++c)
                if (outer[c].flag == kRun) {
                    iters[c] += cols[c].iter;
                    refs[c] = ref + 1;
                }
            G.launches += 1;
            kb_add<float><<<G.grid_cap, kBThreads, 0, s>>>(static_cast<int64_t>(G.n_all) * R, G.x64, v.x);
        }
        gspmm<double, 1>(G, G.x64, nullptr, G.r64, G.col64);
        LAP_LTRY(gpoll(G, G.col64, cols));
        G.launches += 2;
        kg_mean<double><<<ggrid(G), kBThreads, 0, s>>>(R, CT, G.rows, G.x64, G.means, G.part, kGroupMaxBlocks,
                                                       G.ticket);
        kg_scatter<double><<<ggrid(G), kBThreads, 0, s>>>(R, CT, G.rows, G.nrhs, G.perm, G.x64, G.means, G.Xp);
    }
    LAP_GCK(cudaStreamSynchronize(s));
    if (infos) {
        size_t off = 0;
        std::vector<size_t> first(ng);
        for (int g = 0; g < ng; ++g) {
            first[g] = off;
            off += static_cast<size_t>(nrhs[g]);
        }
        for (int t = 0; t < ng; ++t) {
            const int g = G.order[t];
            for (int c = 0; c < nrhs[g]; ++c) {
                const size_t k = static_cast<size_t>(t) * R + c;
                lap_solve_info &inf = infos[first[g] + c];
                std::memset(&inf, 0, sizeof(inf));
                inf.iterations = iters[k];
                inf.refinements = refs[k];
                inf.relres = cols[k].bnorm > 0.0 ? cols[k].relres : 0.0;
                inf.relres_recurrence = inf.relres;
                inf.status = result != LAP_OK ? result : (inf.relres <= o.tol ? LAP_OK : LAP_ERR_NO_CONVERGENCE);
            }
        }
    }
    return result;
}

}  // namespace
}  // namespace lap

extern "C" lap_status lap_group_create(int32_t ng, const lap_handle *hs, lap_group *out)
{
    using namespace lap;
    if (!out || ng < 1 || !hs) return LAP_ERR_INVALID_ARG;
    *out = nullptr;
    for (int g = 0; g < ng; ++g) {
        if (!hs[g] || hs[g]->host_only) return LAP_ERR_INVALID_ARG;
        const lap_handle_s &h = *hs[g];
        const lap_options &a = h.m.opt, &b = hs[0]->m.opt;
        if (a.prec != LAP_PREC_MSP && a.prec != LAP_PREC_NONE) return LAP_ERR_UNSUPPORTED;
        if (a.prec != b.prec || a.precision != b.precision || h.m.mu != hs[0]->m.mu || h.device != hs[0]->device)
            return LAP_ERR_INVALID_ARG;
        if (h.m.levels < 2) return LAP_ERR_UNSUPPORTED;
    }
    auto G = std::make_unique<lap_group_s>();
    G->G = ng;
    G->hs.assign(hs, hs + ng);
    G->opt = hs[0]->m.opt;
    G->device = hs[0]->device;
    G->grid_cap = hs[0]->grid_cap;
    G->mixed = G->opt.precision == LAP_MIXED;
    G->plain = G->opt.prec == LAP_PREC_NONE;
    if (cudaSetDevice(G->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&G->s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&G->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&G->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        (void)cudaGetLastError();
        return LAP_ERR_CUDA;
    }
    lap_status st = build_group(*G);
    if (st != LAP_OK) return st;
    *out = G.release();
    return LAP_OK;
}

extern "C" lap_status lap_pcg_solve_group(lap_group grp, const int32_t *nrhs, const double *const *d_B,
                                          double *const *d_X, void *stream, lap_solve_info *infos)
{
    using namespace lap;
    if (!grp || !nrhs || !d_B || !d_X) return LAP_ERR_INVALID_ARG;
    lap_group_s &G = *grp;
    int total = 0;
    for (int g = 0; g < G.G; ++g) {
        if (nrhs[g] < 0 || nrhs[g] > 256 || (nrhs[g] > 0 && (!d_B[g] || !d_X[g]))) return LAP_ERR_INVALID_ARG;
        total += nrhs[g];
    }
    if (total == 0) return LAP_OK;
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t l0 = G.launches;
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    LAP_GCK(cudaSetDevice(G.device));
    // the caller's pointers in merged order
    std::vector<const double *> B(G.G);
    std::vector<double *> X(G.G);
    for (int t = 0; t < G.G; ++t) {
        B[t] = d_B[G.order[t]];
        X[t] = d_X[G.order[t]];
    }
    LAP_GCK(cudaEventRecord(G.ev_in, user));
    LAP_GCK(cudaStreamWaitEvent(G.s, G.ev_in, 0));
    LAP_GCK(cudaMemcpyAsync(G.Bp, B.data(), sizeof(double *) * G.G, cudaMemcpyHostToDevice, G.s));
    LAP_GCK(cudaMemcpyAsync(G.Xp, X.data(), sizeof(double *) * G.G, cudaMemcpyHostToDevice, G.s));
    lap_status st = group_solve(G, nrhs, infos);
    LAP_GCK(cudaEventRecord(G.ev_out, G.s));
    LAP_GCK(cudaStreamWaitEvent(user, G.ev_out, 0));
    if (infos) {
        const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int c = 0; c < total; ++c) {
            infos[c].seconds = secs;
            infos[c].kernel_launches = static_cast<int32_t>(G.launches - l0);
        }
    }
    return st;
}

extern "C" void lap_group_destroy(lap_group grp)
{
    if (!grp) return;
    cudaSetDevice(grp->device);
    delete grp;
}
