// Setup on the device: the aggregation hierarchy with the handshake matching
// (Section 2.2, its data-parallel variant) and the Laplacian of PEGP's
// positive subgraph H (Section 3.2), bit-exact with the host build of
// setup.cpp.  Two rules make the results equal bit for bit:
//   * every floating-point sum is taken by one thread, from 0.0, in the order
//     the host takes it (a vertex's CSR entries in order);
//   * where the host groups values before summing (coarse weights by
//     aggregate pair, H's even-distance weights by ancestor) the device sorts
//     (key, value) pairs with a stable LSD radix sort of its own, so that the
//     values of one key stay in the host's order, and sums each run.
// The tree order, the sparsifier's elimination data and the level-1
// Laplacian stay on the host (finish_model): they are linear passes.
//
// Data layout: every level's adjacency is CSR (int64 row pointers, int32
// columns, FP64 weights) in the hierarchy's own numbering; sort keys are
// row * ncols + col in 64 bits, values the FP64 weights' bit patterns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <utility>
#include <vector>

#include "lap_internal.h"

namespace lap {
namespace {

constexpr int kTpb = 256;

lap_status cu(cudaError_t e)
{
    if (e == cudaSuccess) return LAP_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? LAP_ERR_OOM : LAP_ERR_CUDA;
}

#define SD_TRY(x)                         \
    do {                                  \
        lap_status s_ = (x);              \
        if (s_ != LAP_OK) return s_;      \
    } while (0)
#define SD_CU(x) SD_TRY(cu(x))
#define SD_LAUNCHED() SD_CU(cudaGetLastError())

unsigned blocks(int64_t n, int per_block = kTpb)
{
    return static_cast<unsigned>((n + per_block - 1) / per_block);
}

// Device buffer from the library's allocator, freed on destruction.
struct Buf {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    Buf() = default;
    Buf(const Buf &) = delete;
    Buf &operator=(const Buf &) = delete;
    Buf(Buf &&o) noexcept : p(o.p), s(o.s) { o.p = nullptr; }
    ~Buf() { release(); }
    void release()
    {
        if (p) dev_free(p, s);
        p = nullptr;
    }
    lap_status alloc(size_t bytes, cudaStream_t st)
    {
        release();
        s = st;
        p = dev_alloc(bytes > 0 ? bytes : 16, st);
        return p ? LAP_OK : LAP_ERR_OOM;
    }
    template <typename T> lap_status alloc_n(int64_t n, cudaStream_t st)
    {
        return alloc(static_cast<size_t>(n > 0 ? n : 1) * sizeof(T), st);
    }
    template <typename T> T *as() const { return static_cast<T *>(p); }
};

void swap_bufs(Buf &a, Buf &b)
{
    std::swap(a.p, b.p);
    std::swap(a.s, b.s);
}

template <typename T> lap_status download(std::vector<T> &dst, const T *src, int64_t n, cudaStream_t s)
{
    dst.resize(static_cast<size_t>(n));
    if (n > 0) SD_CU(cudaMemcpyAsync(dst.data(), src, sizeof(T) * n, cudaMemcpyDeviceToHost, s));
    return LAP_OK;
}

template <typename T> lap_status upload(Buf &dst, const T *src, int64_t n, cudaStream_t s)
{
    SD_TRY(dst.alloc_n<T>(n, s));
    if (n > 0) SD_CU(cudaMemcpyAsync(dst.p, src, sizeof(T) * n, cudaMemcpyHostToDevice, s));
    return LAP_OK;
}

lap_status read_scalar(int64_t *dst, const int64_t *src, cudaStream_t s)
{
    SD_CU(cudaMemcpyAsync(dst, src, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SD_CU(cudaStreamSynchronize(s));
    return LAP_OK;
}

// ---------------------------------------------------------------------------
// Exclusive scan of int64 counts: out[0..n], out[n] = the total.  Tiles of
// 2048 entries (8 per thread) scanned in shared memory, the tile totals
// scanned recursively, then added back.
// ---------------------------------------------------------------------------
constexpr int kScanPer = 8, kScanTile = kTpb * kScanPer;

__global__ void __launch_bounds__(kTpb) k_scan_tiles(const int64_t *in, int64_t *out, int64_t n,
                                                     int64_t *tile_total)
{
    __shared__ int64_t wsum[kTpb / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + threadIdx.x * kScanPer;
    int64_t v[kScanPer], s = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        v[i] = base + i < n ? in[base + i] : 0;
        s += v[i];
    }
    int64_t x = s;                                     // inclusive over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t t = lane < kTpb / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kTpb / 32) wsum[lane] = t;
    }
    __syncthreads();
    int64_t run = x - s + (wid > 0 ? wsum[wid - 1] : 0);
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == kTpb - 1) tile_total[blockIdx.x] = run;
}

__global__ void k_scan_add(int64_t *out, int64_t n, const int64_t *tile_offset)
{
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + threadIdx.x * kScanPer;
    const int64_t add = tile_offset[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanPer; ++i)
        if (base + i < n) out[base + i] += add;
}

__global__ void k_scan_total(const int64_t *in, int64_t *out, int64_t n)
{
    out[n] = out[n - 1] + in[n - 1];
}

// in and out distinct; out has n + 1 entries
lap_status exclusive_scan(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cu(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    const int64_t nt = (n + kScanTile - 1) / kScanTile;
    Buf tot, off;
    SD_TRY(tot.alloc_n<int64_t>(nt, s));
    k_scan_tiles<<<static_cast<unsigned>(nt), kTpb, 0, s>>>(in, out, n, tot.as<int64_t>());
    SD_LAUNCHED();
    if (nt > 1) {
        SD_TRY(off.alloc_n<int64_t>(nt + 1, s));
        SD_TRY(exclusive_scan(tot.as<int64_t>(), off.as<int64_t>(), nt, s));
        k_scan_add<<<static_cast<unsigned>(nt), kTpb, 0, s>>>(out, n, off.as<int64_t>());
        SD_LAUNCHED();
    }
    k_scan_total<<<1, 1, 0, s>>>(in, out, n);
    SD_LAUNCHED();
    return LAP_OK;
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (uint64 key, uint64 value) pairs, 8 bits a pass.
// A pass: per-tile digit counts (tiles of 4096 pairs), one exclusive scan of
// the counts laid out digit-major (all tiles' digit-0 counts, then digit 1,
// ...), and a scatter in which every pair goes to its digit's offset plus the
// number of earlier pairs of its tile with the same digit.  Warp w of a tile
// holds pairs [512 w, 512 w + 512) in 16 rounds of 32 consecutive pairs, so
// "earlier" = earlier warp, earlier round, or lower lane: the order is kept.
// ---------------------------------------------------------------------------
constexpr int kRsItems = 16, kRsTile = kTpb * kRsItems, kRsWarps = kTpb / 32;

__global__ void __launch_bounds__(kTpb) k_rs_hist(const uint64_t *key, int64_t n, int shift,
                                                  int64_t ntiles, int64_t *cnt)
{
    __shared__ int c[256];
    c[threadIdx.x] = 0;
    __syncthreads();
    const int64_t t0 = static_cast<int64_t>(blockIdx.x) * kRsTile;
    for (int i = 0; i < kRsItems; ++i) {
        const int64_t e = t0 + static_cast<int64_t>(i) * kTpb + threadIdx.x;
        if (e < n) atomicAdd(&c[(key[e] >> shift) & 255u], 1);
    }
    __syncthreads();
    cnt[static_cast<int64_t>(threadIdx.x) * ntiles + blockIdx.x] = c[threadIdx.x];
}

__global__ void __launch_bounds__(kTpb) k_rs_scatter(const uint64_t *key, const uint64_t *val,
                                                     uint64_t *okey, uint64_t *oval, int64_t n, int shift,
                                                     int64_t ntiles, const int64_t *offset)
{
    __shared__ int wc[kRsWarps][256];
    __shared__ int64_t base[256];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) wc[w][threadIdx.x] = 0;
    base[threadIdx.x] = offset[static_cast<int64_t>(threadIdx.x) * ntiles + blockIdx.x];
    __syncthreads();
    const int64_t w0 = static_cast<int64_t>(blockIdx.x) * kRsTile + wid * (32 * kRsItems);
    uint64_t k[kRsItems];
    int d[kRsItems];
    // counts of each digit in each warp's part of the tile
#pragma unroll
    for (int i = 0; i < kRsItems; ++i) {
        const int64_t e = w0 + i * 32 + lane;
        k[i] = e < n ? key[e] : 0;
        d[i] = e < n ? static_cast<int>((k[i] >> shift) & 255u) : 256;
        const unsigned m = __match_any_sync(0xffffffffu, d[i]);
        if (d[i] < 256 && (m & below) == 0) wc[wid][d[i]] += __popc(m);
        __syncwarp();
    }
    __syncthreads();
    {   // exclusive prefix over the warps, per digit
        int run = 0;
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) {
            const int c = wc[w][threadIdx.x];
            wc[w][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kRsItems; ++i) {
        const int64_t e = w0 + i * 32 + lane;
        const unsigned m = __match_any_sync(0xffffffffu, d[i]);
        if (d[i] < 256) {
            const int64_t pos = base[d[i]] + wc[wid][d[i]] + __popc(m & below);
            okey[pos] = k[i];
            oval[pos] = val[e];
        }
        __syncwarp();
        if (d[i] < 256 && (m & below) == 0) wc[wid][d[i]] += __popc(m);
        __syncwarp();
    }
}

int bit_length(uint64_t x)
{
    int b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

// Sorts (key, val) by the low `bits` bits of key, stably; the result is left
// in (key, val) (the buffers may be swapped with the spare ones).
lap_status radix_sort(Buf &key, Buf &val, Buf &key2, Buf &val2, int64_t n, int bits, cudaStream_t s)
{
    if (n <= 1 || bits <= 0) return LAP_OK;
    const int64_t ntiles = (n + kRsTile - 1) / kRsTile;
    Buf cnt, off;
    SD_TRY(cnt.alloc_n<int64_t>(256 * ntiles, s));
    SD_TRY(off.alloc_n<int64_t>(256 * ntiles + 1, s));
    for (int shift = 0; shift < bits; shift += 8) {
        k_rs_hist<<<static_cast<unsigned>(ntiles), kTpb, 0, s>>>(key.as<uint64_t>(), n, shift, ntiles,
                                                                 cnt.as<int64_t>());
        SD_LAUNCHED();
        SD_TRY(exclusive_scan(cnt.as<int64_t>(), off.as<int64_t>(), 256 * ntiles, s));
        k_rs_scatter<<<static_cast<unsigned>(ntiles), kTpb, 0, s>>>(
            key.as<uint64_t>(), val.as<uint64_t>(), key2.as<uint64_t>(), val2.as<uint64_t>(), n, shift, ntiles,
            off.as<int64_t>());
        SD_LAUNCHED();
        swap_bufs(key, key2);
        swap_bufs(val, val2);
    }
    return LAP_OK;
}

// ---------------------------------------------------------------------------
// Hierarchy kernels (one thread per vertex of the level)
// ---------------------------------------------------------------------------
__global__ void k_degrees(int64_t n, const int64_t *rp, const double *w, double *deg)
{
    const int64_t u = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (u >= n) return;
    double d = 0.0;
    for (int64_t p = rp[u]; p < rp[u + 1]; ++p) d += w[p];
    deg[u] = d;
}

// Heaviest neighbour of u (ties to the smaller id), among the unmatched ones
// when free_only; -1 if there is none.
__device__ int heaviest(int64_t u, const int64_t *rp, const int *ci, const double *w, const int *mate,
                        bool free_only)
{
    int best = -1;
    double bw = 0.0;
    for (int64_t p = rp[u]; p < rp[u + 1]; ++p) {
        const int v = ci[p];
        if (free_only && mate[v] >= 0) continue;
        const double x = w[p];
        if (best < 0 || x > bw || (x == bw && v < best)) {
            best = v;
            bw = x;
        }
    }
    return best;
}

// Matching round, phase 1: every unmatched vertex that still has an unmatched
// neighbour points at its heaviest one.  A vertex without one keeps none for
// good (neighbours are never unmatched again).
__global__ void k_hs_point(int64_t n, const int64_t *rp, const int *ci, const double *w, const int *mate,
                           int *cand, unsigned char *done)
{
    const int64_t u = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (u >= n) return;
    if (mate[u] >= 0 || done[u]) {
        cand[u] = -1;
        return;
    }
    const int c = heaviest(u, rp, ci, w, mate, true);
    cand[u] = c;
    if (c < 0) done[u] = 1;
}

// Phase 2: vertices pointing at each other are matched.
__global__ void k_hs_match(int64_t n, const int *cand, int *mate, unsigned long long *matched)
{
    const int64_t u = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (u >= n || mate[u] >= 0) return;
    const int c = cand[u];
    if (c >= 0 && cand[c] == static_cast<int>(u)) {
        mate[u] = c;
        atomicAdd(matched, 1ull);
    }
}

__global__ void k_pair_flags(int64_t n, const int *mate, int64_t *flag)
{
    const int64_t u = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (u < n) flag[u] = mate[u] > u ? 1 : 0;
}

// Pairs numbered by their smaller end, ascending (id = exclusive scan of the flags).
__global__ void k_pairs(int64_t n, const int *mate, const int64_t *id, int *agg, int *pa, int *pb)
{
    const int64_t u = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (u >= n || mate[u] <= u) return;
    const int a = static_cast<int>(id[u]);
    agg[u] = a;
    agg[mate[u]] = a;
    pa[a] = static_cast<int>(u);
    pb[a] = mate[u];
}

// A leftover joins the aggregate of its heaviest neighbour, which is matched
// (no two unmatched vertices are adjacent once the rounds end).
__global__ void k_leftovers(int64_t n, const int64_t *rp, const int *ci, const double *w, const int *mate,
                            int *agg)
{
    const int64_t u = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (u >= n || mate[u] >= 0) return;
    const int v = heaviest(u, rp, ci, w, mate, false);
    agg[u] = agg[v];
}

// Galerkin coarse graph, step 1: every fine entry (u, v) keyed by its
// aggregate pair (agg u, agg v), in CSR order.
__global__ void k_coarse_keys(int64_t n, const int64_t *rp, const int *ci, const double *w, const int *agg,
                              int64_t nc, uint64_t *key, uint64_t *val)
{
    const int64_t u = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const uint64_t I = static_cast<uint64_t>(agg[u]);
    for (int64_t p = rp[u]; p < rp[u + 1]; ++p) {
        key[p] = I * static_cast<uint64_t>(nc) + static_cast<uint64_t>(agg[ci[p]]);
        val[p] = static_cast<uint64_t>(__double_as_longlong(w[p]));
    }
}

// Heads of the runs of equal keys in sorted pairs; keys with row == col
// (entries inside one aggregate) start no run when drop_diagonal.
__global__ void k_run_heads(int64_t m, const uint64_t *key, uint64_t ncols, bool drop_diagonal, int64_t *head)
{
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const uint64_t k = key[e];
    bool h = e == 0 || key[e - 1] != k;
    if (drop_diagonal && k / ncols == k % ncols) h = false;
    head[e] = h ? 1 : 0;
}

// Sum of each run, in its (stable) order, from 0.0; written compacted with
// its column, and counted in its row.
__global__ void k_coarse_runs(int64_t m, const uint64_t *key, const uint64_t *val, uint64_t nc,
                              const int64_t *head_pos, const int64_t *head, int *cci, double *cw,
                              unsigned long long *rowcnt)
{
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= m || !head[e]) return;
    const uint64_t k = key[e];
    double s = 0.0;
    for (int64_t t = e; t < m && key[t] == k; ++t) s += __longlong_as_double(static_cast<long long>(val[t]));
    const int64_t c = head_pos[e];
    cci[c] = static_cast<int>(k % nc);
    cw[c] = s;
    atomicAdd(&rowcnt[k / nc], 1ull);
}

// out_k(u): weight from u to other aggregates, in CSR order.
__global__ void k_out(int64_t n, const int64_t *rp, const int *ci, const double *w, const int *agg, double *out)
{
    const int64_t u = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int a = agg[u];
    double o = 0.0;
    for (int64_t p = rp[u]; p < rp[u + 1]; ++p)
        if (agg[ci[p]] != a) o += w[p];
    out[u] = o;
}

__global__ void k_u64_to_i64(int64_t n, const unsigned long long *in, int64_t *out)
{
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) out[i] = static_cast<int64_t>(in[i]);
}

// One level of the hierarchy on the device.
struct DevLevel {
    int64_t n = 0, nnz = 0;
    Buf rp, ci, w, agg;
};

// Builds level k+1 from level k (F, device) when the handshake matching
// leaves at least two aggregates; fills the host level's agg, pa, pb, out
// and the coarse host level.  Returns the number of aggregates (0: stop).
lap_status coarsen(DevLevel &F, HostLevel &hF, DevLevel &C, HostLevel &hC, int64_t *nagg_out, cudaStream_t s)
{
    const int64_t n = F.n;
    const unsigned nb = blocks(n);
    Buf mate, cand, done, matched;
    SD_TRY(mate.alloc_n<int>(n, s));
    SD_TRY(cand.alloc_n<int>(n, s));
    SD_TRY(done.alloc_n<unsigned char>(n, s));
    SD_TRY(matched.alloc_n<unsigned long long>(1, s));
    SD_CU(cudaMemsetAsync(mate.p, 0xff, sizeof(int) * n, s));
    SD_CU(cudaMemsetAsync(done.p, 0, n, s));
    unsigned long long hm = 0;
    for (int64_t round = 0; round <= n; ++round) {
        SD_CU(cudaMemsetAsync(matched.p, 0, sizeof(unsigned long long), s));
        k_hs_point<<<nb, kTpb, 0, s>>>(n, F.rp.as<int64_t>(), F.ci.as<int>(), F.w.as<double>(), mate.as<int>(),
                                       cand.as<int>(), done.as<unsigned char>());
        SD_LAUNCHED();
        k_hs_match<<<nb, kTpb, 0, s>>>(n, cand.as<int>(), mate.as<int>(), matched.as<unsigned long long>());
        SD_LAUNCHED();
        SD_CU(cudaMemcpyAsync(&hm, matched.p, sizeof(hm), cudaMemcpyDeviceToHost, s));
        SD_CU(cudaStreamSynchronize(s));
        if (hm == 0) break;
    }
    cand.release();
    done.release();
    Buf flag, id;
    SD_TRY(flag.alloc_n<int64_t>(n, s));
    SD_TRY(id.alloc_n<int64_t>(n + 1, s));
    k_pair_flags<<<nb, kTpb, 0, s>>>(n, mate.as<int>(), flag.as<int64_t>());
    SD_LAUNCHED();
    SD_TRY(exclusive_scan(flag.as<int64_t>(), id.as<int64_t>(), n, s));
    int64_t nc = 0;
    SD_TRY(read_scalar(&nc, id.as<int64_t>() + n, s));
    *nagg_out = nc;
    if (nc < 2) return LAP_OK;
    Buf pa, pb;
    SD_TRY(F.agg.alloc_n<int>(n, s));
    SD_TRY(pa.alloc_n<int>(nc, s));
    SD_TRY(pb.alloc_n<int>(nc, s));
    k_pairs<<<nb, kTpb, 0, s>>>(n, mate.as<int>(), id.as<int64_t>(), F.agg.as<int>(), pa.as<int>(), pb.as<int>());
    SD_LAUNCHED();
    k_leftovers<<<nb, kTpb, 0, s>>>(n, F.rp.as<int64_t>(), F.ci.as<int>(), F.w.as<double>(), mate.as<int>(),
                                    F.agg.as<int>());
    SD_LAUNCHED();
    flag.release();
    id.release();
    mate.release();

    // coarse graph: stable sort of the fine entries by aggregate pair
    const int64_t m = F.nnz;
    Buf key, val, key2, val2;
    SD_TRY(key.alloc_n<uint64_t>(m, s));
    SD_TRY(val.alloc_n<uint64_t>(m, s));
    SD_TRY(key2.alloc_n<uint64_t>(m, s));
    SD_TRY(val2.alloc_n<uint64_t>(m, s));
    k_coarse_keys<<<nb, kTpb, 0, s>>>(n, F.rp.as<int64_t>(), F.ci.as<int>(), F.w.as<double>(), F.agg.as<int>(),
                                      nc, key.as<uint64_t>(), val.as<uint64_t>());
    SD_LAUNCHED();
    SD_TRY(radix_sort(key, val, key2, val2, m, bit_length(static_cast<uint64_t>(nc) * nc - 1), s));
    key2.release();
    val2.release();
    Buf head, hpos, rowcnt;
    SD_TRY(head.alloc_n<int64_t>(m, s));
    SD_TRY(hpos.alloc_n<int64_t>(m + 1, s));
    k_run_heads<<<blocks(m), kTpb, 0, s>>>(m, key.as<uint64_t>(), static_cast<uint64_t>(nc), true,
                                           head.as<int64_t>());
    SD_LAUNCHED();
    SD_TRY(exclusive_scan(head.as<int64_t>(), hpos.as<int64_t>(), m, s));
    int64_t cnnz = 0;
    SD_TRY(read_scalar(&cnnz, hpos.as<int64_t>() + m, s));
    C.n = nc;
    C.nnz = cnnz;
    SD_TRY(C.ci.alloc_n<int>(cnnz, s));
    SD_TRY(C.w.alloc_n<double>(cnnz, s));
    SD_TRY(C.rp.alloc_n<int64_t>(nc + 1, s));
    SD_TRY(rowcnt.alloc_n<unsigned long long>(nc, s));
    SD_CU(cudaMemsetAsync(rowcnt.p, 0, sizeof(unsigned long long) * nc, s));
    k_coarse_runs<<<blocks(m), kTpb, 0, s>>>(m, key.as<uint64_t>(), val.as<uint64_t>(), static_cast<uint64_t>(nc),
                                             hpos.as<int64_t>(), head.as<int64_t>(), C.ci.as<int>(),
                                             C.w.as<double>(), rowcnt.as<unsigned long long>());
    SD_LAUNCHED();
    {
        Buf cnt64;
        SD_TRY(cnt64.alloc_n<int64_t>(nc, s));
        k_u64_to_i64<<<blocks(nc), kTpb, 0, s>>>(nc, rowcnt.as<unsigned long long>(), cnt64.as<int64_t>());
        SD_LAUNCHED();
        SD_TRY(exclusive_scan(cnt64.as<int64_t>(), C.rp.as<int64_t>(), nc, s));
        SD_CU(cudaStreamSynchronize(s));
    }
    key.release();
    val.release();

    // degrees of the coarse level, out-weights of the fine level
    Buf cdeg, fout;
    SD_TRY(cdeg.alloc_n<double>(nc, s));
    SD_TRY(fout.alloc_n<double>(n, s));
    k_degrees<<<blocks(nc), kTpb, 0, s>>>(nc, C.rp.as<int64_t>(), C.w.as<double>(), cdeg.as<double>());
    SD_LAUNCHED();
    k_out<<<nb, kTpb, 0, s>>>(n, F.rp.as<int64_t>(), F.ci.as<int>(), F.w.as<double>(), F.agg.as<int>(),
                              fout.as<double>());
    SD_LAUNCHED();
    SD_TRY(download(hF.agg, F.agg.as<int>(), n, s));
    SD_TRY(download(hF.pa, pa.as<int>(), nc, s));
    SD_TRY(download(hF.pb, pb.as<int>(), nc, s));
    SD_TRY(download(hF.out, fout.as<double>(), n, s));
    hC.n = nc;
    SD_TRY(download(hC.rp, C.rp.as<int64_t>(), nc + 1, s));
    SD_TRY(download(hC.ci, C.ci.as<int>(), cnnz, s));
    SD_TRY(download(hC.w, C.w.as<double>(), cnnz, s));
    SD_TRY(download(hC.deg, cdeg.as<double>(), nc, s));
    SD_CU(cudaStreamSynchronize(s));
    return LAP_OK;
}

// ---------------------------------------------------------------------------
// L_H (Section 3.2).  For u on level k and its level-j ancestor a_j (j > k),
// the entry of the expanded operator is (-mu)^(k+j) times (L_k Pi_{k->j})
// (u, J): H keeps the same-level edges (weight mu^(2k) w), the ancestor edges
// at odd distance j - k with out_{k->j}(u) > 0 (weight mu^(k+j) out), and at
// even distance the edges to every other level-j vertex J that u's
// neighbours reach (weight mu^(k+j) times the summed weight of u's entries
// into J's subtree).  Indices are 0-based levels; expanded vertices are
// numbered in tree order, x(k, u) = offset_k + pos_k(u).
// ---------------------------------------------------------------------------
struct PegpLevels {
    int l = 0;
    int64_t nt = 0;
    const int *const *agg = nullptr;     // [l - 1] device pointers
    const int *const *pos = nullptr;     // [l]
    const int64_t *offset = nullptr;     // [l + 1]
    const double *mpow = nullptr;        // [2 l + 2], mu^t by repeated products
};

// Per vertex u of level k: counts of its same-level and ancestor edges (E)
// and of its even-distance entries (T); with `fill`, also writes them at the
// scanned offsets, the entries in (entry, level) order.
template <bool FILL>
__global__ void k_pegp_vertex(PegpLevels P, int k, int64_t n, const int64_t *rp, const int *ci, const double *w,
                              int64_t *ecnt, int64_t *tcnt, const int64_t *eoff, const int64_t *toff,
                              uint64_t *ekey, uint64_t *eval, uint64_t *tkey, uint64_t *tval)
{
    const int64_t u = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int l = P.l;
    const uint64_t nt = static_cast<uint64_t>(P.nt);
    int anc[LAP_MAX_LEVELS];
    double out[LAP_MAX_LEVELS];
    anc[k] = static_cast<int>(u);
    for (int j = k + 1; j < l; ++j) {
        anc[j] = P.agg[j - 1][anc[j - 1]];
        out[j] = 0.0;
    }
    const int64_t g = P.offset[k] + u;                 // slot of u in the count arrays
    const uint64_t xu = static_cast<uint64_t>(P.offset[k] + P.pos[k][u]);
    int64_t ne = 0, ntup = 0;
    const int64_t e0 = FILL ? eoff[g] : 0, t0 = FILL ? toff[g] : 0;
    for (int64_t p = rp[u]; p < rp[u + 1]; ++p) {
        const int v = ci[p];
        const double wq = w[p];
        if (v > u) {
            if (FILL) {
                const uint64_t xv = static_cast<uint64_t>(P.offset[k] + P.pos[k][v]);
                ekey[e0 + ne] = xu * nt + xv;
                eval[e0 + ne] = static_cast<uint64_t>(__double_as_longlong(P.mpow[2 * k] * wq));
            }
            ++ne;
        }
        int a = v;
        for (int j = k + 1; j < l; ++j) {
            a = P.agg[j - 1][a];
            if (a == anc[j]) continue;
            if ((j - k) & 1) {
                out[j] += wq;
            } else {
                if (FILL) {
                    tkey[t0 + ntup] = xu * nt + static_cast<uint64_t>(P.offset[j] + P.pos[j][a]);
                    tval[t0 + ntup] = static_cast<uint64_t>(__double_as_longlong(wq));
                }
                ++ntup;
            }
        }
    }
    for (int j = k + 1; j < l; j += 2) {
        if (!(out[j] > 0.0)) continue;
        if (FILL) {
            ekey[e0 + ne] = xu * nt + static_cast<uint64_t>(P.offset[j] + P.pos[j][anc[j]]);
            eval[e0 + ne] = static_cast<uint64_t>(__double_as_longlong(P.mpow[k + j] * out[j]));
        }
        ++ne;
    }
    if (!FILL) {
        ecnt[g] = ne;
        tcnt[g] = ntup;
    }
}

__device__ int level_of(const int64_t *offset, int l, int64_t x)
{
    int lo = 0, hi = l - 1;                            // offset[lo] <= x < offset[hi + 1]
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (offset[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Even-distance edges: each run of equal (row, col) entries summed in order,
// then scaled by mu^(k+j); appended after the first `base` edges.
__global__ void k_pegp_runs(PegpLevels P, int64_t m, const uint64_t *key, const uint64_t *val,
                            const int64_t *head, const int64_t *hpos, int64_t base, uint64_t *ekey,
                            uint64_t *eval)
{
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= m || !head[e]) return;
    const uint64_t k = key[e];
    double s = 0.0;
    for (int64_t t = e; t < m && key[t] == k; ++t) s += __longlong_as_double(static_cast<long long>(val[t]));
    const uint64_t nt = static_cast<uint64_t>(P.nt);
    const int kr = level_of(P.offset, P.l, static_cast<int64_t>(k / nt));
    const int kc = level_of(P.offset, P.l, static_cast<int64_t>(k % nt));
    const int64_t c = base + hpos[e];
    ekey[c] = k;
    eval[c] = static_cast<uint64_t>(__double_as_longlong(P.mpow[kr + kc] * s));
}

// Both directions of every edge.
__global__ void k_directed(int64_t ne, uint64_t nt, const uint64_t *ekey, const uint64_t *eval, uint64_t *dkey,
                           uint64_t *dval)
{
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const uint64_t k = ekey[e];
    dkey[2 * e] = k;
    dkey[2 * e + 1] = (k % nt) * nt + k / nt;
    dval[2 * e] = dval[2 * e + 1] = eval[e];
}

__global__ void k_csr_split(int64_t m, uint64_t nt, const uint64_t *key, int *ci, unsigned long long *rowcnt)
{
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= m) return;
    ci[e] = static_cast<int>(key[e] % nt);
    atomicAdd(&rowcnt[key[e] / nt], 1ull);
}

lap_status device_pegp(HostModel &m, std::vector<DevLevel> &dl, cudaStream_t s)
{
    const int l = m.levels;
    const int64_t nt = m.offset[l];
    // level tables on the device
    std::vector<Buf> pos(static_cast<size_t>(l));
    std::vector<const int *> hagg(static_cast<size_t>(l > 1 ? l - 1 : 1), nullptr), hpos(static_cast<size_t>(l));
    for (int k = 0; k < l; ++k) {
        SD_TRY(upload(pos[k], m.lev[k].pos.data(), m.lev[k].n, s));
        hpos[k] = pos[k].as<int>();
        if (k + 1 < l) hagg[k] = dl[k].agg.as<int>();
    }
    std::vector<double> mpow(static_cast<size_t>(2 * l + 2), 1.0);
    for (size_t t = 1; t < mpow.size(); ++t) mpow[t] = mpow[t - 1] * m.mu;
    Buf dagg, dpos, doff, dmpow;
    SD_TRY(upload(dagg, hagg.data(), static_cast<int64_t>(hagg.size()), s));
    SD_TRY(upload(dpos, hpos.data(), l, s));
    SD_TRY(upload(doff, m.offset.data(), l + 1, s));
    SD_TRY(upload(dmpow, mpow.data(), static_cast<int64_t>(mpow.size()), s));
    PegpLevels P;
    P.l = l;
    P.nt = nt;
    P.agg = dagg.as<const int *>();
    P.pos = dpos.as<const int *>();
    P.offset = doff.as<int64_t>();
    P.mpow = dmpow.as<double>();

    // counts, offsets, then the edges and the even-distance entries
    Buf ecnt, tcnt, eoff, toff;
    SD_TRY(ecnt.alloc_n<int64_t>(nt, s));
    SD_TRY(tcnt.alloc_n<int64_t>(nt, s));
    SD_TRY(eoff.alloc_n<int64_t>(nt + 1, s));
    SD_TRY(toff.alloc_n<int64_t>(nt + 1, s));
    for (int k = 0; k < l; ++k) {
        const DevLevel &L = dl[k];
        k_pegp_vertex<false><<<blocks(L.n), kTpb, 0, s>>>(P, k, L.n, L.rp.as<int64_t>(), L.ci.as<int>(),
                                                          L.w.as<double>(), ecnt.as<int64_t>(), tcnt.as<int64_t>(),
                                                          nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
        SD_LAUNCHED();
    }
    SD_TRY(exclusive_scan(ecnt.as<int64_t>(), eoff.as<int64_t>(), nt, s));
    SD_TRY(exclusive_scan(tcnt.as<int64_t>(), toff.as<int64_t>(), nt, s));
    int64_t ne1 = 0, ntup = 0;
    SD_TRY(read_scalar(&ne1, eoff.as<int64_t>() + nt, s));
    SD_TRY(read_scalar(&ntup, toff.as<int64_t>() + nt, s));
    ecnt.release();
    tcnt.release();
    Buf ekey, eval, tkey, tval;
    SD_TRY(ekey.alloc_n<uint64_t>(ne1 + ntup, s));
    SD_TRY(eval.alloc_n<uint64_t>(ne1 + ntup, s));
    SD_TRY(tkey.alloc_n<uint64_t>(ntup, s));
    SD_TRY(tval.alloc_n<uint64_t>(ntup, s));
    for (int k = 0; k < l; ++k) {
        const DevLevel &L = dl[k];
        k_pegp_vertex<true><<<blocks(L.n), kTpb, 0, s>>>(
            P, k, L.n, L.rp.as<int64_t>(), L.ci.as<int>(), L.w.as<double>(), nullptr, nullptr, eoff.as<int64_t>(),
            toff.as<int64_t>(), ekey.as<uint64_t>(), eval.as<uint64_t>(), tkey.as<uint64_t>(), tval.as<uint64_t>());
        SD_LAUNCHED();
    }
    eoff.release();
    toff.release();
    const int key_bits = bit_length(static_cast<uint64_t>(nt) * static_cast<uint64_t>(nt) - 1);
    int64_t ne = ne1;
    if (ntup > 0) {
        Buf tkey2, tval2, head, hpos2;
        SD_TRY(tkey2.alloc_n<uint64_t>(ntup, s));
        SD_TRY(tval2.alloc_n<uint64_t>(ntup, s));
        SD_TRY(radix_sort(tkey, tval, tkey2, tval2, ntup, key_bits, s));
        tkey2.release();
        tval2.release();
        SD_TRY(head.alloc_n<int64_t>(ntup, s));
        SD_TRY(hpos2.alloc_n<int64_t>(ntup + 1, s));
        k_run_heads<<<blocks(ntup), kTpb, 0, s>>>(ntup, tkey.as<uint64_t>(), static_cast<uint64_t>(nt), false,
                                                  head.as<int64_t>());
        SD_LAUNCHED();
        SD_TRY(exclusive_scan(head.as<int64_t>(), hpos2.as<int64_t>(), ntup, s));
        int64_t ne2 = 0;
        SD_TRY(read_scalar(&ne2, hpos2.as<int64_t>() + ntup, s));
        k_pegp_runs<<<blocks(ntup), kTpb, 0, s>>>(P, ntup, tkey.as<uint64_t>(), tval.as<uint64_t>(),
                                                  head.as<int64_t>(), hpos2.as<int64_t>(), ne1, ekey.as<uint64_t>(),
                                                  eval.as<uint64_t>());
        SD_LAUNCHED();
        ne += ne2;
        SD_CU(cudaStreamSynchronize(s));
    }
    tkey.release();
    tval.release();

    // symmetric CSR: both directions, sorted by (row, column)
    const int64_t nd = 2 * ne;
    Buf dkey, dval, dkey2, dval2;
    SD_TRY(dkey.alloc_n<uint64_t>(nd, s));
    SD_TRY(dval.alloc_n<uint64_t>(nd, s));
    k_directed<<<blocks(ne), kTpb, 0, s>>>(ne, static_cast<uint64_t>(nt), ekey.as<uint64_t>(), eval.as<uint64_t>(),
                                           dkey.as<uint64_t>(), dval.as<uint64_t>());
    SD_LAUNCHED();
    SD_CU(cudaStreamSynchronize(s));
    ekey.release();
    eval.release();
    SD_TRY(dkey2.alloc_n<uint64_t>(nd, s));
    SD_TRY(dval2.alloc_n<uint64_t>(nd, s));
    SD_TRY(radix_sort(dkey, dval, dkey2, dval2, nd, key_bits, s));
    dkey2.release();
    dval2.release();
    Buf hci, rowcnt, cnt64, hrp, hdiag;
    SD_TRY(hci.alloc_n<int>(nd, s));
    SD_TRY(rowcnt.alloc_n<unsigned long long>(nt, s));
    SD_TRY(cnt64.alloc_n<int64_t>(nt, s));
    SD_TRY(hrp.alloc_n<int64_t>(nt + 1, s));
    SD_TRY(hdiag.alloc_n<double>(nt, s));
    SD_CU(cudaMemsetAsync(rowcnt.p, 0, sizeof(unsigned long long) * nt, s));
    k_csr_split<<<blocks(nd), kTpb, 0, s>>>(nd, static_cast<uint64_t>(nt), dkey.as<uint64_t>(), hci.as<int>(),
                                            rowcnt.as<unsigned long long>());
    SD_LAUNCHED();
    k_u64_to_i64<<<blocks(nt), kTpb, 0, s>>>(nt, rowcnt.as<unsigned long long>(), cnt64.as<int64_t>());
    SD_LAUNCHED();
    SD_TRY(exclusive_scan(cnt64.as<int64_t>(), hrp.as<int64_t>(), nt, s));
    // the sorted values are the FP64 weights; the diagonal is each row's sum in column order
    k_degrees<<<blocks(nt), kTpb, 0, s>>>(nt, hrp.as<int64_t>(), dval.as<double>(), hdiag.as<double>());
    SD_LAUNCHED();
    HostCsr &H = m.LH;
    H.n = nt;
    SD_TRY(download(H.rp, hrp.as<int64_t>(), nt + 1, s));
    SD_TRY(download(H.ci, hci.as<int>(), nd, s));
    SD_TRY(download(H.w, dval.as<double>(), nd, s));
    SD_TRY(download(H.diag, hdiag.as<double>(), nt, s));
    SD_CU(cudaStreamSynchronize(s));
    m.has_LH = true;
    return LAP_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
lap_status device_build_model(int64_t n, const int64_t *rp, const int32_t *ci, const double *w, HostModel &m,
                              void *stream)
{
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    const lap_options &opt = m.opt;
    std::vector<DevLevel> dl;
    dl.emplace_back();
    m.lev.clear();
    m.lev.emplace_back();
    {
        DevLevel &D = dl.back();
        HostLevel &L = m.lev.back();
        L.n = n;
        L.rp.assign(rp, rp + n + 1);
        L.ci.assign(ci, ci + rp[n]);
        L.w.assign(w, w + rp[n]);
        D.n = n;
        D.nnz = rp[n];
        SD_TRY(upload(D.rp, rp, n + 1, s));
        SD_TRY(upload(D.ci, ci, D.nnz, s));
        SD_TRY(upload(D.w, w, D.nnz, s));
        Buf deg;
        SD_TRY(deg.alloc_n<double>(n, s));
        k_degrees<<<blocks(n), kTpb, 0, s>>>(n, D.rp.as<int64_t>(), D.w.as<double>(), deg.as<double>());
        SD_LAUNCHED();
        SD_TRY(download(L.deg, deg.as<double>(), n, s));
        SD_CU(cudaStreamSynchronize(s));
    }
    for (int k = 1;; ++k) {
        if (m.lev.back().n <= opt.coarse_max) break;
        if (opt.max_levels && k >= opt.max_levels) break;
        if (k >= LAP_MAX_LEVELS) break;
        DevLevel C;
        HostLevel hC;
        int64_t nc = 0;
        SD_TRY(coarsen(dl.back(), m.lev.back(), C, hC, &nc, s));
        if (nc < 2) {
            HostLevel &F = m.lev.back();
            F.agg.clear();
            F.pa.clear();
            F.pb.clear();
            break;
        }
        dl.push_back(std::move(C));
        m.lev.push_back(std::move(hC));
    }
    SD_TRY(finish_model(m));
    if (opt.prec == LAP_PREC_PEGP_INNER || opt.prec == LAP_PREC_PEGP_EXACT) SD_TRY(device_pegp(m, dl, s));
    return LAP_OK;
}

}  // namespace lap
