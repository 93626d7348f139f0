// Band sweeps: several levels of the sparsifier solve in one launch.
//
// In tree order the descendants of a contiguous range of level-k1 vertices
// form one contiguous range on every level below (each aggregate's members
// are contiguous and aggregates follow their parents' order).  A band covers
// levels [k0, k1); its tiles are runs of consecutive level-k1 vertices, cut at
// setup so that everything a tile touches fits in shared memory.  Setup also
// packs each tile's segments (as tile-local offsets) and elimination
// coefficients of all its levels into one contiguous block, so that one bulk
// (TMA) copy, completing on an mbarrier, brings them in.  The upward kernel
// eliminates level after level -- a block barrier between levels instead of
// a kernel launch, one warp alone on the small top levels -- and stores the
// deltas of all levels in a tile-packed scratch block, which the downward
// kernel brings back with one more bulk copy.  A tile whose single subtree is
// too large (a hub aggregate) runs the same steps in place in global memory.
#pragma once

#include <cstdint>

#include "kernels.cuh"
#include "lap_internal.h"

namespace lap {

constexpr int kBandThreads = 512;
constexpr int kBandSmemBytes = 96 * 1024;      // shared memory per tile (two tiles per SM)
constexpr int kBandWarpAggs = 64;              // levels with at most this many aggregates: one warp

// Per tile: packed coefficient block (byte offset, bytes, bytes of its
// segment prefix; cbytes < 0: the tile runs in global memory) and the byte
// offset of its delta block in the scratch.
struct BandRec {
    long long cb, ds;
    int cbytes, sbytes;
};

template <typename V> struct BandLevel {
    const int *seg;           // level-k aggregates' member ranges (tree order)
    const V *inv;             // pair coefficients, 4 per aggregate
    const V *lcf;             // leftover coefficients, 3 per leftover
    int64_t off;              // expanded offset of level k
    V gamma;                  // restriction factor to level k + 1
    V dcoef;                  // downward: out = pc * parent + dcoef * delta
};

template <typename V> struct BandParams {
    int nlev;                 // k1 - k0 levels
    int ntiles;
    int smem;                 // shared-memory bytes of a launch (kBandSmemBytes)
    int grid_up, grid_down;   // blocks: the tiles, at most what stays resident
    const int *tstart;        // [(ntiles + 1) * (nlev + 1)]: first index of tile t on level k0 + j
    const BandRec *rec;       // [ntiles]
    const unsigned char *coef;  // packed segments and coefficients of every tile
    V *scratch;               // packed deltas of every tile (written up, read down)
    int64_t off_top;          // expanded offset of level k1
    V pc;                     // downward parent coefficient
    // expanded-space CG fused into the sweep (k_band_up MODE 3, k_band_down
    // XRED): first band (level k0 = 0 taken from r), offsets (in doubles)
    // of this band's per-block partial pairs in the reduction scratch: up
    // (||r||^2, sum r) and, for bands above the first, down (sum z, r.z);
    // the first band's down pass sums its blocks through red_gs and then the
    // xred_n pairs from xred_base (the tail's, then the upper bands')
    int first;
    int red_up, red_dn, red_gs, xred_base, xred_n;
    BandLevel<V> lev[kBandMaxLevels];
};

// ---------------------------------------------------------------------------
// Bulk copies global -> shared (cp.async.bulk, completion counted in bytes on
// an mbarrier).  Source, destination and size must be multiples of 16 bytes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// order this thread's earlier shared-memory accesses before later bulk copies
__device__ __forceinline__ void fence_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    if (bytes == 0) return;
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Wait for the phase with the given parity; gives up after about a second
// (2^31 cycles) and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > (1ll << 31)) return false;
    }
}

__device__ __forceinline__ int r16(int x) { return (x + 15) & ~15; }

// A range of `count` elements of `esize` bytes starting at element `first`
// of the 16-byte aligned array `base`, rounded out to 16 bytes: its aligned
// source, its byte count, and the offset of element `first` in the copy.
struct Span {
    const unsigned char *src;
    int bytes, head;
};

__device__ __forceinline__ Span span(const void *base, int64_t first, int count, int esize)
{
    const int64_t b0 = first * esize;
    Span s;
    s.head = static_cast<int>(b0 & 15);
    s.src = static_cast<const unsigned char *>(base) + (b0 - s.head);
    s.bytes = count > 0 ? r16(s.head + count * esize) : 0;
    return s;
}

// Tile t: first indices and counts per level, its record, the shared-memory
// offsets of each level's values, segments and coefficients, and the first
// level handled by one warp alone.
struct BandTile {
    int st[kBandMaxLevels + 1];
    int cnt[kBandMaxLevels + 1];
    int vs[kBandMaxLevels + 1];     // values of level j (byte offset of element 0)
    int ss[kBandMaxLevels];         // segments of level j (tile-local member offsets)
    int is[kBandMaxLevels];         // pair coefficients of level j
    int ls[kBandMaxLevels];         // leftover coefficients of level j
    int xs[kBandMaxLevels + 1];     // downward: start of each copied region
    int rsm;                        // downward, finest: r of level 0 (byte offset of element 0)
    int jw;                         // levels jw.. have at most kBandWarpAggs aggregates
    BandRec rec;
};

template <typename V>
__device__ __forceinline__ void band_load_tile(const BandParams<V> &P, int t, BandTile &T)
{
    const int L = P.nlev, i = threadIdx.x;
    if (i <= L) {
        const int a = P.tstart[(size_t)t * (L + 1) + i];
        T.st[i] = a;
        T.cnt[i] = P.tstart[(size_t)(t + 1) * (L + 1) + i] - a;
    }
    if (i == 32) T.rec = P.rec[t];
}

// Offsets within the packed coefficient block: segments of every level, then
// pair coefficients of every level, then leftover coefficients (thread 0).
template <typename V>
__device__ __forceinline__ void band_coef_offsets(int L, BandTile &T)
{
    int s = 0, c4 = 0;
    for (int j = 0; j < L; ++j) {
        T.ss[j] = 4 * s;
        s += T.cnt[j + 1] + 1;
    }
    const int seg_bytes = r16(4 * s);
    for (int j = 0; j < L; ++j) {
        T.is[j] = seg_bytes + (int)sizeof(V) * c4;
        c4 += 4 * T.cnt[j + 1];
    }
    int c3 = c4;
    for (int j = 0; j < L; ++j) {
        T.ls[j] = seg_bytes + (int)sizeof(V) * c3;
        c3 += 3 * (T.cnt[j] - 2 * T.cnt[j + 1]);
    }
    int jw = L;
    while (jw > 0 && T.cnt[jw] <= kBandWarpAggs) --jw;
    T.jw = jw;
}

// One level of the upward elimination of a staged tile, by threads
// [tid0, tid0 + nthr).
// SMEMF: the right-hand side added on restriction is the staged value of the
// next level itself (a_{j+1} = gamma sum + f_{j+1} in place); else F (global,
// optional) at the next level's expanded indices.
template <typename V, bool SMEMF = false>
__device__ __forceinline__ void band_up_level(const BandParams<V> &P, const BandTile &T, unsigned char *sm, int j,
                                              const V *F, int tid0, int nthr)
{
    const int64_t onext = j + 1 < P.nlev ? P.lev[j + 1].off : P.off_top;
    V *an = reinterpret_cast<V *>(sm + T.vs[j + 1]);
    elim_level(reinterpret_cast<V *>(sm + T.vs[j]), an, reinterpret_cast<const int *>(sm + T.ss[j]), 0,
               reinterpret_cast<const V *>(sm + T.is[j]), reinterpret_cast<const V *>(sm + T.ls[j]),
               P.lev[j].gamma, SMEMF ? an : F, SMEMF ? 0 : onext + T.st[j + 1], T.cnt[j + 1], tid0, nthr);
}

// Expanded index of element 0 of level j of tile T (j = nlev: the band's top).
template <typename V>
__device__ __forceinline__ int64_t band_level_base(const BandParams<V> &P, const BandTile &T, int j)
{
    return (j < P.nlev ? P.lev[j].off : P.off_top) + T.st[j];
}

// CG step x += alpha p, r -= alpha q on `cnt` consecutive expanded entries
// from g0, the updated r also written to dst (shared or global); adds
// ||r||^2 and sum r (groups of four in V, then FP64).
template <typename V>
__device__ __forceinline__ void band_cg_step(int64_t g0, int cnt, V al, V *__restrict__ x, V *__restrict__ r,
                                             const V *__restrict__ p, const V *__restrict__ q, V *dst,
                                             double &rr, double &rs)
{
    constexpr int G = sizeof(V) == 4 ? 4 : 2;      // elements in flight per thread
    for (int i0 = threadIdx.x; i0 < cnt; i0 += G * kBandThreads) {
        V xv[G], pv[G], qv[G], rv[G];
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const int i = i0 + k * kBandThreads;
            if (i < cnt) {
                const int64_t u = g0 + i;
                xv[k] = x[u];
                pv[k] = p[u];
                qv[k] = q[u];
                rv[k] = r[u];
            }
        }
        V r2 = V(0), r1 = V(0);
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const int i = i0 + k * kBandThreads;
            if (i < cnt) {
                const int64_t u = g0 + i;
                x[u] = xv[k] + al * pv[k];
                const V v = rv[k] - al * qv[k];
                r[u] = v;
                dst[i] = v;
                r2 += v * v;
                r1 += v;
            }
        }
        rr += (double)r2;
        rs += (double)r1;
    }
}

// Upward band: levels k0..k1-1 eliminated (deltas to the scratch, or in place
// in A for a tile in global memory) and the accumulated right-hand side of
// level k1 written to A.
// MODE 1: k0 = 0 with the CG step (x += alpha p, r -= alpha q), a_0 = r,
//         per-block partials of ||r||^2, sum r to part[2 b], part[2 b + 1]
//         (finished by the coarse tail: the convergence test);
// MODE 2: k0 = 0, a_0 = r, the same partials without the step;
// MODE 0: a_{k0} read from A.
// MODE 3: a step of the expanded-space CG (the PEGP inner solve) fused in:
//         x += alpha p, r -= alpha q on every level of the tile (level k0
//         only in the first band, whose a_{k0} = r; the other bands read
//         a_{k0} from A), the updated r staged as the right-hand side added
//         on restriction, per-block partials of ||r||^2, sum r at
//         part[red_up + 2 b] (finished by the coarse tail).
// F (optional, MODE 0): expanded right-hand side added on restriction (a_{k+1}
// += F_{k+1}; may alias A, read before it is overwritten).
template <typename V, int MODE>
__global__ void __launch_bounds__(kBandThreads, 2)
k_band_up(const BandParams<V> P, V *__restrict__ x, V *r, const V *__restrict__ p,
          const V *__restrict__ q, V *A, const V *F, CgScalars *sc, double *part, unsigned *ticket)
{
    if (halted(sc)) return;
    extern __shared__ __align__(16) unsigned char band_raw[];
    __shared__ BandTile T;
    __shared__ __align__(8) uint64_t bar;
    const int tid = threadIdx.x, L = P.nlev;
    const V al = MODE == 1 || MODE == 3 ? (V)sc->alpha : V(0);
    double rr = 0.0, rs = 0.0;
    if (tid == 0) {
        mbar_init(&bar);
        fence_async_smem();
    }
    uint32_t parity = 0;
    for (int t = blockIdx.x; t < P.ntiles; t += gridDim.x) {
        band_load_tile(P, t, T);
        __syncthreads();
        const int64_t o0 = P.lev[0].off;
        // level k0 comes from A (copied) or from r
        const bool copy0 = MODE == 0 || (MODE == 3 && !P.first);
        if (T.rec.cbytes >= 0) {
            // thread 0 lays the tile out and starts the copies while the
            // block takes level 0 from r (MODE 1, 2, 3 first band) into the
            // region after the coefficients
            if (tid == 0) {
                band_coef_offsets<V>(L, T);
                // coefficients at 0, level-0 values after them (with the
                // source's 16-byte phase when copied), levels 1..L after that
                const int u0 = T.rec.cbytes;
                const Span s0 = span(A, o0 + T.st[0], T.cnt[0], sizeof(V));
                T.vs[0] = u0 + (copy0 ? s0.head : 0);
                int v = u0 + r16(16 + T.cnt[0] * (int)sizeof(V));
                for (int j = 1; j <= L; ++j) {
                    T.vs[j] = v;
                    v += T.cnt[j] * (int)sizeof(V);
                }
                fence_async_smem();
                mbar_expect(&bar, T.rec.cbytes + (copy0 ? s0.bytes : 0));
                bulk_load(band_raw, P.coef + T.rec.cb, T.rec.cbytes, &bar);
                if (copy0) bulk_load(band_raw + u0, s0.src, s0.bytes, &bar);
            }
            if (MODE == 3) {
                // the CG step on levels 0 (first band) or 1 .. L, staged where
                // the elimination adds them (the layout above must be visible
                // first)
                __syncthreads();
                band_cg_levels(P, T, band_raw, copy0 ? 1 : 0, L, al, x, r, p, q, rr, rs);
            }
            if (MODE != 3 && !copy0) {
                // level 0 from r (after the CG step), four elements per thread in flight
                V *v0 = reinterpret_cast<V *>(band_raw + T.rec.cbytes);
                for (int i0 = tid; i0 < T.cnt[0]; i0 += 4 * kBandThreads) {
                    V xv[4], pv[4], qv[4], rv[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int i = i0 + k * kBandThreads;
                        if (i < T.cnt[0]) {
                            const int64_t u = T.st[0] + i;
                            rv[k] = r[u];
                            if (MODE == 1 || MODE == 3) {
                                xv[k] = x[u];
                                pv[k] = p[u];
                                qv[k] = q[u];
                            }
                        }
                    }
                    // the four products and values summed in V, the rest in FP64
                    V r2 = V(0), r1 = V(0);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int i = i0 + k * kBandThreads;
                        if (i < T.cnt[0]) {
                            const int64_t u = T.st[0] + i;
                            V v = rv[k];
                            if (MODE == 1 || MODE == 3) {
                                x[u] = xv[k] + al * pv[k];
                                v = v - al * qv[k];
                                r[u] = v;
                            }
                            r2 += v * v;
                            r1 += v;
                            v0[i] = v;
                        }
                    }
                    rr += (double)r2;
                    rs += (double)r1;
                }
            }
            if (!mbar_wait(&bar, parity)) {
                if (tid == 0) sc->flag = kBreakdown;
                return;
            }
            parity ^= 1u;
            __syncthreads();
            const int jw = T.jw;
            for (int j = 0; j < jw; ++j) {
                band_up_level<V, MODE == 3>(P, T, band_raw, j, F, 0, kBandThreads);
                __syncthreads();
            }
            // the small top levels by warp 0 while the other warps store the
            // deltas of the levels already done
            V *ds = P.scratch + T.rec.ds / (long long)sizeof(V);
            if (tid < 32) {
                for (int j = jw; j < L; ++j) {
                    band_up_level<V, MODE == 3>(P, T, band_raw, j, F, 0, 32);
                    __syncwarp();
                }
            } else {
                int base = 0;
                for (int j = 0; j < jw; ++j) {
                    const V *src = reinterpret_cast<const V *>(band_raw + T.vs[j]);
                    for (int i = tid - 32; i < T.cnt[j]; i += kBandThreads - 32) ds[base + i] = src[i];
                    base += T.cnt[j];
                }
            }
            __syncthreads();
            {
                int base = 0;
                for (int j = 0; j < jw; ++j) base += T.cnt[j];
                for (int j = jw; j < L; ++j) {
                    const V *src = reinterpret_cast<const V *>(band_raw + T.vs[j]);
                    for (int i = tid; i < T.cnt[j]; i += kBandThreads) ds[base + i] = src[i];
                    base += T.cnt[j];
                }
                const V *src = reinterpret_cast<const V *>(band_raw + T.vs[L]);
                V *dst = A + P.off_top + T.st[L];
                for (int i = tid; i < T.cnt[L]; i += kBandThreads) dst[i] = src[i];
            }
        } else {
            // oversized subtree: the same steps in place in global memory
            V *b0 = A + o0 + T.st[0];
            if (MODE == 3)
                for (int j = P.first ? 0 : 1; j <= L; ++j) {
                    const int64_t g0 = band_level_base(P, T, j);
                    band_cg_step(g0, T.cnt[j], al, x, r, p, q, A + g0, rr, rs);
                }
            for (int i = tid; MODE != 3 && i < T.cnt[0]; i += kBandThreads) {
                const int64_t u = T.st[0] + i;
                V v;
                if (MODE == 1) {
                    x[u] += al * p[u];
                    v = r[u] - al * q[u];
                    r[u] = v;
                } else if (MODE == 2) {
                    v = r[u];
                } else {
                    v = b0[i];
                }
                if (MODE != 0) {
                    rr += (double)v * (double)v;
                    rs += (double)v;
                    b0[i] = v;
                }
            }
            __syncthreads();
            for (int j = 0; j < L; ++j) {
                const BandLevel<V> &Lv = P.lev[j];
                const int64_t onext = j + 1 < L ? P.lev[j + 1].off : P.off_top;
                const int J0 = T.st[j + 1];
                elim_level(A + Lv.off + T.st[j], A + onext + J0, Lv.seg + J0, T.st[j], Lv.inv + 4 * (int64_t)J0,
                           Lv.lcf + 3 * ((int64_t)T.st[j] - 2 * (int64_t)J0), Lv.gamma,
                           MODE == 3 ? static_cast<const V *>(A) : F, onext + J0, T.cnt[j + 1], 0, kBandThreads);
                __syncthreads();
            }
        }
        __syncthreads();
    }
    if (MODE == 0) return;
    // per-block partials of ||r||^2 and sum r; the next single-block kernel
    // (the coarse tail) adds them up and finishes the iteration's test
    double v[2] = {rr, rs};
    block_sum<2>(v);
    if (threadIdx.x == 0) {
        const int o = (MODE == 3 ? P.red_up : 0) + 2 * blockIdx.x;
        part[o] = v[0];
        part[o + 1] = v[1];
    }
    (void)ticket;
}

// One level of the downward pass of a staged tile (in place), by threads
// [tid0, tid0 + nthr).
template <typename V>
__device__ __forceinline__ void band_down_level(const BandParams<V> &P, const BandTile &T, unsigned char *sm, int j,
                                                int tid0, int nthr)
{
    V *o = reinterpret_cast<V *>(sm + T.vs[j]);
    prolong_level(o, o, reinterpret_cast<const V *>(sm + T.vs[j + 1]), reinterpret_cast<const int *>(sm + T.ss[j]),
                  0, P.pc, P.lev[j].dcoef, T.cnt[j + 1], tid0, nthr);
}

// The elements of levels j0..j1 of a staged tile taken as one sequence:
// element t lies on level lv at index ix.  `lv`, `base` carry the level of an
// earlier element and the sequence index of that level's first element, so
// a thread walking t upwards steps through the levels once.
__device__ __forceinline__ void band_locate(const BandTile &T, int t, int &lv, int &base)
{
    while (t >= base + T.cnt[lv]) {
        base += T.cnt[lv];
        ++lv;
    }
}

// CG step on every level j0..j1 of a staged tile, the updated r staged at
// the level's values in shared memory: the levels taken as one sequence, so
// that each thread keeps G elements in flight across level boundaries.
template <typename V>
__device__ __forceinline__ void band_cg_levels(const BandParams<V> &P, const BandTile &T, unsigned char *sm, int j0,
                                               int j1, V al, V *__restrict__ x, V *__restrict__ r,
                                               const V *__restrict__ p, const V *__restrict__ q, double &rr,
                                               double &rs)
{
    constexpr int G = sizeof(V) == 4 ? 4 : 2;
    int tot = 0;
    for (int j = j0; j <= j1; ++j) tot += T.cnt[j];
    int lv0 = j0, base0 = 0;
    for (int t0 = threadIdx.x; t0 < tot; t0 += G * kBandThreads) {
        int lv[G], ix[G];
        V xv[G], pv[G], qv[G], rv[G];
        int l = lv0, b = base0;
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const int t = t0 + k * kBandThreads;
            lv[k] = -1;
            if (t < tot) {
                band_locate(T, t, l, b);
                if (k == 0) {
                    lv0 = l;
                    base0 = b;
                }
                lv[k] = l;
                ix[k] = t - b;
                const int64_t u = band_level_base(P, T, l) + ix[k];
                xv[k] = x[u];
                pv[k] = p[u];
                qv[k] = q[u];
                rv[k] = r[u];
            }
        }
        V r2 = V(0), r1 = V(0);
#pragma unroll
        for (int k = 0; k < G; ++k) {
            if (lv[k] >= 0) {
                const int64_t u = band_level_base(P, T, lv[k]) + ix[k];
                x[u] = xv[k] + al * pv[k];
                const V v = rv[k] - al * qv[k];
                r[u] = v;
                reinterpret_cast<V *>(sm + T.vs[lv[k]])[ix[k]] = v;
                r2 += v * v;
                r1 += v;
            }
        }
        rr += (double)r2;
        rs += (double)r1;
    }
}

// sum z and r.z over levels 0..L-1 of a staged tile (z at the levels' values
// in shared memory, r global), as one sequence with G loads in flight.
template <typename V>
__device__ __forceinline__ void band_zred_levels(const BandParams<V> &P, const BandTile &T, const unsigned char *sm,
                                                 const V *__restrict__ r, double &sz, double &srz)
{
    constexpr int G = sizeof(V) == 4 ? 8 : 4;
    int tot = 0;
    for (int j = 0; j < P.nlev; ++j) tot += T.cnt[j];
    int lv0 = 0, base0 = 0;
    for (int t0 = threadIdx.x; t0 < tot; t0 += G * kBandThreads) {
        int lv[G], ix[G];
        V rv[G];
        int l = lv0, b = base0;
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const int t = t0 + k * kBandThreads;
            lv[k] = -1;
            if (t < tot) {
                band_locate(T, t, l, b);
                if (k == 0) {
                    lv0 = l;
                    base0 = b;
                }
                lv[k] = l;
                ix[k] = t - b;
                rv[k] = r[P.lev[l].off + T.st[l] + ix[k]];
            }
        }
        V a1 = V(0), a2 = V(0);
#pragma unroll
        for (int k = 0; k < G; ++k) {
            if (lv[k] >= 0) {
                const V zv = reinterpret_cast<const V *>(sm + T.vs[lv[k]])[ix[k]];
                a1 += zv;
                a2 += rv[k] * zv;
            }
        }
        sz += (double)a1;
        srz += (double)a2;
    }
}

// sum z and r.z over `cnt` consecutive values z (shared or global) whose
// expanded indices start at g0 (groups of four in V, then FP64).
template <typename V>
__device__ __forceinline__ void band_zred(const V *z, int64_t g0, int cnt, const V *__restrict__ r, double &sz,
                                          double &srz)
{
    for (int i0 = threadIdx.x; i0 < cnt; i0 += 4 * kBandThreads) {
        V rv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + k * kBandThreads;
            if (i < cnt) rv[k] = r[g0 + i];
        }
        V a1 = V(0), a2 = V(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + k * kBandThreads;
            if (i < cnt) {
                const V zv = z[i];
                a1 += zv;
                a2 += rv[k] * zv;
            }
        }
        sz += (double)a1;
        srz += (double)a2;
    }
}

// Downward band: for j = k1-1 .. k0, out_j(u) = pc * out_{j+1}(J) + dcoef_j *
// D_j(u), starting from the level-k1 values in Yp.  The deltas come from the
// band's scratch (DEXP false, written by the upward band) or from the
// expanded array D (DEXP true).  Level k0 goes to out0 (indexed from the
// level's first vertex); with write_all the levels above k0 go to Y
// (expanded).  FINEST: out0 is the preconditioned residual z of the n-space
// CG; reduces sum z, r.z, z.q and finalises zmean, rho, beta.  A tile in
// global memory reads its deltas in place from D (A for the sweeps).
// XRED (expanded-space CG, write_all, out0 = Y + offset of level k0): sums
// z and r.z over every level of the band with r the expanded residual; the
// first band finishes them with the tail's and the upper bands' partials
// (n = ntilde) and sets the next direction's coefficients.
template <typename V, bool FINEST, bool DEXP, bool XRED = false>
__global__ void __launch_bounds__(kBandThreads, 2)
k_band_down(const BandParams<V> P, const V *__restrict__ D, const V *Yp, V *Y, V *out0, int write_all,
            int n, const V *__restrict__ r, const V *__restrict__ q, CgScalars *sc, double *part,
            unsigned *ticket)
{
    if (halted(sc)) return;
    extern __shared__ __align__(16) unsigned char band_raw[];
    __shared__ BandTile T;
    __shared__ __align__(8) uint64_t bar;
    const int tid = threadIdx.x, L = P.nlev;
    const bool flex = FINEST && sc->flexible && !sc->first;
    double sz = 0.0, srz = 0.0, szq = 0.0;
    if (tid == 0) {
        mbar_init(&bar);
        fence_async_smem();
    }
    uint32_t parity = 0;
    for (int t = blockIdx.x; t < P.ntiles; t += gridDim.x) {
        band_load_tile(P, t, T);
        __syncthreads();
        if (T.rec.cbytes >= 0) {
            if (tid == 0) {
                band_coef_offsets<V>(L, T);
                // segments at 0, then the deltas (one packed block, or level
                // by level with each source's 16-byte phase), then the parents
                int cur = T.rec.sbytes;
                uint32_t tx = T.rec.sbytes;
                if (!DEXP) {
                    int v = cur;
                    for (int j = 0; j < L; ++j) {
                        T.vs[j] = v;
                        v += T.cnt[j] * (int)sizeof(V);
                    }
                    const int db = r16(v - cur);
                    T.xs[0] = db;
                    cur += db;
                    tx += db;
                } else {
                    for (int j = 0; j < L; ++j) {
                        const Span s = span(D, P.lev[j].off + T.st[j], T.cnt[j], sizeof(V));
                        T.xs[j] = cur;
                        T.vs[j] = cur + s.head;
                        cur += r16(16 + T.cnt[j] * (int)sizeof(V));
                        tx += s.bytes;
                    }
                }
                const Span sp = span(Yp, P.off_top + T.st[L], T.cnt[L], sizeof(V));
                T.xs[L] = cur;
                T.vs[L] = cur + sp.head;
                cur += r16(16 + T.cnt[L] * (int)sizeof(V));
                tx += sp.bytes;
                Span sr{nullptr, 0, 0};
                if (FINEST) {
                    sr = span(r, T.st[0], T.cnt[0], sizeof(V));
                    T.rsm = cur + sr.head;
                    tx += sr.bytes;
                }
                const int rdst = cur;
                fence_async_smem();
                mbar_expect(&bar, tx);
                bulk_load(band_raw, P.coef + T.rec.cb, T.rec.sbytes, &bar);
                if (!DEXP) {
                    bulk_load(band_raw + T.rec.sbytes, P.scratch + T.rec.ds / (long long)sizeof(V), T.xs[0], &bar);
                } else {
                    for (int j = 0; j < L; ++j) {
                        const Span s = span(D, P.lev[j].off + T.st[j], T.cnt[j], sizeof(V));
                        bulk_load(band_raw + T.xs[j], s.src, s.bytes, &bar);
                    }
                }
                bulk_load(band_raw + T.xs[L], sp.src, sp.bytes, &bar);
                if (FINEST) bulk_load(band_raw + rdst, sr.src, sr.bytes, &bar);
            }
            __syncthreads();
            if (!mbar_wait(&bar, parity)) {
                if (tid == 0) sc->flag = kBreakdown;
                return;
            }
            parity ^= 1u;
            const int jw = T.jw;
            if (tid < 32)
                for (int j = L - 1; j >= jw; --j) {
                    band_down_level(P, T, band_raw, j, 0, 32);
                    __syncwarp();
                }
            __syncthreads();
            for (int j = jw - 1; j >= 0; --j) {
                band_down_level(P, T, band_raw, j, 0, kBandThreads);
                __syncthreads();
            }
            const V *z0 = reinterpret_cast<const V *>(band_raw + T.vs[0]);
            const V *r0 = reinterpret_cast<const V *>(band_raw + T.rsm);
            for (int i0 = tid; i0 < T.cnt[0]; i0 += 4 * kBandThreads) {
                V qv[4];
                if (flex) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int i = i0 + k * kBandThreads;
                        if (i < T.cnt[0]) qv[k] = q[T.st[0] + i];
                    }
                }
                // the four values and products summed in V, the rest in FP64
                V a1 = V(0), a2 = V(0), a3 = V(0);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int i = i0 + k * kBandThreads;
                    if (i < T.cnt[0]) {
                        const V zv = z0[i];
                        out0[T.st[0] + i] = zv;
                        if (FINEST) {
                            a1 += zv;
                            a2 += r0[i] * zv;
                            if (flex) a3 += zv * qv[k];
                        }
                    }
                }
                if (FINEST) {
                    sz += (double)a1;
                    srz += (double)a2;
                    szq += (double)a3;
                }
            }
            if (write_all)
                for (int j = 1; j < L; ++j) {
                    const V *src = reinterpret_cast<const V *>(band_raw + T.vs[j]);
                    V *dst = Y + P.lev[j].off + T.st[j];
                    for (int i = tid; i < T.cnt[j]; i += kBandThreads) dst[i] = src[i];
                }
            if (XRED) band_zred_levels(P, T, band_raw, r, sz, srz);
        } else {
            for (int j = L - 1; j >= 0; --j) {
                const BandLevel<V> &Lv = P.lev[j];
                const int64_t oup = j + 1 < L ? P.lev[j + 1].off : P.off_top;
                const V *par = j + 1 < L ? Y + oup + T.st[j + 1] : Yp + P.off_top + T.st[L];
                V *o = j == 0 ? out0 + T.st[0] : Y + Lv.off + T.st[j];
                prolong_level(o, D + Lv.off + T.st[j], par, Lv.seg + T.st[j + 1], T.st[j], P.pc, Lv.dcoef,
                              T.cnt[j + 1], 0, kBandThreads);
                __syncthreads();
            }
            if (FINEST)
                for (int i = tid; i < T.cnt[0]; i += kBandThreads) {
                    const int64_t u = T.st[0] + i;
                    const V zv = out0[u];
                    sz += (double)zv;
                    srz += (double)r[u] * (double)zv;
                    if (flex) szq += (double)zv * (double)q[u];
                }
            if (XRED) {
                __syncthreads();
                for (int j = 0; j < L; ++j) {
                    const int64_t g0 = P.lev[j].off + T.st[j];
                    band_zred<V>(Y + g0, g0, T.cnt[j], r, sz, srz);
                }
            }
        }
        __syncthreads();
    }
    if (XRED) {
        double v[2] = {sz, srz};
        if (!P.first) {
            block_sum<2>(v);
            if (threadIdx.x == 0) {
                part[P.red_dn + 2 * blockIdx.x] = v[0];
                part[P.red_dn + 2 * blockIdx.x + 1] = v[1];
            }
            return;
        }
        if (grid_sum<2>(v, part + P.red_gs, ticket) && threadIdx.x == 0) {
            // then the tail's pair and the upper bands' blocks, in order
            for (int k = 0; k < P.xred_n; ++k) {
                v[0] += __ldcg(part + P.xred_base + 2 * k);
                v[1] += __ldcg(part + P.xred_base + 2 * k + 1);
            }
            const double m = v[0] / (double)n;
            set_direction(sc, m, v[1] - m * sc->rs, 0.0);
        }
        return;
    }
    if (!FINEST) return;
    double v[3] = {sz, srz, szq};
    if (grid_sum<3>(v, part, ticket) && threadIdx.x == 0) {
        const double m = v[0] / (double)n;
        set_direction(sc, m, v[1] - m * sc->rs, v[2]);
    }
}

}  // namespace lap
