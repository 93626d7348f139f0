// Device kernels of the GB300 graph-Laplacian solver (sm_103a).
//
// Everything on this path is bound by HBM bandwidth or latency: CSR matvecs,
// segmented sums and broadcasts over the aggregation tree, and vector updates
// with dot products.  No kernel here is a dense contraction, so none uses the
// tensor cores.  Vectors are stored in tree order (see lap_internal.h), which
// makes every restriction/prolongation a pass over contiguous segments.
//
// V is the storage and arithmetic type of vectors, matrix values and sweeps
// (double, or float for the mixed-precision inner solves); every reduction and
// every CG scalar is accumulated and kept in double.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#ifndef LAP_TAIL_MAX_LEVELS
#define LAP_TAIL_MAX_LEVELS 24
#endif

namespace lap {

constexpr int kBlock = 256;
constexpr int kMaxRedBlocks = 2048;   // capacity of the block-partials buffer
constexpr int kRedSlots = 4;          // values reduced per kernel, at most

// CG state kept on the device so that a whole iteration runs without the host.
struct CgScalars {
    double rho;        // r^T z (z projected)
    double alpha;      // step length
    double beta;       // direction update coefficient
    double zmean;      // mean of the latest preconditioned residual
    double pq;         // p^T L p
    double qsum;       // sum of L p (zero up to rounding)
    double rr, rs;     // ||r||^2 and sum(r) after the latest update
    double bnorm;      // ||Pi b|| of the system being solved
    double bmean;      // mean of b (projection)
    double tol;        // recurrence tolerance on ||r|| / ||Pi b||
    double relres;     // latest recurrence relative residual
    double tmp;        // scratch sum
    int iter;          // completed iterations
    int maxit;
    int flag;          // kRun, kConverged, kBreakdown, kMaxit
    int flexible;      // 1: flexible (FCG) beta
    int first;         // 1 while preparing the initial direction
    int hist_cap;      // capacity of hist
    double *hist;      // optional recurrence-residual history (device), or null
    double *lz;        // optional (alpha, beta) of every step, 2 * hist_cap, or null
    int stop;          // FGMRES: the flag that ended the latest cycle
    int inner_total;   // inner iterations of the device-sequenced PEGP solves
};

enum : int { kRun = 0, kConverged = 1, kBreakdown = 2, kMaxit = 3 };

// A completed step (x += alpha p, r -= alpha q, rr = ||r||^2): count it,
// record its recurrence residual and alpha, test convergence.
__device__ __forceinline__ void finish_step(CgScalars *sc, double rr)
{
    sc->iter += 1;
    const double rel = sqrt(rr) / sc->bnorm;
    sc->relres = rel;
    if (sc->iter <= sc->hist_cap) {
        sc->hist[sc->iter - 1] = rel;
        if (sc->lz) sc->lz[2 * (sc->iter - 1)] = sc->alpha;
    }
    if (!isfinite(rel)) sc->flag = kBreakdown;
    else if (rel <= sc->tol) sc->flag = kConverged;
    else if (sc->iter >= sc->maxit) sc->flag = kMaxit;
}

// Next direction's coefficients from z = B r: m = mean(z), rho_new = r^T Pi z,
// zq = z^T q (flexible CG only).  beta = rho_new / rho, or Notay's FCG(1)
// choice -alpha (Pi z)^T q / rho when the preconditioner varies; recorded
// beside the step's alpha (the pairs define CG's Lanczos tridiagonal).
__device__ __forceinline__ void set_direction(CgScalars *sc, double m, double rho_new, double zq)
{
    sc->zmean = m;
    if (sc->first) sc->beta = 0.0;
    else if (sc->flexible) sc->beta = -sc->alpha * (zq - m * sc->qsum) / sc->rho;
    else sc->beta = rho_new / sc->rho;
    if (!sc->first && sc->lz && sc->iter >= 1 && sc->iter <= sc->hist_cap)
        sc->lz[2 * (sc->iter - 1) + 1] = sc->beta;
    sc->rho = rho_new;
    sc->first = 0;
    if (!isfinite(rho_new)) sc->flag = kBreakdown;
}

// ---------------------------------------------------------------------------
// Deterministic grid reduction: every block reduces its NV partial sums, the
// last block to finish (ticket) adds the per-block partials in block order.
// All threads of every block must call it.  Returns true in the last block,
// where tot[] holds the grid totals (valid in thread 0).
// ---------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV])
{
    __shared__ double sm[32][NV];              // blocks of up to 1024 threads
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double x = v[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        v[i] = x;
    }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) sm[wid][i] = v[i];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double x = lane < (int)(blockDim.x >> 5) ? sm[lane][i] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            v[i] = x;
        }
    }
}

template <int NV>
__device__ __forceinline__ bool grid_sum(double (&v)[NV], double *part, unsigned *ticket)
{
    __shared__ bool last;
    block_sum<NV>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) part[blockIdx.x * NV + i] = v[i];
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double x = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) x += __ldcg(part + b * NV + i);
        v[i] = x;
    }
    block_sum<NV>(v);
    if (threadIdx.x == 0) *ticket = 0u;
    return true;
}

__device__ __forceinline__ bool halted(const CgScalars *sc) { return sc && sc->flag != kRun; }

// Solve the 2x2 Schur complement [[alpha+c, -c], [-c, beta+c]] (da, db) = (ha, hb)
// of one aggregate's matched pair from cf = (beta/det, alpha/det, 1/(alpha+beta),
// alpha/(alpha+beta)): the difference D = da - db and the weighted sum
// alpha da + beta db = ha + hb carry no cancellation, unlike the inverse.
template <typename V>
__device__ __forceinline__ void pair_solve(const V *cf, V ha, V hb, V &da, V &db)
{
    const V D = cf[0] * ha - cf[1] * hb;
    db = cf[2] * (ha + hb) - cf[3] * D;
    da = db + D;
}

// ---------------------------------------------------------------------------
// CSR Laplacian matvec in edge-difference form, TPR threads per row:
//     y_i = sum_j w_ij (x_i - x_j)
// which equals (D - A) x but never forms d_i x_i - sum_j w_ij x_j, whose
// cancellation loses every digit of a smooth x in FP32 when the weights span
// several decades; x_i - x_j of nearby values is exact (Sterbenz).
// MODE 0: y = L x, reduce (x.y, sum y) and set alpha = rho / x.y
// MODE 1: yres(double) = bs - L x, reduce (||yres||^2, sum yres) [true residual]
// MODE 2: y = L x, no reduction
// ---------------------------------------------------------------------------
template <typename V, int TPR, int MODE>
__global__ void __launch_bounds__(kBlock)
k_spmv(int n, const int *__restrict__ rp, const int *__restrict__ ci, const V *__restrict__ w,
       const V *__restrict__ x, V *__restrict__ y, const double *__restrict__ bs,
       double *__restrict__ yres, CgScalars *sc, double *part, unsigned *ticket)
{
    if (MODE != 2 && halted(sc)) return;
    constexpr int RPW = 32 / TPR;      // rows per warp
    const int lane = threadIdx.x & 31;
    const int sub = lane / TPR, l = lane % TPR;
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    double a0 = 0.0, a1 = 0.0;
    for (int r0 = gwarp * RPW; r0 < n; r0 += nwarp * RPW) {   // warp-uniform loop
        const int row = r0 + sub;
        const bool valid = row < n;
        const int b = valid ? rp[row] : 0, e = valid ? rp[row + 1] : 0;
        const V xi = valid ? x[row] : V(0);
        V s = V(0);
        for (int p = b + l; p < e; p += TPR) s += w[p] * (xi - x[ci[p]]);
#pragma unroll
        for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, TPR);
        if (valid && l == 0) {
            if (MODE == 1) {
                const double ri = bs[row] - (double)s;
                yres[row] = ri;
                a0 += ri * ri;
                a1 += ri;
            } else {
                y[row] = s;
                if (MODE == 0) {
                    a0 += (double)xi * (double)s;
                    a1 += (double)s;
                }
            }
        }
    }
    if (MODE == 2) return;
    double v[2] = {a0, a1};
    if (grid_sum<2>(v, part, ticket) && threadIdx.x == 0) {
        if (MODE == 0) {
            sc->pq = v[0];
            sc->qsum = v[1];
            const double alpha = sc->rho / v[0];
            if (!(v[0] > 0.0) || !isfinite(alpha)) sc->flag = kBreakdown;
            sc->alpha = alpha;
        } else {
            sc->rr = v[0];
            sc->rs = v[1];
            sc->relres = sqrt(v[0]) / sc->bnorm;
        }
    }
}

// ---------------------------------------------------------------------------
// The same matvec on the SELL-32 layout: one warp per slice of 32 rows, lane =
// row; entry j of all 32 rows is one coalesced load of column indices and one
// of weights, and the gathers of x over j are independent.  Warp tasks past the
// slices take one long row each (CSR, lanes stride the row).
// ---------------------------------------------------------------------------
template <typename V, int MODE>
__device__ __forceinline__ void spmv_finish(int row, V xi, V s, V *y, const double *bs, double *yres,
                                            double &a0, double &a1)
{
    if (MODE == 1) {
        const double ri = bs[row] - (double)s;
        yres[row] = ri;
        a0 += ri * ri;
        a1 += ri;
    } else {
        y[row] = s;
        if (MODE == 0) {
            a0 += (double)xi * (double)s;
            a1 += (double)s;
        }
    }
}

// Loads of a matrix entry stream: HINT marks them evict-first (each entry is
// read once per product), so that the gathered vector stays in L2.
template <bool HINT, typename T>
__device__ __forceinline__ T ldm(const T *p)
{
    if (HINT) return __ldcs(p);
    return __ldg(p);
}

// One entry of a row sum: w (x_i - x_j) in the edge-difference form, w x_j
// in the stored-diagonal form (DIAG; the row then finishes as d_i x_i - sum).
template <bool DIAG, typename V>
__device__ __forceinline__ V edge_term(V s, V w, V xi, V xj)
{
    if (DIAG) return s + w * xj;
    return s + w * (xi - xj);
}

// VEC consecutive entries of one lane (a lane group of the SELL layout) with
// vector loads; the row sum is still accumulated entry by entry.
template <typename V, int VEC, bool HINT = false, bool DIAG = false> struct LaneGroup;
template <typename V, bool HINT, bool DIAG> struct LaneGroup<V, 1, HINT, DIAG> {
    __device__ __forceinline__ static V add(V s, V xi, const int *c, const V *w, const V *__restrict__ x)
    {
        return edge_term<DIAG>(s, ldm<HINT>(w), xi, x[ldm<HINT>(c)]);
    }
};
template <bool HINT, bool DIAG> struct LaneGroup<float, 2, HINT, DIAG> {
    __device__ __forceinline__ static float add(float s, float xi, const int *c, const float *w,
                                                const float *__restrict__ x)
    {
        const int2 cc = ldm<HINT>(reinterpret_cast<const int2 *>(c));
        const float2 ww = ldm<HINT>(reinterpret_cast<const float2 *>(w));
        s = edge_term<DIAG>(s, ww.x, xi, x[cc.x]);
        return edge_term<DIAG>(s, ww.y, xi, x[cc.y]);
    }
};
template <bool HINT, bool DIAG> struct LaneGroup<float, 4, HINT, DIAG> {
    __device__ __forceinline__ static float add(float s, float xi, const int *c, const float *w,
                                                const float *__restrict__ x)
    {
        const int4 cc = ldm<HINT>(reinterpret_cast<const int4 *>(c));
        const float4 ww = ldm<HINT>(reinterpret_cast<const float4 *>(w));
        s = edge_term<DIAG>(s, ww.x, xi, x[cc.x]);
        s = edge_term<DIAG>(s, ww.y, xi, x[cc.y]);
        s = edge_term<DIAG>(s, ww.z, xi, x[cc.z]);
        return edge_term<DIAG>(s, ww.w, xi, x[cc.w]);
    }
};
template <bool HINT, bool DIAG> struct LaneGroup<double, 2, HINT, DIAG> {
    __device__ __forceinline__ static double add(double s, double xi, const int *c, const double *w,
                                                 const double *__restrict__ x)
    {
        const int2 cc = ldm<HINT>(reinterpret_cast<const int2 *>(c));
        const double2 ww = ldm<HINT>(reinterpret_cast<const double2 *>(w));
        s = edge_term<DIAG>(s, ww.x, xi, x[cc.x]);
        return edge_term<DIAG>(s, ww.y, xi, x[cc.y]);
    }
};
template <bool HINT, bool DIAG> struct LaneGroup<double, 4, HINT, DIAG> {
    __device__ __forceinline__ static double add(double s, double xi, const int *c, const double *w,
                                                 const double *__restrict__ x)
    {
        const int4 cc = ldm<HINT>(reinterpret_cast<const int4 *>(c));
        const double2 w0 = ldm<HINT>(reinterpret_cast<const double2 *>(w));
        const double2 w1 = ldm<HINT>(reinterpret_cast<const double2 *>(w) + 1);
        s = edge_term<DIAG>(s, w0.x, xi, x[cc.x]);
        s = edge_term<DIAG>(s, w0.y, xi, x[cc.y]);
        s = edge_term<DIAG>(s, w1.x, xi, x[cc.z]);
        return edge_term<DIAG>(s, w1.y, xi, x[cc.w]);
    }
};

// Partial sums of the long rows, one warp per chunk of <= 4096 entries.
template <typename V, bool HINT = false, bool DIAG = false>
__global__ void __launch_bounds__(kBlock)
k_long_chunks(int nchunks, const int *__restrict__ chunk_row, const int64_t *__restrict__ chunk_beg,
              const int *__restrict__ lrow, const int *__restrict__ lci, const V *__restrict__ lw,
              const V *__restrict__ x, V *__restrict__ chunk_part, const CgScalars *sc, int check)
{
    if (check && halted(sc)) return;
    const int lane = threadIdx.x & 31;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks; c += nwarp) {
        const V xi = x[lrow[chunk_row[c]]];
        V s = V(0);
        // chunks hold a multiple of 128 entries from a multiple-of-128 start:
        // lane l takes entries 128 g + 4 l .. + 3 with one vector load each
#pragma unroll 2
        for (int64_t p = chunk_beg[c] + 4 * lane; p < chunk_beg[c + 1]; p += 128)
            s = LaneGroup<V, 4, HINT, DIAG>::add(s, xi, lci + p, lw + p, x);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) chunk_part[c] = s;
    }
}

// SELL-32 matvec in edge-difference form: one warp per slice of 32 rows,
// lane l owning the row of slot 32 s + l and reading its entries VEC at a
// time (see make_sell for the layout); long rows add their chunk partials.
// The warps stride over the slices; the grid (one or more waves of resident
// blocks) is chosen per matrix at setup by timing.  DIAG: the stored-diagonal
// form y_i = dg_i x_i - sum_j w_ij x_j instead (one multiply-add per entry
// instead of a subtraction and a multiply-add; timed, not used by the solves).
template <typename V, int MODE, int VEC, bool HINT = false, bool DIAG = false>
__global__ void __launch_bounds__(kBlock)
k_sell(int n, int nslices, const int64_t *__restrict__ sptr, const unsigned *__restrict__ lmask,
       const int *__restrict__ rowperm, const int *__restrict__ eci, const V *__restrict__ ew, int nlong,
       const int *__restrict__ lrow,
       const int *__restrict__ lchunk_ptr, const V *__restrict__ chunk_part,
       const V *__restrict__ x, V *__restrict__ y, const double *__restrict__ bs,
       double *__restrict__ yres, CgScalars *sc, double *part, unsigned *ticket,
       const V *__restrict__ dg = nullptr)
{
    if (MODE != 2 && halted(sc)) return;
    const int lane = threadIdx.x & 31;
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    double a0 = 0.0, a1 = 0.0;
    // MODE 0 in FP32: the products of up to four rows summed in V, then in FP64
    V g0 = V(0), g1 = V(0);
    int gc = 0;
    auto finish = [&](int row, V xi, V s) {
        if (MODE == 0 && sizeof(V) == 4) {
            y[row] = s;
            g0 += xi * s;
            g1 += s;
            if (++gc == 4) {
                a0 += (double)g0;
                a1 += (double)g1;
                g0 = g1 = V(0);
                gc = 0;
            }
        } else {
            spmv_finish<V, MODE>(row, xi, s, y, bs, yres, a0, a1);
        }
    };
    auto slice = [&](int task) {
        const int slot = task * 32 + lane;
        const int row = rowperm ? rowperm[slot] : (slot < n ? slot : -1);
        const bool valid = row >= 0;
        const int64_t base = sptr[task];
        const int width = static_cast<int>((sptr[task + 1] - base) >> 5);
        const V xi = valid ? x[row] : V(0);
        V s = V(0);
        const int *pc = eci + base + lane * VEC;
        const V *pw = ew + base + lane * VEC;
        const int ng = width / VEC;
#pragma unroll(VEC == 1 ? 4 : 2)
        for (int g = 0; g < ng; ++g)
            s = LaneGroup<V, VEC, HINT, DIAG>::add(s, xi, pc + 32 * VEC * g, pw + 32 * VEC * g, x);
        if (valid && !((lmask[task] >> lane) & 1u)) finish(row, xi, DIAG ? dg[row] * xi - s : s);
    };
    auto long_row = [&](int li) {
        // long row: add its chunk partials in chunk order
        const int row = lrow[li];
        V s = V(0);
        for (int c = lchunk_ptr[li]; c < lchunk_ptr[li + 1]; ++c) s += chunk_part[c];
        const V xi = x[row];
        finish(row, xi, DIAG ? dg[row] * xi - s : s);
    };
    const int ntask = nslices + nlong;
    for (int task = gwarp; task < ntask; task += nwarp) {          // warp-uniform
        if (task < nslices) slice(task);
        else if (lane == 0) long_row(task - nslices);
    }
    if (MODE == 2) return;
    a0 += (double)g0;
    a1 += (double)g1;
    double v[2] = {a0, a1};
    if (grid_sum<2>(v, part, ticket) && threadIdx.x == 0) {
        if (MODE == 0) {
            sc->pq = v[0];
            sc->qsum = v[1];
            const double alpha = sc->rho / v[0];
            if (!(v[0] > 0.0) || !isfinite(alpha)) sc->flag = kBreakdown;
            sc->alpha = alpha;
        } else {
            sc->rr = v[0];
            sc->rs = v[1];
            sc->relres = sqrt(v[0]) / sc->bnorm;
        }
    }
}

// ---------------------------------------------------------------------------
// CG step without a sweep: x += alpha p, r -= alpha q (UPDATE), reduce ||r||^2
// and sum r, test convergence; rcopy (if given) receives the updated r.  PLAIN
// (unpreconditioned CG) also forms rho = r^T Pi r and beta.
// ---------------------------------------------------------------------------
template <typename V, bool UPDATE, bool PLAIN>
__global__ void __launch_bounds__(kBlock)
k_update(int n, V *__restrict__ x, V *__restrict__ r, const V *__restrict__ p,
         const V *__restrict__ q, V *__restrict__ rcopy, CgScalars *sc, double *part,
         unsigned *ticket)
{
    if (halted(sc)) return;
    double rr = 0.0, rs = 0.0;
    const V al = UPDATE ? (V)sc->alpha : V(0);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        V ri = r[i];
        if (UPDATE) {
            x[i] += al * p[i];
            ri -= al * q[i];
            r[i] = ri;
        }
        if (rcopy) rcopy[i] = ri;
        rr += (double)ri * ri;
        rs += (double)ri;
    }
    double v[2] = {rr, rs};
    if (grid_sum<2>(v, part, ticket) && threadIdx.x == 0) {
        sc->rr = v[0];
        sc->rs = v[1];
        if (UPDATE) {
            finish_step(sc, v[0]);
        }
        if (PLAIN) {
            // unpreconditioned CG: z = Pi r
            const double m = v[1] / (double)n;
            set_direction(sc, m, v[0] - m * v[1], 0.0);
        }
    }
}

// Top level: y = scale * G a with G the dense pseudo-inverse of mu^(2(l-1)) L_l
// (FP64 whatever V is), one warp per row.
template <typename V>
__global__ void __launch_bounds__(kBlock)
k_coarse(int m, const double *__restrict__ G, const V *__restrict__ a, V *__restrict__ y,
         double scale, const CgScalars *sc)
{
    if (halted(sc)) return;
    const int lane = threadIdx.x & 31;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= m) return;
    double s = 0.0;
    for (int j = lane; j < m; j += 32) s += G[(size_t)row * m + j] * (double)a[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = (V)(scale * s);
}

// ---------------------------------------------------------------------------
// Shared-memory-staged sweeps.  A block takes kTA consecutive aggregates of a
// level; in tree order their members are one contiguous range [v0, v1), which
// the block reads (and updates) with coalesced accesses, stages in shared
// memory, solves aggregate by aggregate (one thread each) and writes back
// coalesced.  A tile whose range exceeds kTV members (a hub aggregate) works
// on global memory directly.
// ---------------------------------------------------------------------------
constexpr int kTA = 256;      // aggregates per tile (= threads per block)
constexpr int kTV = 1536;     // staged members per tile

// Elimination of one aggregate (Section 3.3): a = its members' right-hand
// sides (pair first, then leftovers), d = their solution (may alias a).
// Returns the sum of a (the restriction to the parent).
template <typename V>
__device__ __forceinline__ V agg_eliminate(const V *a, V *d, int cnt, const V *lc, const V *cf)
{
    const V aa = a[0], ab = a[1];
    V sum = aa + ab, ha = aa, hb = ab;
    for (int t = 2; t < cnt; ++t) {
        const V al = a[t];
        const V *c = lc + 3 * (t - 2);
        sum += al;
        ha += c[0] * al;
        hb += c[1] * al;
    }
    V da, db;
    pair_solve(cf, ha, hb, da, db);
    for (int t = 2; t < cnt; ++t) {
        const V *c = lc + 3 * (t - 2);
        d[t] = a[t] * c[2] + c[0] * da + c[1] * db;
    }
    d[0] = da;
    d[1] = db;
    return sum;
}

// A warp eliminates one large aggregate: lanes take the leftovers in turn,
// their sums are combined by a fixed shuffle tree, every lane solves the pair
// and writes its leftovers.  Returns the sum of a (all lanes).
template <typename V>
__device__ __forceinline__ V warp_eliminate(V *a, int cnt, const V *lc, const V *cf, int lane)
{
    V s = V(0), ha = V(0), hb = V(0);
    for (int t = 2 + lane; t < cnt; t += 32) {
        const V al = a[t];
        const V *c = lc + 3 * (t - 2);
        s += al;
        ha += c[0] * al;
        hb += c[1] * al;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        ha += __shfl_xor_sync(0xffffffffu, ha, o);
        hb += __shfl_xor_sync(0xffffffffu, hb, o);
    }
    const V aa = a[0], ab = a[1];
    s += aa + ab;
    ha += aa;
    hb += ab;
    V da, db;
    pair_solve(cf, ha, hb, da, db);
    for (int t = 2 + lane; t < cnt; t += 32) {
        const V *c = lc + 3 * (t - 2);
        a[t] = a[t] * c[2] + c[0] * da + c[1] * db;
    }
    __syncwarp();
    if (lane == 0) {
        a[0] = da;
        a[1] = db;
    }
    return s;
}

constexpr int kBigAgg = 32;   // aggregates with more members are eliminated by a warp
constexpr int kBatchBigAgg = 64;   // batched sweeps: aggregates with more members take a block

// Upward elimination of one level of a tile, in place: aggregate jl (of na)
// holds the members [sg[jl] - sbase, sg[jl + 1] - sbase) of a, its pair
// coefficients at ci + 4 jl and the leftover coefficients of member b + t at
// cl + 3 (b - 2 jl) + 3 (t - 2); an[jl] = gamma * (sum of its members) +
// F[fofs + jl] (if F).  Threads [tid0, tid0 + nthr) take part, whole warps;
// aggregates of more than kBigAgg members go to a warp each.
template <typename V>
__device__ __forceinline__ void elim_level(V *a, V *an, const int *sg, int sbase, const V *ci, const V *cl, V gamma,
                                           const V *F, int64_t fofs, int na, int tid0, int nthr)
{
    const int t = threadIdx.x - tid0;
    for (int jl = t; jl < na; jl += nthr) {
        const int b = sg[jl] - sbase, e = sg[jl + 1] - sbase;
        if (e - b > kBigAgg) continue;
        const V sum = agg_eliminate(a + b, a + b, e - b, cl + 3 * (b - 2 * jl), ci + 4 * jl);
        V nx = gamma * sum;
        if (F) nx += F[fofs + jl];
        an[jl] = nx;
    }
    const int lane = t & 31, nw = nthr >> 5;
    for (int q = t >> 5; q * 32 < na; q += nw) {
        const int j0 = q * 32 + lane;
        const bool big = j0 < na && sg[j0 + 1] - sg[j0] > kBigAgg;
        unsigned m = __ballot_sync(0xffffffffu, big);
        while (m) {
            const int jl = q * 32 + __ffs(m) - 1;
            m &= m - 1;
            const int b = sg[jl] - sbase, e = sg[jl + 1] - sbase;
            const V sum = warp_eliminate(a + b, e - b, cl + 3 * (b - 2 * jl), ci + 4 * jl, lane);
            if (lane == 0) {
                V nx = gamma * sum;
                if (F) nx += F[fofs + jl];
                an[jl] = nx;
            }
        }
    }
}

// Downward pass of one level of a tile: o[u] = pc * par[jl] + dc * d[u] for
// the members u of aggregate jl (o may alias d); large aggregates by a warp.
template <typename V>
__device__ __forceinline__ void prolong_level(V *o, const V *d, const V *par, const int *sg, int sbase, V pc, V dc,
                                              int na, int tid0, int nthr)
{
    const int t = threadIdx.x - tid0;
    for (int jl = t; jl < na; jl += nthr) {
        const int b = sg[jl] - sbase, e = sg[jl + 1] - sbase;
        if (e - b > kBigAgg) continue;
        const V base = pc * par[jl];
        for (int u = b; u < e; ++u) o[u] = base + dc * d[u];
    }
    const int lane = t & 31, nw = nthr >> 5;
    for (int q = t >> 5; q * 32 < na; q += nw) {
        const int j0 = q * 32 + lane;
        const bool big = j0 < na && sg[j0 + 1] - sg[j0] > kBigAgg;
        unsigned m = __ballot_sync(0xffffffffu, big);
        while (m) {
            const int jl = q * 32 + __ffs(m) - 1;
            m &= m - 1;
            const int b = sg[jl] - sbase, e = sg[jl + 1] - sbase;
            const V base = pc * par[jl];
            for (int u = b + lane; u < e; u += 32) o[u] = base + dc * d[u];
        }
    }
}

// Upward pass over one level, tiled.
// MODE 0: a (the r argument) holds a_k and is overwritten by delta_k (dout == r)
// MODE 1: finest level with the CG step: x += alpha p, r -= alpha q, then
//         a_1 = r, delta_1 -> dout; reduces ||r||^2, sum r and finalises the
//         convergence test
// MODE 2: finest level without the step (start of a solve), reduces as MODE 1
// anext(J) = gamma * sum_{u in J} a(u) (+ fnext(J) if given; may alias anext).
template <typename V, int MODE>
__global__ void __launch_bounds__(kTA)
k_up_tiled(int nagg, const int *__restrict__ seg, const V *__restrict__ inv,
           const V *__restrict__ lcf, V *__restrict__ x, V *r, const V *__restrict__ p,
           const V *__restrict__ q, V *dout, V *anext, V gamma, const V *fnext, CgScalars *sc,
           double *part, unsigned *ticket)
{
    if (halted(sc)) return;
    __shared__ V sa[kTV];
    __shared__ int sseg[kTA + 1];
    const int tid = threadIdx.x;
    const V al = MODE == 1 ? (V)sc->alpha : V(0);
    double rr = 0.0, rs = 0.0;
    const int ntiles = (nagg + kTA - 1) / kTA;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int J0 = tile * kTA;
        const int na = min(kTA, nagg - J0);
        for (int i = tid; i <= na; i += kTA) sseg[i] = seg[J0 + i];
        __syncthreads();
        const int v0 = sseg[0], nv = sseg[na] - v0;
        const bool staged = nv <= kTV;
        for (int i = tid; i < nv; i += kTA) {
            V ri;
            if (MODE == 1) {
                x[v0 + i] += al * p[v0 + i];
                ri = r[v0 + i] - al * q[v0 + i];
                r[v0 + i] = ri;
            } else {
                ri = r[v0 + i];
            }
            if (MODE != 0) {
                rr += (double)ri * (double)ri;
                rs += (double)ri;
            }
            if (staged) sa[i] = ri;
        }
        __syncthreads();
        if (tid < na) {
            const int J = J0 + tid;
            const int b = sseg[tid] - v0, e = sseg[tid + 1] - v0;
            const V *src = staged ? sa + b : r + v0 + b;
            V *dst = staged ? sa + b : dout + v0 + b;
            const V sum = agg_eliminate(src, dst, e - b, lcf + 3 * (v0 + b - 2 * J), inv + 4 * J);
            V nx = gamma * sum;
            if (fnext) nx += fnext[J];
            anext[J] = nx;
        }
        __syncthreads();
        if (staged)
            for (int i = tid; i < nv; i += kTA) dout[v0 + i] = sa[i];
        __syncthreads();
    }
    if (MODE == 0) return;
    double v[2] = {rr, rs};
    if (grid_sum<2>(v, part, ticket) && threadIdx.x == 0) {
        sc->rr = v[0];
        sc->rs = v[1];
        if (MODE == 1) {
            finish_step(sc, v[0]);
        }
    }
}

// Downward pass over one level, tiled: out(u) = pc * parent(J) + dc * delta(u).
// (pc, dc) = (1, c_k): MSP prolongation z = sum_k c_k delta_k(anc_k(u)), with
//   c_k = sum_{i<k} (-mu)^i > 0: P(mu) applied to the back-substituted
//   sparsifier solution without the alternating Horner sum (Section 3.3);
// (1, 1): back-substitution y_k = y_{k+1}(J) + delta_k (expanded-space solve);
// (-mu, 1): Horner step t_k = y_k - mu t_{k+1}(J) of P(mu) y (Section 2.2).
// FINEST: out is the preconditioned residual z; reduces sum z, r.z, z.q and
// finalises zmean, rho and beta (standard, or flexible FCG).
template <typename V, bool FINEST>
__global__ void __launch_bounds__(kTA)
k_down_tiled(int n, int nagg, const int *__restrict__ seg, const V *__restrict__ delta,
             const V *__restrict__ parent, V *__restrict__ out, V pc, V dc, const V *__restrict__ r,
             const V *__restrict__ q, CgScalars *sc, double *part, unsigned *ticket)
{
    if (halted(sc)) return;
    __shared__ V sb[kTV];
    __shared__ int sseg[kTA + 1];
    const int tid = threadIdx.x;
    const bool flex = FINEST && sc->flexible && !sc->first;
    double sz = 0.0, srz = 0.0, szq = 0.0;
    const int ntiles = (nagg + kTA - 1) / kTA;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int J0 = tile * kTA;
        const int na = min(kTA, nagg - J0);
        for (int i = tid; i <= na; i += kTA) sseg[i] = seg[J0 + i];
        __syncthreads();
        const int v0 = sseg[0], nv = sseg[na] - v0;
        const bool staged = nv <= kTV;
        if (tid < na) {
            const V base = pc * parent[J0 + tid];
            for (int u = sseg[tid]; u < sseg[tid + 1]; ++u) {
                if (staged) {
                    sb[u - v0] = base;
                } else {
                    const V o = base + dc * delta[u];
                    out[u] = o;
                    if (FINEST) {
                        sz += (double)o;
                        srz += (double)r[u] * (double)o;
                        if (flex) szq += (double)o * (double)q[u];
                    }
                }
            }
        }
        __syncthreads();
        if (staged) {
            for (int i = tid; i < nv; i += kTA) {
                const V o = sb[i] + dc * delta[v0 + i];
                out[v0 + i] = o;
                if (FINEST) {
                    sz += (double)o;
                    srz += (double)r[v0 + i] * (double)o;
                    if (flex) szq += (double)o * (double)q[v0 + i];
                }
            }
        }
        __syncthreads();
    }
    if (!FINEST) return;
    double v[3] = {sz, srz, szq};
    if (grid_sum<3>(v, part, ticket) && threadIdx.x == 0) {
        const double m = v[0] / (double)n;
        set_direction(sc, m, v[1] - m * sc->rs, v[2]);
    }
}

// ---------------------------------------------------------------------------
// Fused coarse tail of the sweep: levels t0..l (0-based t0 >= 1) whose
// values, segments and elimination coefficients all fit in shared memory are
// restricted + eliminated upwards, solved on top and prolongated downwards by
// ONE block, with a barrier per level instead of a kernel launch per level.
// Everything is brought in at the start by bulk copies (one per array, in
// flight together); the shared-memory layout is computed at setup.
// ---------------------------------------------------------------------------
constexpr int kTailMaxLevels = LAP_TAIL_MAX_LEVELS;

template <typename V> struct TailLevel {
    int nagg;                 // aggregates = vertices of the next level
    int loc;                  // offset of this level inside the tail
    const int *seg;
    const V *inv;
    const V *lcf;
    int seg_s, inv_s, lcf_s;  // byte offsets of the staged copies in shared memory
    int seg_b, inv_b, lcf_b;  // bytes copied (16-byte multiples, 0: none)
    V gamma;                  // restriction factor to the next level
    V dcoef;                  // down pass: out = pc * parent + dcoef * delta
};

template <typename V> struct TailParams {
    int nlev;                 // levels below the top inside the tail
    int ntail;                // vertices in the tail (all its levels)
    int ntop, loc_top;
    int64_t off0;             // expanded offset of the tail's first level
    int n0;                   // vertices of the tail's first level
    int sa_s, sz_s;           // byte offsets of the value arrays (sa: after its 16-byte head)
    int a0_head;              // bytes between the copy of A's first tail level and sa
    int smem;                 // shared-memory bytes of the launch
    const double *G;
    double top_scale;
    V pc;
    V *A;                     // global a/delta (expanded, tree order)
    V *Y;                     // global output (expanded, tree order)
    const V *F;               // expanded right-hand side added on restriction, or null
    int write_all;            // write every tail level of Y (else the first only)
    // finishing the first band's reductions: 0 none, 1 after the CG step
    // (iteration count, relative residual, convergence test), 2 without it;
    // fin_n per-block pairs (||r||^2, sum r) in fin_part.  3: the expanded-
    // space CG fused into the sweep: the step x += alpha p, r -= alpha q on
    // the tail's levels above its first (expanded vectors cx, cr, cp, cq; F
    // is cr), then as 1 over every band's pairs and the tail's own terms
    int fin, fin_n;
    const double *fin_part;
    V *cx = nullptr, *cr = nullptr;
    const V *cp = nullptr, *cq = nullptr;
    // >= 0 (with fin 3): sum z and r.z over the tail's levels to
    // xred_part[xred_slot], xred_part[xred_slot + 1]
    int xred_slot = -1;
    double *xred_part = nullptr;
    TailLevel<V> lev[kTailMaxLevels];
};

template <typename V>
__global__ void __launch_bounds__(1024)
k_msp_tail(const TailParams<V> P, CgScalars *sc)
{
    if (halted(sc)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int stop;
    V *sa = reinterpret_cast<V *>(smem_raw + P.sa_s);
    V *sz = reinterpret_cast<V *>(smem_raw + P.sz_s);
    const int tid = threadIdx.x, nth = blockDim.x;
    // the copies first: they do not depend on the step below
    if (tid == 0) {
        stop = 0;
        const uint32_t b = static_cast<uint32_t>(__cvta_generic_to_shared(&bar));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        const int a0_bytes = (P.a0_head + P.n0 * (int)sizeof(V) + 15) & ~15;
        uint32_t tx = a0_bytes;
        for (int k = 0; k < P.nlev; ++k) tx += P.lev[k].seg_b + P.lev[k].inv_b + P.lev[k].lcf_b;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(b), "r"(tx) : "memory");
        auto copy = [&](int dst, const void *src, int bytes) {
            if (bytes <= 0) return;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                    static_cast<uint32_t>(__cvta_generic_to_shared(smem_raw + dst))),
                "l"(src), "r"(bytes), "r"(b)
                : "memory");
        };
        copy(P.sa_s - P.a0_head, reinterpret_cast<const unsigned char *>(P.A + P.off0) - P.a0_head, a0_bytes);
        for (int k = 0; k < P.nlev; ++k) {
            const TailLevel<V> &L = P.lev[k];
            copy(L.seg_s, L.seg, L.seg_b);
            copy(L.inv_s, L.inv, L.inv_b);
            copy(L.lcf_s, L.lcf, L.lcf_b);
        }
    }
    if (P.fin) {
        // the first band's partials, summed in block order
        double v[2] = {0.0, 0.0};
        for (int b = threadIdx.x; b < P.fin_n; b += blockDim.x) {
            v[0] += P.fin_part[2 * b];
            v[1] += P.fin_part[2 * b + 1];
        }
        if (P.fin == 3) {
            // the CG step on the levels above the tail's first, four
            // elements per thread in flight
            const V al = (V)sc->alpha;
            const int nup = P.ntail - P.n0;
            const int64_t b0 = P.off0 + P.n0;
            for (int i0 = threadIdx.x; i0 < nup; i0 += 4 * (int)blockDim.x) {
                V xv[4], pv[4], qv[4], rv[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int i = i0 + k * (int)blockDim.x;
                    if (i < nup) {
                        xv[k] = P.cx[b0 + i];
                        pv[k] = P.cp[b0 + i];
                        qv[k] = P.cq[b0 + i];
                        rv[k] = P.cr[b0 + i];
                    }
                }
                // the four values and squares summed in V, then in FP64
                // (one SM's FP64 rate would dominate this block otherwise)
                V r2 = V(0), r1s = V(0);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int i = i0 + k * (int)blockDim.x;
                    if (i < nup) {
                        P.cx[b0 + i] = xv[k] + al * pv[k];
                        const V r1 = rv[k] - al * qv[k];
                        P.cr[b0 + i] = r1;
                        r2 += r1 * r1;
                        r1s += r1;
                    }
                }
                v[0] += (double)r2;
                v[1] += (double)r1s;
            }
        }
        block_sum<2>(v);
        if (threadIdx.x == 0) {
            sc->rr = v[0];
            sc->rs = v[1];
            if (P.fin == 1 || P.fin == 3) {
                finish_step(sc, v[0]);
            }
            stop = sc->flag != kRun;
        }
    }
    __syncthreads();
    {
        const uint32_t b = static_cast<uint32_t>(__cvta_generic_to_shared(&bar));
        const long long t0 = clock64();
        for (;;) {
            uint32_t done;
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(b)
                : "memory");
            if (done) break;
            if (clock64() - t0 > (1ll << 31)) {          // about a second: give up, flag it
                if (tid == 0 && sc) sc->flag = kBreakdown;
                return;
            }
        }
    }
    if (stop) return;                                   // converged: nothing to apply
    if (P.fin == 3) {
        // the updated r of the levels above the first, staged where the
        // elimination adds it (after the copies have landed)
        const int nup = P.ntail - P.n0;
        for (int i0 = tid; i0 < nup; i0 += 8 * nth) {
            V rv[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int i = i0 + k * nth;
                if (i < nup) rv[k] = P.cr[P.off0 + P.n0 + i];
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int i = i0 + k * nth;
                if (i < nup) sa[P.n0 + i] = rv[k];
            }
        }
        __syncthreads();
    }
    for (int k = 0; k < P.nlev; ++k) {
        const TailLevel<V> &L = P.lev[k];
        const int nloc = (k + 1 < P.nlev) ? P.lev[k + 1].loc : P.loc_top;
        // fin 3: a_{k+1} = gamma sum + (staged r_{k+1}) in place
        elim_level(sa + L.loc, sa + nloc, reinterpret_cast<const int *>(smem_raw + L.seg_s), 0,
                   reinterpret_cast<const V *>(smem_raw + L.inv_s), reinterpret_cast<const V *>(smem_raw + L.lcf_s),
                   L.gamma, P.fin == 3 ? static_cast<const V *>(sa + nloc) : P.F, P.fin == 3 ? 0 : P.off0 + nloc,
                   L.nagg, 0, nth);
        __syncthreads();
    }
    {   // top: dense pseudo-inverse, one warp per row
        const int lane = tid & 31, nw = nth >> 5;
        for (int row = tid >> 5; row < P.ntop; row += nw) {
            double s = 0.0;
            for (int j = lane; j < P.ntop; j += 32)
                s += P.G[(size_t)row * P.ntop + j] * (double)sa[P.loc_top + j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) sz[P.loc_top + row] = (V)(P.top_scale * s);
        }
    }
    __syncthreads();
    for (int k = P.nlev - 1; k >= 0; --k) {
        const TailLevel<V> &L = P.lev[k];
        const int nloc = (k + 1 < P.nlev) ? P.lev[k + 1].loc : P.loc_top;
        prolong_level(sz + L.loc, sa + L.loc, sz + nloc, reinterpret_cast<const int *>(smem_raw + L.seg_s), 0, P.pc,
                      L.dcoef, L.nagg, 0, nth);
        __syncthreads();
    }
    const int nout = P.write_all ? P.ntail : P.n0;
    for (int i = tid; i < nout; i += nth) P.Y[P.off0 + i] = sz[i];
    if (P.xred_slot >= 0) {
        // sum z and r.z over the tail's levels for the expanded-space CG
        double v[2] = {0.0, 0.0};
        for (int i0 = tid; i0 < P.ntail; i0 += 8 * nth) {
            V rv[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int i = i0 + k * nth;
                if (i < P.ntail) rv[k] = P.cr[P.off0 + i];
            }
            V a1 = V(0), a2 = V(0);             // eight terms in V, then FP64
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int i = i0 + k * nth;
                if (i < P.ntail) {
                    const V zv = sz[i];
                    a1 += zv;
                    a2 += rv[k] * zv;
                }
            }
            v[0] += (double)a1;
            v[1] += (double)a2;
        }
        block_sum<2>(v);
        if (tid == 0) {
            P.xred_part[P.xred_slot] = v[0];
            P.xred_part[P.xred_slot + 1] = v[1];
        }
    }
}

// Restriction of one level: s_{k+1}(J) = sum_{u in J} s_k(u); the scaled value
// coef * s_{k+1} goes to rt and (if given) to a.  Section 2.2: the level-k
// block of P(mu)^T r is (-mu)^(k-1) (P^k)^T r.
template <typename V>
__global__ void __launch_bounds__(kBlock)
k_restrict_level(int nagg, const int *__restrict__ seg, const V *__restrict__ s_in,
                 V *__restrict__ s_out, V *__restrict__ rt, V *__restrict__ a, V coef,
                 const CgScalars *sc)
{
    if (halted(sc)) return;
    for (int J = blockIdx.x * blockDim.x + threadIdx.x; J < nagg; J += gridDim.x * blockDim.x) {
        V sum = V(0);
        for (int u = seg[J]; u < seg[J + 1]; ++u) sum += s_in[u];
        s_out[J] = sum;
        const V v = coef * sum;
        if (rt) rt[J] = v;
        if (a) a[J] = v;
    }
}

// out1 = out2 = in (either output may be null)
template <typename V>
__global__ void __launch_bounds__(kBlock)
k_copy2(int64_t n, const V *__restrict__ in, V *__restrict__ o1, V *__restrict__ o2,
        const CgScalars *sc)
{
    if (halted(sc)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const V v = in[i];
        if (o1) o1[i] = v;
        if (o2) o2[i] = v;
    }
}

// Single-level hierarchy: z = G r directly (dense pseudo-inverse), with the
// same reductions as the finest tiled down pass.  One warp per row.
template <typename V>
__global__ void __launch_bounds__(kBlock)
k_dense_z(int n, const double *__restrict__ G, const V *__restrict__ r, const V *__restrict__ q,
          V *__restrict__ z, CgScalars *sc, double *part, unsigned *ticket)
{
    if (halted(sc)) return;
    const int lane = threadIdx.x & 31;
    const bool flex = sc->flexible && !sc->first;
    double sz = 0.0, srz = 0.0, szq = 0.0;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n; row += nw) {
        double s = 0.0;
        for (int j = lane; j < n; j += 32) s += G[(size_t)row * n + j] * (double)r[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const V zu = (V)s;
            z[row] = zu;
            sz += (double)zu;
            srz += (double)r[row] * (double)zu;
            if (flex) szq += (double)zu * (double)q[row];
        }
    }
    double v[3] = {sz, srz, szq};
    if (grid_sum<3>(v, part, ticket) && threadIdx.x == 0) {
        const double m = v[0] / (double)n;
        set_direction(sc, m, v[1] - m * sc->rs, v[2]);
    }
}

// p.q and sum q of a direction p and its product q = A p, and the step length
// alpha = rho / p.q (as the matvec's MODE 0 epilogue, for a matvec launched
// without reductions): groups of four in V, then FP64.
template <typename V>
__global__ void __launch_bounds__(kBlock)
k_pq(int64_t n, const V *__restrict__ p, const V *__restrict__ q, CgScalars *sc, double *part, unsigned *ticket)
{
    if (halted(sc)) return;
    double a0 = 0.0, a1 = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
        V pv[4], qv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = i0 + k * stride;
            pv[k] = i < n ? p[i] : V(0);
            qv[k] = i < n ? q[i] : V(0);
        }
        V s0 = V(0), s1 = V(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            s0 += pv[k] * qv[k];
            s1 += qv[k];
        }
        a0 += (double)s0;
        a1 += (double)s1;
    }
    double v[2] = {a0, a1};
    if (grid_sum<2>(v, part, ticket) && threadIdx.x == 0) {
        sc->pq = v[0];
        sc->qsum = v[1];
        const double alpha = sc->rho / v[0];
        if (!(v[0] > 0.0) || !isfinite(alpha)) sc->flag = kBreakdown;
        sc->alpha = alpha;
    }
}

// p = (z - zmean) + beta p
template <typename V>
__global__ void __launch_bounds__(kBlock)
k_pupdate(int64_t n, const V *__restrict__ z, V *__restrict__ p, const CgScalars *sc)
{
    if (halted(sc)) return;
    const V m = (V)sc->zmean, be = (V)sc->beta;
    // a fresh direction (beta == 0) never reads the previous p
    if (be == V(0)) {
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            p[i] = z[i] - m;
        return;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (z[i] - m) + be * p[i];
}

// ---------------------------------------------------------------------------
// Permutation between the caller's numbering and tree order, projection.
// ---------------------------------------------------------------------------
// out[i] = (V) in[perm[i]], reduce sum -> sc->bmean = sum / n
template <typename V>
__global__ void __launch_bounds__(kBlock)
k_gather_sum(int n, const int *__restrict__ perm, const double *__restrict__ in, V *__restrict__ out,
             CgScalars *sc, double *part, unsigned *ticket)
{
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = in[perm ? perm[i] : i];
        out[i] = (V)v;
        s += v;
    }
    double v[1] = {s};
    if (grid_sum<1>(v, part, ticket) && threadIdx.x == 0) sc->bmean = v[0] / (double)n;
}

// b -= bmean (double, in place), r = (V) b, x = 0; reduce ||b||^2 and sum(r) ->
// bnorm, rr, rs; converged at once when b projects to zero.
template <typename V>
__global__ void __launch_bounds__(kBlock)
k_center_init(int n, double *__restrict__ b, V *__restrict__ r, V *__restrict__ x, CgScalars *sc,
              double *part, unsigned *ticket)
{
    const double m = sc->bmean;
    double s2 = 0.0, s1 = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = b[i] - m;
        b[i] = v;
        const V rv = (V)v;
        r[i] = rv;
        if (x) x[i] = V(0);
        s2 += (double)rv * (double)rv;
        s1 += (double)rv;
    }
    double v[2] = {s2, s1};
    if (grid_sum<2>(v, part, ticket) && threadIdx.x == 0) {
        sc->bnorm = sqrt(v[0]);
        sc->rr = v[0];
        sc->rs = v[1];
        sc->relres = 1.0;
        sc->iter = 0;
        sc->first = 1;
        sc->flag = (v[0] > 0.0) ? kRun : kConverged;
    }
}

// mean of x -> sc->tmp
template <typename V>
__global__ void __launch_bounds__(kBlock)
k_mean(int n, const V *__restrict__ x, CgScalars *sc, double *part, unsigned *ticket)
{
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s += (double)x[i];
    double v[1] = {s};
    if (grid_sum<1>(v, part, ticket) && threadIdx.x == 0) sc->tmp = v[0] / (double)n;
}

// out[perm[i]] = x[i] - *shift  (back to the caller's numbering; shift may be null)
template <typename V>
__global__ void __launch_bounds__(kBlock)
k_scatter_shift(int n, const int *__restrict__ perm, const V *__restrict__ x, double *__restrict__ out,
                const double *shift)
{
    const double m = shift ? *shift : 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[perm ? perm[i] : i] = (double)x[i] - m;
}

// out[i] = (V) in[perm[i]]
template <typename V>
__global__ void __launch_bounds__(kBlock)
k_gather(int n, const int *__restrict__ perm, const double *__restrict__ in, V *__restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = (V)in[perm ? perm[i] : i];
}

// x = 0; reduce ||r||^2, sum r -> bnorm, rr, rs; start a CG (expanded-space inner solve)
// (a stopped CG, e.g. gated by k_inner_reset, is left as it is)
template <typename V>
__global__ void __launch_bounds__(kBlock)
k_vec_init(int64_t n, const V *__restrict__ r, V *__restrict__ x, CgScalars *sc, double *part,
           unsigned *ticket)
{
    if (halted(sc)) return;
    double s2 = 0.0, s1 = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
        V a2 = V(0), a1 = V(0);            // groups of four in V, then FP64
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = i0 + k * stride;
            if (i < n) {
                const V v = r[i];
                x[i] = V(0);
                a2 += v * v;
                a1 += v;
            }
        }
        s2 += (double)a2;
        s1 += (double)a1;
    }
    double v[2] = {s2, s1};
    if (grid_sum<2>(v, part, ticket) && threadIdx.x == 0) {
        sc->bnorm = sqrt(v[0]);
        sc->rr = v[0];
        sc->rs = v[1];
        sc->relres = 1.0;
        sc->iter = 0;
        sc->first = 1;
        sc->flag = (v[0] > 0.0) ? kRun : kConverged;
    }
}

// Reductions of a flat preconditioned residual z (expanded-space CG):
// sum z, r.z -> zmean, rho, beta (standard CG).
template <typename V>
__global__ void __launch_bounds__(kBlock)
k_zred(int64_t n, const V *__restrict__ z, const V *__restrict__ r, CgScalars *sc, double *part,
       unsigned *ticket)
{
    if (halted(sc)) return;
    double sz = 0.0, srz = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double zu = (double)z[i];
        sz += zu;
        srz += (double)r[i] * zu;
    }
    double v[2] = {sz, srz};
    if (grid_sum<2>(v, part, ticket) && threadIdx.x == 0) {
        const double m = v[0] / (double)n;
        set_direction(sc, m, v[1] - m * sc->rs, 0.0);
    }
}

// CG bookkeeping written from the host side of the stream.
static __global__ void k_cg_reset(CgScalars *sc, double tol, int maxit, int flexible, double *hist,
                                  int hist_cap, double *lz = nullptr)
{
    sc->inner_total = 0;
    sc->tol = tol;
    sc->maxit = maxit;
    sc->flexible = flexible;
    sc->iter = 0;
    sc->flag = kRun;
    sc->first = 1;
    sc->hist = hist;
    sc->hist_cap = hist ? hist_cap : 0;
    sc->lz = hist ? lz : nullptr;
}

// scalars for timing runs: running, never converging, unit norms
// Fixed values in [-1, 1) for timing runs (a hash of the index; not random
// numbers of the method).
template <typename V>
__global__ void k_bench_fill(int64_t n, V *v, uint32_t salt)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = static_cast<uint32_t>(i) * 2654435761u ^ salt;
        h ^= h >> 15;
        h *= 2246822519u;
        h ^= h >> 13;
        v[i] = static_cast<V>(static_cast<double>(h) * (2.0 / 4294967296.0) - 1.0);
    }
}

static __global__ void k_bench_scalars(CgScalars *sc)
{
    sc->tol = -1.0;                 // never met, even by a zero residual
    sc->maxit = 0x7fffffff;
    sc->flexible = 0;
    sc->iter = 0;
    sc->flag = kRun;
    sc->first = 0;
    sc->bnorm = 1.0;
    sc->rho = 1.0;
    sc->alpha = 0.0;
    sc->beta = 0.0;
    sc->zmean = 0.0;
    sc->hist = nullptr;
    sc->hist_cap = 0;
    sc->lz = nullptr;
}

// Start of a PEGP inner solve sequenced on the device: the inner CG's
// bookkeeping as k_cg_reset, already stopped if the outer CG is not running
// (its step just converged, broke down or reached maxit), so that the whole
// inner solve and the prolongation after it return at once.
static __global__ void k_inner_reset(CgScalars *inner, const CgScalars *outer, double tol, int maxit)
{
    inner->tol = tol;
    inner->maxit = maxit;
    inner->flexible = 0;
    inner->iter = 0;
    inner->first = 1;
    inner->hist = nullptr;
    inner->hist_cap = 0;
    inner->lz = nullptr;
    inner->flag = outer->flag == kRun ? kRun : kConverged;
}

// The inner solve's iterations added to the outer CG's tally.
static __global__ void k_inner_tally(const CgScalars *inner, CgScalars *outer)
{
    if (outer->flag == kRun) outer->inner_total += inner->iter;
}

static __global__ void k_cg_restart(CgScalars *sc)
{
    sc->flag = kRun;
    sc->first = 1;
}

// x64 += (double) d  (iterative refinement correction)
template <typename V>
__global__ void __launch_bounds__(kBlock)
k_add_correction(int n, double *__restrict__ x, const V *__restrict__ d)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        x[i] += (double)d[i];
}

// out[i] = (VO) in[i]
template <typename VI, typename VO>
__global__ void __launch_bounds__(kBlock)
k_convert(int64_t n, const VI *__restrict__ in, VO *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (VO)in[i];
}

// plain gather/scatter by a permutation (expanded-space building blocks)
template <typename V>
__global__ void __launch_bounds__(kBlock)
k_permute(int64_t n, const int64_t *__restrict__ idx, const V *__restrict__ in, V *__restrict__ out,
          int scatter)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (scatter) out[idx[i]] = in[i];
        else out[i] = in[idx[i]];
    }
}

}  // namespace lap
