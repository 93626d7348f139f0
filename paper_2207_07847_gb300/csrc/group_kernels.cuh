// Kernels of a solve group: many graphs of uneven size solved together, each
// with its own right-hand sides, in one launch per phase of the PCG.
//
// The graphs are merged block-diagonally.  Every level of the merged
// hierarchy holds the level's vertices of every graph that has that level,
// graphs ordered by decreasing depth, so that on each level the graphs that
// aggregate further form a prefix: one segment array per level covers them,
// in merged indices, and the per-aggregate pair and leftover coefficients
// are the graphs' own arrays concatenated (see group.cu).  Block vectors are
// row-major over the merged vertices ([vertex][R], as the batched kernels).
//
// Each (graph, column) runs its own CG: its scalars live in col[g R + c].
// Reductions are per graph: kernels that reduce run on a grid of
// (blocks, graphs); block (bx, g) covers work items of graph g only
// (GRange: the graph's items [lo, hi) and the nb blocks sharing them), and
// the last of graph g's blocks (a per-graph ticket) adds the block partials
// in block order.  Elementwise kernels look a row's graph up in gid[].
#pragma once

#include "batched_kernels.cuh"

namespace lap {

struct GRange {
    int lo, hi;      // work items of this graph in the launch (merged indices)
    int nb;          // blocks of the graph (blockIdx.x < nb)
    int pad;
};

// Per-graph reduction over the graph's nb blocks: the same steps as
// bcol_reduce, with the graph's partials, ticket and block count.
template <int NV, int MAXJ>
__device__ __forceinline__ bool gcol_reduce(double (&acc)[NV][MAXJ], int R, int CT, int bx, int nb, double *part,
                                            unsigned *ticket, double *tot)
{
    __shared__ double red[kBThreads];
    __shared__ bool last;
    const int tid = threadIdx.x;
    const int S = kBThreads / CT;
    const int o = tid / CT, cl = tid % CT;
    const int nj = R / CT;
    for (int q = 0; q < NV; ++q) {
        for (int j = 0; j < nj; ++j) {
            red[tid] = acc[q][j];
            __syncthreads();
            for (int s = S / 2; s > 0; s >>= 1) {
                if (o < s) red[tid] += red[tid + s * CT];
                __syncthreads();
            }
            if (o == 0) part[((size_t)bx * NV + q) * R + cl + j * CT] = red[tid];
            __syncthreads();
        }
    }
    if (tid == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == static_cast<unsigned>(nb - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    for (int idx = tid; idx < NV * R; idx += kBThreads) {
        const int q = idx / R, c = idx % R;
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += __ldcg(part + ((size_t)b * NV + q) * R + c);
        tot[idx] = s;
    }
    __syncthreads();
    if (tid == 0) *ticket = 0u;
    return true;
}

// The graph's slice of the reduction scratch: nbmax blocks x NV x R doubles.
__device__ __forceinline__ double *gpart(double *part, int g, int nbmax, int NV, int R)
{
    return part + (size_t)g * nbmax * NV * R;
}

// Gather the caller's column-major B_g (one device pointer per graph) into
// the merged tree order; per-column sums -> bmean.
__global__ void __launch_bounds__(kBThreads)
kg_gather(int R, int CT, const GRange *__restrict__ rows, const int *__restrict__ nrhs,
          const int *__restrict__ perm, const double *const *__restrict__ B, double *__restrict__ Bs,
          BCol *col, double *part, int nbmax, unsigned *ticket)
{
    const int g = blockIdx.y;
    const GRange rg = rows[g];
    if ((int)blockIdx.x >= rg.nb) return;
    __shared__ double tot[256];
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    const int ng = rg.hi - rg.lo, nr = nrhs[g];
    const double *Bg = B[g];
    double acc[1][8];
    for (int j = 0; j < 8; ++j) acc[0][j] = 0.0;
    for (int i = rg.lo + blockIdx.x * S + o; i < rg.hi; i += rg.nb * S) {
        const int src = perm[i];
        for (int j = 0; j < R / CT; ++j) {
            const int c = cl + j * CT;
            const double v = c < nr ? Bg[(size_t)c * ng + src] : 0.0;
            Bs[(size_t)i * R + c] = v;
            acc[0][j] += v;
        }
    }
    if (gcol_reduce<1, 8>(acc, R, CT, blockIdx.x, rg.nb, gpart(part, g, nbmax, 1, R), ticket + g, tot))
        for (int c = threadIdx.x; c < R; c += kBThreads) col[g * R + c].bmean = tot[c] / (double)ng;
}

// Start every (graph, column) CG: as kb_center per graph (subtract the
// column means, r = (V) v, x = 0, ||r||^2 and sum r); with `outer`
// (refinement) only columns still running there start.
template <typename V>
__global__ void __launch_bounds__(kBThreads)
kg_center(int R, int CT, const GRange *__restrict__ rows, const int *__restrict__ nrhs, int subtract,
          double *__restrict__ src, V *__restrict__ r, V *__restrict__ x, const BCol *meancol, BCol *col,
          double tol, int maxit, const BCol *outer, double refine_tol, double *part, int nbmax,
          unsigned *ticket)
{
    const int g = blockIdx.y;
    const GRange rg = rows[g];
    if ((int)blockIdx.x >= rg.nb) return;
    __shared__ double tot[512];
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    const BCol *mc = meancol + g * R;
    const BCol *oc = outer ? outer + g * R : nullptr;
    double acc[2][8];
    for (int j = 0; j < 8; ++j) acc[0][j] = acc[1][j] = 0.0;
    for (int i = rg.lo + blockIdx.x * S + o; i < rg.hi; i += rg.nb * S) {
        for (int j = 0; j < R / CT; ++j) {
            const int c = cl + j * CT;
            const size_t k = (size_t)i * R + c;
            double v = src[k];
            if (subtract) {
                v -= mc[c].bmean;
                src[k] = v;
            }
            if (oc && oc[c].flag != kRun) v = 0.0;
            const V rv = (V)v;
            r[k] = rv;
            if (x) x[k] = V(0);
            acc[0][j] += (double)rv * (double)rv;
            acc[1][j] += (double)rv;
        }
    }
    if (gcol_reduce<2, 8>(acc, R, CT, blockIdx.x, rg.nb, gpart(part, g, nbmax, 2, R), ticket + g, tot)) {
        for (int c = threadIdx.x; c < R; c += kBThreads) {
            BCol &C = col[g * R + c];
            C.bnorm = sqrt(tot[c]);
            C.rr = tot[c];
            C.rs = tot[R + c];
            C.relres = 1.0;
            C.iter = 0;
            C.first = 1;
            C.maxit = maxit;
            C.tol = oc ? fmin(0.5, fmax(refine_tol, 0.3 * tol / oc[c].relres)) : tol;
            const bool run = c < nrhs[g] && tot[c] > 0.0 && (!oc || oc[c].flag == kRun);
            C.flag = run ? kRun : kConverged;
        }
    }
}

// Refinement bookkeeping of every (graph, column).
static __global__ void kg_refine_flags(int G, int R, const int *__restrict__ nrhs, BCol *col, double tol)
{
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < G * R; idx += gridDim.x * blockDim.x) {
        const int g = idx / R, c = idx % R;
        BCol &C = col[idx];
        if (C.flag == kRun && (c >= nrhs[g] || C.relres <= tol)) C.flag = kConverged;
        if (C.flag == kRun && !isfinite(C.relres)) C.flag = kBreakdown;
    }
}

// SpMM y = L x over the merged CSR (edge-difference form).  MODE 0: p.q and
// sum q per (graph, column) -> alpha; MODE 1: yres = Bs - L x, ||.||^2 and
// sum -> true relative residual; MODE 2: no reduction.
template <typename V, int MODE>
__global__ void __launch_bounds__(kBThreads)
kg_spmm(int R, int CT, const GRange *__restrict__ rows, const int *__restrict__ rp, const int *__restrict__ ci,
        const V *__restrict__ w, const V *__restrict__ x, V *__restrict__ y, const double *__restrict__ Bs,
        double *__restrict__ yres, BCol *col, double *part, int nbmax, unsigned *ticket)
{
    const int g = blockIdx.y;
    const GRange rg = rows[g];
    if ((int)blockIdx.x >= rg.nb) return;
    __shared__ double tot[512];
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    double acc[2][8];
    for (int j = 0; j < 8; ++j) acc[0][j] = acc[1][j] = 0.0;
    for (int i = rg.lo + blockIdx.x * S + o; i < rg.hi; i += rg.nb * S) {
        const int b = rp[i], e = rp[i + 1];
        for (int j = 0; j < R / CT; ++j) {
            const int c = cl + j * CT;
            const size_t k = (size_t)i * R + c;
            const V xi = x[k];
            V s = V(0);
            for (int p = b; p < e; ++p) s += w[p] * (xi - x[(size_t)ci[p] * R + c]);
            if (MODE == 1) {
                const double rv = Bs[k] - (double)s;
                yres[k] = rv;
                acc[0][j] += rv * rv;
                acc[1][j] += rv;
            } else {
                y[k] = s;
                if (MODE == 0) {
                    acc[0][j] += (double)xi * (double)s;
                    acc[1][j] += (double)s;
                }
            }
        }
    }
    if (MODE == 2) return;
    if (gcol_reduce<2, 8>(acc, R, CT, blockIdx.x, rg.nb, gpart(part, g, nbmax, 2, R), ticket + g, tot)) {
        for (int c = threadIdx.x; c < R; c += kBThreads) {
            BCol &C = col[g * R + c];
            if (MODE == 0) {
                if (C.flag != kRun) continue;
                C.pq = tot[c];
                C.qs = tot[R + c];
                C.alpha = C.rho / tot[c];
                if (!(tot[c] > 0.0) || !isfinite(C.alpha)) C.flag = kBreakdown;
            } else if (C.bnorm > 0.0) {
                C.rr = tot[c];
                C.rs = tot[R + c];
                C.relres = sqrt(tot[c]) / C.bnorm;
            }
        }
    }
}

// Elimination of one aggregate on column c of the block vectors (Section
// 3.3, as agg_eliminate): returns the sum of its right-hand sides; writes the
// members' deltas to dout.
template <typename V>
__device__ __forceinline__ V g_eliminate(const V *__restrict__ r, V *__restrict__ dout, int b0, int e, const V *cf,
                                         const V *lc, int R, int c)
{
    const V aa = r[(size_t)b0 * R + c], ab = r[(size_t)(b0 + 1) * R + c];
    V sum = aa + ab, ha = aa, hb = ab;
    for (int t = b0 + 2; t < e; ++t) {
        const V al = r[(size_t)t * R + c];
        const V *cc = lc + 3 * (t - b0 - 2);
        sum += al;
        ha += cc[0] * al;
        hb += cc[1] * al;
    }
    V da, db;
    pair_solve(cf, ha, hb, da, db);
    for (int t = b0 + 2; t < e; ++t) {
        const V *cc = lc + 3 * (t - b0 - 2);
        dout[(size_t)t * R + c] = r[(size_t)t * R + c] * cc[2] + cc[0] * da + cc[1] * db;
    }
    dout[(size_t)b0 * R + c] = da;
    dout[(size_t)(b0 + 1) * R + c] = db;
    return sum;
}

// Upward pass of one merged level (all graphs that aggregate on it).  MODE 0
// (a level above the finest): one grid over all the level's aggregates, in
// place (a -> delta), anext = gamma * sum.  MODE 1 (finest, with the CG step
// x += alpha p, r -= alpha q of every running column) and MODE 2 (finest,
// no step): per-graph blocks and ||r||^2, sum r per (graph, column), the
// step's convergence test.
template <typename V, int MODE>
__global__ void __launch_bounds__(kBThreads)
kg_up(int nagg_all, int R, int CT, const GRange *__restrict__ aggs, const int *__restrict__ seg,
      const V *__restrict__ inv, const V *__restrict__ lcf, V *__restrict__ x, V *r, const V *__restrict__ p,
      const V *__restrict__ q, V *dout, V *anext, V gamma, BCol *col, double *part, int nbmax, unsigned *ticket)
{
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    if (MODE == 0) {
        for (int J = blockIdx.x * S + o; J < nagg_all; J += gridDim.x * S) {
            const int b0 = seg[J], e = seg[J + 1];
            for (int jj = 0; jj < R / CT; ++jj) {
                const int c = cl + jj * CT;
                const V sum = g_eliminate(r, dout, b0, e, inv + 4 * J, lcf + 3 * (b0 - 2 * J), R, c);
                anext[(size_t)J * R + c] = gamma * sum;
            }
        }
        return;
    }
    const int g = blockIdx.y;
    const GRange ra = aggs[g];
    if ((int)blockIdx.x >= ra.nb) return;
    __shared__ double tot[512];
    BCol *cg = col + g * R;
    double acc[2][8];
    for (int j = 0; j < 8; ++j) acc[0][j] = acc[1][j] = 0.0;
    for (int J = ra.lo + blockIdx.x * S + o; J < ra.hi; J += ra.nb * S) {
        const int b0 = seg[J], e = seg[J + 1];
        for (int jj = 0; jj < R / CT; ++jj) {
            const int c = cl + jj * CT;
            if (MODE == 1 && bactive(cg, c)) {
                const V al = (V)cg[c].alpha;
                for (int u = b0; u < e; ++u) {
                    const size_t k = (size_t)u * R + c;
                    x[k] += al * p[k];
                    r[k] -= al * q[k];
                }
            }
            for (int u = b0; u < e; ++u) {
                const double v = (double)r[(size_t)u * R + c];
                acc[0][jj] += v * v;
                acc[1][jj] += v;
            }
            const V sum = g_eliminate(r, dout, b0, e, inv + 4 * J, lcf + 3 * (b0 - 2 * J), R, c);
            anext[(size_t)J * R + c] = gamma * sum;
        }
    }
    if (gcol_reduce<2, 8>(acc, R, CT, blockIdx.x, ra.nb, gpart(part, g, nbmax, 2, R), ticket + g, tot)) {
        for (int c = threadIdx.x; c < R; c += kBThreads) {
            BCol &C = cg[c];
            if (C.flag != kRun) continue;
            C.rr = tot[c];
            C.rs = tot[R + c];
            if (MODE == 1) {
                C.iter += 1;
                const double rel = sqrt(tot[c]) / C.bnorm;
                C.relres = rel;
                if (!isfinite(rel)) C.flag = kBreakdown;
                else if (rel <= C.tol) C.flag = kConverged;
                else if (C.iter >= C.maxit) C.flag = kMaxit;
            }
        }
    }
}

// Every graph's top level: Y(i, c) = c_top(g) * sum_k G_g(i, k) A(k, c) with
// the graph's dense pseudo-inverse (FP64 accumulation); block row g.
template <typename V>
__global__ void __launch_bounds__(kBThreads)
kg_coarse(int R, const int *__restrict__ top_row, const int *__restrict__ ntop, const double *const *__restrict__ Gs,
          const double *__restrict__ scale, const V *__restrict__ A, V *__restrict__ Y)
{
    const int g = blockIdx.y;
    const int m = ntop[g];
    const double *G = Gs[g];
    const size_t base = (size_t)top_row[g] * R;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < m * R; idx += gridDim.x * blockDim.x) {
        const int i = idx / R, c = idx % R;
        double s = 0.0;
        for (int k = 0; k < m; ++k) s += G[(size_t)i * m + k] * (double)A[base + (size_t)k * R + c];
        Y[base + idx] = (V)(scale[g] * s);
    }
}

// Downward pass of one merged level: out(u, c) = pc * parent(J, c) + dc *
// delta(u, c).  Not FINEST: one grid over all aggregates.  FINEST: per-graph
// blocks, and sum z, r.z per (graph, column) finalise zmean, rho, beta
// (n_of[g]: the graph's vertex count).
template <typename V, bool FINEST>
__global__ void __launch_bounds__(kBThreads)
kg_down(int nagg_all, int R, int CT, const GRange *__restrict__ aggs, const int *__restrict__ n_of,
        const int *__restrict__ seg, const V *__restrict__ delta, const V *__restrict__ parent, V *__restrict__ out,
        V pc, V dc, const V *__restrict__ r, BCol *col, double *part, int nbmax, unsigned *ticket)
{
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    if (!FINEST) {
        for (int J = blockIdx.x * S + o; J < nagg_all; J += gridDim.x * S)
            for (int jj = 0; jj < R / CT; ++jj) {
                const int c = cl + jj * CT;
                const V base = pc * parent[(size_t)J * R + c];
                for (int u = seg[J]; u < seg[J + 1]; ++u) out[(size_t)u * R + c] = base + dc * delta[(size_t)u * R + c];
            }
        return;
    }
    const int g = blockIdx.y;
    const GRange ra = aggs[g];
    if ((int)blockIdx.x >= ra.nb) return;
    __shared__ double tot[512];
    BCol *cg = col + g * R;
    double acc[2][8];
    for (int j = 0; j < 8; ++j) acc[0][j] = acc[1][j] = 0.0;
    for (int J = ra.lo + blockIdx.x * S + o; J < ra.hi; J += ra.nb * S) {
        for (int jj = 0; jj < R / CT; ++jj) {
            const int c = cl + jj * CT;
            const V base = pc * parent[(size_t)J * R + c];
            for (int u = seg[J]; u < seg[J + 1]; ++u) {
                const size_t k = (size_t)u * R + c;
                const V z = base + dc * delta[k];
                out[k] = z;
                acc[0][jj] += (double)z;
                acc[1][jj] += (double)r[k] * (double)z;
            }
        }
    }
    if (gcol_reduce<2, 8>(acc, R, CT, blockIdx.x, ra.nb, gpart(part, g, nbmax, 2, R), ticket + g, tot)) {
        for (int c = threadIdx.x; c < R; c += kBThreads) {
            BCol &C = cg[c];
            if (C.flag != kRun) continue;
            const double m = tot[c] / (double)n_of[g];
            const double rho_new = tot[R + c] - m * C.rs;
            C.zmean = m;
            C.beta = C.first ? 0.0 : rho_new / C.rho;
            C.rho = rho_new;
            C.first = 0;
            if (!isfinite(rho_new)) C.flag = kBreakdown;
        }
    }
}

// Plain CG of every (graph, column): the step and z = Pi r statistics.
template <typename V, bool UPDATE>
__global__ void __launch_bounds__(kBThreads)
kg_plain(int R, int CT, const GRange *__restrict__ rows, V *__restrict__ x, V *__restrict__ r,
         const V *__restrict__ p, const V *__restrict__ q, BCol *col, double *part, int nbmax, unsigned *ticket)
{
    const int g = blockIdx.y;
    const GRange rg = rows[g];
    if ((int)blockIdx.x >= rg.nb) return;
    __shared__ double tot[512];
    BCol *cg = col + g * R;
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    double acc[2][8];
    for (int j = 0; j < 8; ++j) acc[0][j] = acc[1][j] = 0.0;
    for (int i = rg.lo + blockIdx.x * S + o; i < rg.hi; i += rg.nb * S) {
        for (int jj = 0; jj < R / CT; ++jj) {
            const int c = cl + jj * CT;
            const size_t k = (size_t)i * R + c;
            V rv = r[k];
            if (UPDATE && bactive(cg, c)) {
                const V al = (V)cg[c].alpha;
                x[k] += al * p[k];
                rv -= al * q[k];
                r[k] = rv;
            }
            acc[0][jj] += (double)rv * rv;
            acc[1][jj] += (double)rv;
        }
    }
    if (gcol_reduce<2, 8>(acc, R, CT, blockIdx.x, rg.nb, gpart(part, g, nbmax, 2, R), ticket + g, tot)) {
        const double n = (double)(rg.hi - rg.lo);
        for (int c = threadIdx.x; c < R; c += kBThreads) {
            BCol &C = cg[c];
            if (C.flag != kRun) continue;
            C.rr = tot[c];
            C.rs = tot[R + c];
            if (UPDATE) {
                C.iter += 1;
                const double rel = sqrt(tot[c]) / C.bnorm;
                C.relres = rel;
                if (!isfinite(rel)) C.flag = kBreakdown;
                else if (rel <= C.tol) C.flag = kConverged;
                else if (C.iter >= C.maxit) C.flag = kMaxit;
            }
            if (C.flag == kRun) {
                const double m = tot[R + c] / n;
                const double rho_new = tot[c] - m * tot[R + c];
                C.zmean = m;
                C.beta = C.first ? 0.0 : rho_new / C.rho;
                C.rho = rho_new;
                C.first = 0;
            }
        }
    }
}

// p = (z - zmean) + beta p for the running (graph, column) pairs; the row's
// graph from gid.
template <typename V>
__global__ void __launch_bounds__(kBThreads)
kg_pupdate(int n, int R, int CT, const int *__restrict__ gid, const V *__restrict__ z, V *__restrict__ p,
           const BCol *col)
{
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    for (int i = blockIdx.x * S + o; i < n; i += gridDim.x * S) {
        const BCol *cg = col + gid[i] * R;
        for (int jj = 0; jj < R / CT; ++jj) {
            const int c = cl + jj * CT;
            if (!bactive(cg, c)) continue;
            const size_t k = (size_t)i * R + c;
            const V m = (V)cg[c].zmean, be = (V)cg[c].beta;
            p[k] = be == V(0) ? z[k] - m : (z[k] - m) + be * p[k];
        }
    }
}

// Per-(graph, column) mean of x, then the scatter to each graph's
// column-major output with the projection.
template <typename V>
__global__ void __launch_bounds__(kBThreads)
kg_mean(int R, int CT, const GRange *__restrict__ rows, const V *__restrict__ x, double *__restrict__ means,
        double *part, int nbmax, unsigned *ticket)
{
    const int g = blockIdx.y;
    const GRange rg = rows[g];
    if ((int)blockIdx.x >= rg.nb) return;
    __shared__ double tot[256];
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    double acc[1][8];
    for (int j = 0; j < 8; ++j) acc[0][j] = 0.0;
    for (int i = rg.lo + blockIdx.x * S + o; i < rg.hi; i += rg.nb * S)
        for (int jj = 0; jj < R / CT; ++jj) acc[0][jj] += (double)x[(size_t)i * R + cl + jj * CT];
    if (gcol_reduce<1, 8>(acc, R, CT, blockIdx.x, rg.nb, gpart(part, g, nbmax, 1, R), ticket + g, tot))
        for (int c = threadIdx.x; c < R; c += kBThreads) means[g * R + c] = tot[c] / (double)(rg.hi - rg.lo);
}

template <typename V>
__global__ void __launch_bounds__(kBThreads)
kg_scatter(int R, int CT, const GRange *__restrict__ rows, const int *__restrict__ nrhs,
           const int *__restrict__ perm, const V *__restrict__ x, const double *__restrict__ means,
           double *const *__restrict__ X)
{
    const int g = blockIdx.y;
    const GRange rg = rows[g];
    if ((int)blockIdx.x >= rg.nb) return;
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    const int ng = rg.hi - rg.lo, nr = nrhs[g];
    double *Xg = X[g];
    for (int i = rg.lo + blockIdx.x * S + o; i < rg.hi; i += rg.nb * S) {
        const int dst = perm[i];
        for (int jj = 0; jj < R / CT; ++jj) {
            const int c = cl + jj * CT;
            if (c < nr) Xg[(size_t)c * ng + dst] = (double)x[(size_t)i * R + c] - means[g * R + c];
        }
    }
}

}  // namespace lap
