// Kernels of the batched (many right-hand sides) preconditioned CG.
//
// Block vectors are row-major: entry (vertex i, column c) at i * R + c, R a
// power of two <= 256, so the R values of one vertex are contiguous.  A
// thread block of 256 threads is laid out as S = 256 / CT row groups times CT
// columns (CT <= R, the column tile; a block covers column tiles in turn):
// every CSR index and weight is loaded once per row group and broadcast, and
// every gather of a neighbour's values is a contiguous run of CT values.
// Every column runs its own CG: its scalars live in BCol[c] and a converged
// column is frozen (its x, r, p are no longer written).
#pragma once

#include "kernels.cuh"

namespace lap {

struct BCol {
    double rho, alpha, beta, zmean, pq, qs, rr, rs, bnorm, relres, tol, bmean;
    int iter, flag, first, maxit;
    int join;          // 1 while a newly admitted column waits for its first direction
    int pad;
};

constexpr int kBThreads = 256;

// ---------------------------------------------------------------------------
// Reduction helper used by every batched kernel: each thread holds partial
// sums acc[NV][j] for the columns c = c0 + j * CT (j < R / CT) it visited.
// ---------------------------------------------------------------------------
template <int NV, int MAXJ>
__device__ __forceinline__ bool bcol_reduce(double (&acc)[NV][MAXJ], int R, int CT, double *part,
                                            unsigned *ticket, double *tot /* [NV][R] smem */)
{
    __shared__ double red[kBThreads];
    __shared__ bool last;
    const int tid = threadIdx.x;
    const int S = kBThreads / CT;
    const int o = tid / CT, cl = tid % CT;
    const int nj = R / CT;
    // reduce over row groups: column c = cl + j * CT
    for (int q = 0; q < NV; ++q) {
        for (int j = 0; j < nj; ++j) {
            red[tid] = acc[q][j];
            __syncthreads();
            for (int s = S / 2; s > 0; s >>= 1) {
                if (o < s) red[tid] += red[tid + s * CT];
                __syncthreads();
            }
            if (o == 0) part[((size_t)blockIdx.x * NV + q) * R + cl + j * CT] = red[tid];
            __syncthreads();
        }
    }
    if (tid == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    for (int idx = tid; idx < NV * R; idx += kBThreads) {
        const int q = idx / R, c = idx % R;
        double s = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(part + ((size_t)b * NV + q) * R + c);
        tot[idx] = s;
    }
    __syncthreads();
    if (tid == 0) *ticket = 0u;
    return true;
}

__device__ __forceinline__ bool bactive(const BCol *col, int c) { return col[c].flag == kRun; }

// ---------------------------------------------------------------------------
// Gather the caller's column-major B into tree order and sum each column.
// ---------------------------------------------------------------------------
template <typename V>
__global__ void __launch_bounds__(kBThreads)
kb_gather(int n, int R, int CT, int nrhs, const int *__restrict__ perm, const double *__restrict__ B,
          double *__restrict__ Bs, BCol *col, double *part, unsigned *ticket)
{
    __shared__ double tot[256];
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    double acc[1][8];
    for (int j = 0; j < 8; ++j) acc[0][j] = 0.0;
    for (int i = blockIdx.x * S + o; i < n; i += gridDim.x * S) {
        const int src = perm[i];
        for (int j = 0; j < R / CT; ++j) {
            const int c = cl + j * CT;
            const double v = c < nrhs ? B[(size_t)c * n + src] : 0.0;
            Bs[(size_t)i * R + c] = v;
            acc[0][j] += v;
        }
    }
    if (bcol_reduce<1, 8>(acc, R, CT, part, ticket, tot)) {
        for (int c = threadIdx.x; c < R; c += kBThreads) col[c].bmean = tot[c] / (double)n;
    }
}

// Start the CG of every column: v = src - mean (subtract: the column means in
// meancol[c].bmean, written back to src), r = (V) v, x = 0, ||r||^2 and sum r
// per column.  With `outer` (refinement), only columns still running there
// start, each with tolerance max(refine_tol, 0.3 tol / outer relres); the
// others get a zero right-hand side and stay stopped.
template <typename V>
__global__ void __launch_bounds__(kBThreads)
kb_center(int n, int R, int CT, int nrhs, int subtract, double *__restrict__ src, V *__restrict__ r,
          V *__restrict__ x, const BCol *meancol, BCol *col, double tol, int maxit,
          const BCol *outer, double refine_tol, double *part, unsigned *ticket)
{
    __shared__ double tot[512];
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    double acc[2][8];
    for (int j = 0; j < 8; ++j) acc[0][j] = acc[1][j] = 0.0;
    for (int i = blockIdx.x * S + o; i < n; i += gridDim.x * S) {
        for (int j = 0; j < R / CT; ++j) {
            const int c = cl + j * CT;
            const size_t k = (size_t)i * R + c;
            double v = src[k];
            if (subtract) {
                v -= meancol[c].bmean;
                src[k] = v;
            }
            if (outer && outer[c].flag != kRun) v = 0.0;
            const V rv = (V)v;
            r[k] = rv;
            if (x) x[k] = V(0);
            acc[0][j] += (double)rv * (double)rv;
            acc[1][j] += (double)rv;
        }
    }
    if (bcol_reduce<2, 8>(acc, R, CT, part, ticket, tot)) {
        for (int c = threadIdx.x; c < R; c += kBThreads) {
            BCol &C = col[c];
            C.bnorm = sqrt(tot[c]);
            C.rr = tot[c];
            C.rs = tot[R + c];
            C.relres = 1.0;
            C.iter = 0;
            C.first = 1;
            C.maxit = maxit;
            C.tol = outer ? fmin(0.5, fmax(refine_tol, 0.3 * tol / outer[c].relres)) : tol;
            const bool run = c < nrhs && tot[c] > 0.0 && (!outer || outer[c].flag == kRun);
            C.flag = run ? kRun : kConverged;
        }
    }
}

// Refinement bookkeeping: a running column whose true residual meets tol stops.
static __global__ void kb_refine_flags(int R, int nrhs, BCol *col, double tol)
{
    for (int c = threadIdx.x; c < R; c += blockDim.x) {
        BCol &C = col[c];
        if (C.flag == kRun && (c >= nrhs || C.relres <= tol)) C.flag = kConverged;
        if (C.flag == kRun && !isfinite(C.relres)) C.flag = kBreakdown;
    }
}

// ---------------------------------------------------------------------------
// SpMM  y = L x (edge-difference form, CSR) for all columns.
// MODE 0: reduce p.q and sum q per column -> alpha; MODE 1: yres(double) =
// Bs - L x with ||.||^2, sum per column -> relres (true residual); MODE 2: none.
// Long rows take the sum of their chunk partials (kb_long_chunks, run first)
// in chunk order instead of walking their entries.
// ---------------------------------------------------------------------------
template <typename V>
__global__ void __launch_bounds__(kBThreads)
kb_long_chunks(int nchunks, int R, int CT, const int *__restrict__ chunk_row,
               const int64_t *__restrict__ chunk_beg, const int *__restrict__ lrow,
               const int64_t *__restrict__ lrp, const int *__restrict__ rp,
               const int *__restrict__ lci, const V *__restrict__ lw, const V *__restrict__ x,
               V *__restrict__ chunk_part)
{
    // entries outermost: each entry's index and weight are loaded once and
    // the R / CT column tiles of its neighbour's row read one after another
    // (every column still sums its entries in the same order)
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    const int nj = R / CT;
    __shared__ V red[8][kBThreads];
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int li = chunk_row[ch];
        const int row = lrow[li];
        V xi[8], sj[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            xi[j] = j < nj ? x[(size_t)row * R + cl + j * CT] : V(0);
            sj[j] = V(0);
        }
        // the chunk's real entries: the layout pads each long row to whole
        // groups of 128 entries (weight 0), which add nothing here
        const int64_t real_end = lrp[li] + (rp[row + 1] - rp[row]);
        const int64_t pe = chunk_beg[ch + 1] < real_end ? chunk_beg[ch + 1] : real_end;
        int64_t p = chunk_beg[ch] + o;
        // U entries in flight (their neighbour rows loaded before any is
        // added), then added in entry order
        constexpr int U = sizeof(V) == 4 ? 4 : 2;
        for (; p + (U - 1) * S < pe; p += U * S) {
            V wu[U], a[U][8];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                wu[u] = lw[p + u * S];
                const V *xu = x + (size_t)lci[p + u * S] * R + cl;
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (j < nj) a[u][j] = xu[j * CT];
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (j < nj) sj[j] += wu[u] * (xi[j] - a[u][j]);
        }
        for (; p < pe; p += S) {
            const V wv = lw[p];
            const V *xr = x + (size_t)lci[p] * R + cl;
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < nj) sj[j] += wv * (xi[j] - xr[j * CT]);
        }
        // reduce over the S row groups, all column tiles at once
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < nj) red[j][threadIdx.x] = sj[j];
        __syncthreads();
        for (int st = S / 2; st > 0; st >>= 1) {
            if (o < st)
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (j < nj) red[j][threadIdx.x] += red[j][threadIdx.x + st * CT];
            __syncthreads();
        }
        if (o == 0)
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < nj) chunk_part[(size_t)ch * R + cl + j * CT] = red[j][threadIdx.x];
        __syncthreads();
    }
}

template <typename V, int MODE>
__global__ void __launch_bounds__(kBThreads)
kb_spmm(int n, int R, int CT, const int *__restrict__ rp, const int *__restrict__ ci,
        const V *__restrict__ w, const unsigned char *__restrict__ is_long,
        const int *__restrict__ lrow_of, const int *__restrict__ lchunk_ptr,
        const V *__restrict__ chunk_part, const V *__restrict__ x, V *__restrict__ y,
        const double *__restrict__ Bs, double *__restrict__ yres, BCol *col, double *part,
        unsigned *ticket, double *tres)
{
    __shared__ double tot[512];
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    double acc[2][8];
    for (int j = 0; j < 8; ++j) acc[0][j] = acc[1][j] = 0.0;
    const int nj = R / CT;
    for (int i = blockIdx.x * S + o; i < n; i += gridDim.x * S) {
        const bool lng = is_long && is_long[i];
        const int b = rp[i], e = rp[i + 1];
        // the row's entries outermost (index and weight loaded once, the
        // neighbour's column tiles read in turn); per column the same order
        V xv[8], sv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            xv[j] = j < nj ? x[(size_t)i * R + cl + j * CT] : V(0);
            sv[j] = V(0);
        }
        if (lng) {
            const int li = lrow_of[i];
            for (int ch = lchunk_ptr[li]; ch < lchunk_ptr[li + 1]; ++ch)
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (j < nj) sv[j] += chunk_part[(size_t)ch * R + cl + j * CT];
        } else {
            for (int p = b; p < e; ++p) {
                const V wv = w[p];
                const V *xr = x + (size_t)ci[p] * R + cl;
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (j < nj) sv[j] += wv * (xv[j] - xr[j * CT]);
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j >= nj) break;
            const int c = cl + j * CT;
            const size_t k = (size_t)i * R + c;
            const V xi = xv[j];
            const V s = sv[j];
            if (MODE == 1 || MODE == 3) {
                const double rv = Bs[k] - (double)s;
                if (MODE == 1 || yres) yres[k] = rv;
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
    if (bcol_reduce<2, 8>(acc, R, CT, part, ticket, tot)) {
        for (int c = threadIdx.x; c < R; c += kBThreads) {
            BCol &C = col[c];
            if (MODE == 3) {                 // true residuals only, state untouched
                tres[c] = C.bnorm > 0.0 ? sqrt(tot[c]) / C.bnorm : 0.0;
            } else if (MODE == 0) {
                if (C.flag != kRun) continue;
                C.pq = tot[c];
                C.qs = tot[R + c];
                C.alpha = C.rho / tot[c];
                if (!(tot[c] > 0.0) || !isfinite(C.alpha)) C.flag = kBreakdown;
            } else if (C.bnorm > 0.0) {      // true residual of every column
                C.rr = tot[c];
                C.rs = tot[R + c];
                C.relres = sqrt(tot[c]) / C.bnorm;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// MSP sweeps on R columns.  Aggregate-level kernels map thread (o, cl) to
// aggregate J0 + o and column cl + j * CT.
// ---------------------------------------------------------------------------
// MODE 0: level k >= 2 in place (a -> delta); MODE 1: finest level with the CG
// step (x += alpha p, r -= alpha q for active columns), delta_1 -> dout,
// reduces ||r||^2, sum r -> convergence per column; MODE 2: finest, no step.
// Aggregates with more than kBatchBigAgg members (big[0..nbig), hubs of
// power-law graphs) are taken by a whole block each: the row groups split
// the members, the per-column sums meet in shared memory.
template <typename V, int MODE>
__global__ void __launch_bounds__(kBThreads)
kb_up(int nagg, int R, int CT, const int *__restrict__ seg, const V *__restrict__ inv,
      const V *__restrict__ lcf, V *__restrict__ x, V *r, const V *__restrict__ p,
      const V *__restrict__ q, V *dout, V *anext, V gamma, const V *fnext, BCol *col, double *part,
      unsigned *ticket, int nbig, const int *__restrict__ big)
{
    __shared__ double tot[512];
    __shared__ V bred[3][kBThreads];
    __shared__ V bsol[2][kBThreads];
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    double acc[2][8];
    for (int j = 0; j < 8; ++j) acc[0][j] = acc[1][j] = 0.0;
    for (int bi = blockIdx.x; bi < nbig; bi += gridDim.x) {
        const int J = big[bi];
        const int b0 = seg[J], e = seg[J + 1];
        const V *cf = inv + 4 * J;
        const V *lc = lcf + 3 * (b0 - 2 * J);
        for (int jj = 0; jj < R / CT; ++jj) {
            const int c = cl + jj * CT;
            if (MODE == 1) {
                const bool act = bactive(col, c);
                const V al = act ? (V)col[c].alpha : V(0);
                if (act)
                    for (int u = b0 + o; u < e; u += S) {
                        const size_t k = (size_t)u * R + c;
                        x[k] += al * p[k];
                        r[k] -= al * q[k];
                    }
                __syncthreads();
            }
            V sm = V(0), ha = V(0), hb = V(0);
            for (int t = b0 + 2 + o; t < e; t += S) {
                const V al = r[(size_t)t * R + c];
                const V *cc = lc + 3 * (t - b0 - 2);
                sm += al;
                ha += cc[0] * al;
                hb += cc[1] * al;
                if (MODE != 0) {
                    acc[0][jj] += (double)al * al;
                    acc[1][jj] += (double)al;
                }
            }
            if (o == 0) {
                const V aa = r[(size_t)b0 * R + c], ab = r[(size_t)(b0 + 1) * R + c];
                sm += aa + ab;
                ha += aa;
                hb += ab;
                if (MODE != 0) {
                    acc[0][jj] += (double)aa * aa + (double)ab * ab;
                    acc[1][jj] += (double)aa + (double)ab;
                }
            }
            bred[0][threadIdx.x] = sm;
            bred[1][threadIdx.x] = ha;
            bred[2][threadIdx.x] = hb;
            __syncthreads();
            for (int st = S / 2; st > 0; st >>= 1) {
                if (o < st)
                    for (int k = 0; k < 3; ++k) bred[k][threadIdx.x] += bred[k][threadIdx.x + st * CT];
                __syncthreads();
            }
            if (o == 0) {
                V da, db;
                pair_solve(cf, bred[1][cl], bred[2][cl], da, db);
                bsol[0][cl] = da;
                bsol[1][cl] = db;
                V nx = gamma * bred[0][cl];
                if (fnext) nx += fnext[(size_t)J * R + c];
                anext[(size_t)J * R + c] = nx;
            }
            __syncthreads();
            const V da = bsol[0][cl], db = bsol[1][cl];
            for (int t = b0 + 2 + o; t < e; t += S) {
                const V *cc = lc + 3 * (t - b0 - 2);
                dout[(size_t)t * R + c] = r[(size_t)t * R + c] * cc[2] + cc[0] * da + cc[1] * db;
            }
            if (o == 0) {
                dout[(size_t)b0 * R + c] = da;
                dout[(size_t)(b0 + 1) * R + c] = db;
            }
            __syncthreads();
        }
    }
    for (int J = blockIdx.x * S + o; J < nagg; J += gridDim.x * S) {
        const int b0 = seg[J], e = seg[J + 1];
        if (e - b0 > kBatchBigAgg) continue;
        const V *cf = inv + 4 * J;
        const V *lc = lcf + 3 * (b0 - 2 * J);
        for (int jj = 0; jj < R / CT; ++jj) {
            const int c = cl + jj * CT;
            if (MODE == 1) {
                const bool act = bactive(col, c);
                const V al = act ? (V)col[c].alpha : V(0);
                for (int u = b0; u < e; ++u) {
                    const size_t k = (size_t)u * R + c;
                    if (act) {
                        x[k] += al * p[k];
                        r[k] -= al * q[k];
                    }
                }
            }
            // gather the aggregate's column into registers-light form
            const V aa = r[(size_t)b0 * R + c], ab = r[(size_t)(b0 + 1) * R + c];
            V sum = aa + ab, ha = aa, hb = ab;
            if (MODE != 0) {
                acc[0][jj] += (double)aa * aa + (double)ab * ab;
                acc[1][jj] += (double)aa + (double)ab;
            }
            for (int t = b0 + 2; t < e; ++t) {
                const V al = r[(size_t)t * R + c];
                const V *cc = lc + 3 * (t - b0 - 2);
                sum += al;
                ha += cc[0] * al;
                hb += cc[1] * al;
                if (MODE != 0) {
                    acc[0][jj] += (double)al * al;
                    acc[1][jj] += (double)al;
                }
            }
            V da, db;
            pair_solve(cf, ha, hb, da, db);
            for (int t = b0 + 2; t < e; ++t) {
                const V *cc = lc + 3 * (t - b0 - 2);
                dout[(size_t)t * R + c] = r[(size_t)t * R + c] * cc[2] + cc[0] * da + cc[1] * db;
            }
            dout[(size_t)b0 * R + c] = da;
            dout[(size_t)(b0 + 1) * R + c] = db;
            V nx = gamma * sum;
            if (fnext) nx += fnext[(size_t)J * R + c];
            anext[(size_t)J * R + c] = nx;
        }
    }
    if (MODE == 0) return;
    if (bcol_reduce<2, 8>(acc, R, CT, part, ticket, tot)) {
        for (int c = threadIdx.x; c < R; c += kBThreads) {
            BCol &C = col[c];
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

// Top level: Y(i, c) = scale * sum_k G(i, k) A(k, c), FP64 accumulation.
template <typename V>
__global__ void __launch_bounds__(kBThreads)
kb_coarse(int m, int R, const double *__restrict__ G, const V *__restrict__ A, V *__restrict__ Y,
          double scale)
{
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < m * R; idx += gridDim.x * blockDim.x) {
        const int i = idx / R, c = idx % R;
        double s = 0.0;
        for (int k = 0; k < m; ++k) s += G[(size_t)i * m + k] * (double)A[(size_t)k * R + c];
        Y[idx] = (V)(scale * s);
    }
}

// out(u, c) = pc * parent(J, c) + dc * delta(u, c); FINEST also reduces
// sum z, r.z, z.q per column and finalises zmean, rho, beta.
template <typename V, bool FINEST>
__global__ void __launch_bounds__(kBThreads)
kb_down(int n, int nagg, int R, int CT, const int *__restrict__ seg, const V *__restrict__ delta,
        const V *__restrict__ parent, V *__restrict__ out, V pc, V dc, const V *__restrict__ r,
        BCol *col, double *part, unsigned *ticket, int nbig, const int *__restrict__ big)
{
    __shared__ double tot[512];
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    double acc[2][8];
    for (int j = 0; j < 8; ++j) acc[0][j] = acc[1][j] = 0.0;
    // large aggregates: a block each, the row groups splitting the members
    for (int bi = blockIdx.x; bi < nbig; bi += gridDim.x) {
        const int J = big[bi];
        for (int jj = 0; jj < R / CT; ++jj) {
            const int c = cl + jj * CT;
            const V base = pc * parent[(size_t)J * R + c];
            for (int u = seg[J] + o; u < seg[J + 1]; u += S) {
                const size_t k = (size_t)u * R + c;
                const V z = base + dc * delta[k];
                out[k] = z;
                if (FINEST) {
                    acc[0][jj] += (double)z;
                    acc[1][jj] += (double)r[k] * (double)z;
                }
            }
        }
    }
    for (int J = blockIdx.x * S + o; J < nagg; J += gridDim.x * S) {
        if (seg[J + 1] - seg[J] > kBatchBigAgg) continue;
        for (int jj = 0; jj < R / CT; ++jj) {
            const int c = cl + jj * CT;
            const V base = pc * parent[(size_t)J * R + c];
            for (int u = seg[J]; u < seg[J + 1]; ++u) {
                const size_t k = (size_t)u * R + c;
                const V z = base + dc * delta[k];
                out[k] = z;
                if (FINEST) {
                    acc[0][jj] += (double)z;
                    acc[1][jj] += (double)r[k] * (double)z;
                }
            }
        }
    }
    if (!FINEST) return;
    if (bcol_reduce<2, 8>(acc, R, CT, part, ticket, tot)) {
        for (int c = threadIdx.x; c < R; c += kBThreads) {
            BCol &C = col[c];
            if (C.flag != kRun) continue;
            const double m = tot[c] / (double)n;
            const double rho_new = tot[R + c] - m * C.rs;
            C.zmean = m;
            C.beta = C.first ? 0.0 : rho_new / C.rho;
            C.rho = rho_new;
            C.first = 0;
            if (!isfinite(rho_new)) C.flag = kBreakdown;
        }
    }
}

// Plain CG (no preconditioner): step and z = Pi r statistics in one pass.
template <typename V, bool UPDATE>
__global__ void __launch_bounds__(kBThreads)
kb_plain(int n, int R, int CT, V *__restrict__ x, V *__restrict__ r, const V *__restrict__ p,
         const V *__restrict__ q, BCol *col, double *part, unsigned *ticket)
{
    __shared__ double tot[512];
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    double acc[2][8];
    for (int j = 0; j < 8; ++j) acc[0][j] = acc[1][j] = 0.0;
    for (int i = blockIdx.x * S + o; i < n; i += gridDim.x * S) {
        for (int jj = 0; jj < R / CT; ++jj) {
            const int c = cl + jj * CT;
            const size_t k = (size_t)i * R + c;
            V rv = r[k];
            if (UPDATE && bactive(col, c)) {
                const V al = (V)col[c].alpha;
                x[k] += al * p[k];
                rv -= al * q[k];
                r[k] = rv;
            }
            acc[0][jj] += (double)rv * rv;
            acc[1][jj] += (double)rv;
        }
    }
    if (bcol_reduce<2, 8>(acc, R, CT, part, ticket, tot)) {
        for (int c = threadIdx.x; c < R; c += kBThreads) {
            BCol &C = col[c];
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
                const double m = tot[R + c] / (double)n;
                const double rho_new = tot[c] - m * tot[R + c];
                C.zmean = m;
                C.beta = C.first ? 0.0 : rho_new / C.rho;
                C.rho = rho_new;
                C.first = 0;
            }
        }
    }
}

// p = (z - zmean) + beta p for active columns (beta == 0 never reads p)
template <typename V>
__global__ void __launch_bounds__(kBThreads)
kb_pupdate(int n, int R, int CT, const V *__restrict__ z, V *__restrict__ p, const BCol *col)
{
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    for (int i = blockIdx.x * S + o; i < n; i += gridDim.x * S) {
        for (int jj = 0; jj < R / CT; ++jj) {
            const int c = cl + jj * CT;
            if (!bactive(col, c)) continue;
            const size_t k = (size_t)i * R + c;
            const V m = (V)col[c].zmean, be = (V)col[c].beta;
            p[k] = be == V(0) ? z[k] - m : (z[k] - m) + be * p[k];
        }
    }
}

// x64 += (double) d for columns `mask` selects (refinement correction)
template <typename V>
__global__ void __launch_bounds__(kBThreads)
kb_add(int64_t nR, double *__restrict__ x, const V *__restrict__ d)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nR; k += (int64_t)gridDim.x * blockDim.x)
        x[k] += (double)d[k];
}

// Per-column mean of x (tree order) and the scatter to the caller's
// column-major layout with the projection.
template <typename V>
__global__ void __launch_bounds__(kBThreads)
kb_mean(int n, int R, int CT, const V *__restrict__ x, double *__restrict__ means, double *part,
        unsigned *ticket)
{
    __shared__ double tot[256];
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    double acc[1][8];
    for (int j = 0; j < 8; ++j) acc[0][j] = 0.0;
    for (int i = blockIdx.x * S + o; i < n; i += gridDim.x * S)
        for (int jj = 0; jj < R / CT; ++jj) acc[0][jj] += (double)x[(size_t)i * R + cl + jj * CT];
    if (bcol_reduce<1, 8>(acc, R, CT, part, ticket, tot))
        for (int c = threadIdx.x; c < R; c += kBThreads) means[c] = tot[c] / (double)n;
}

template <typename V>
__global__ void __launch_bounds__(kBThreads)
kb_scatter(int n, int R, int CT, int nrhs, const int *__restrict__ perm, const V *__restrict__ x,
           const double *__restrict__ means, double *__restrict__ X)
{
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    for (int i = blockIdx.x * S + o; i < n; i += gridDim.x * S) {
        const int dst = perm[i];
        for (int jj = 0; jj < R / CT; ++jj) {
            const int c = cl + jj * CT;
            if (c < nrhs) X[(size_t)c * n + dst] = (double)x[(size_t)i * R + c] - means[c];
        }
    }
}

// ---------------------------------------------------------------------------
// Continuous batching: columns [c0, c0 + k) of a running batch start a new
// request while the other columns keep iterating.
// ---------------------------------------------------------------------------
// Bs(:, c0..c0+k) = the request's columns in tree order; their sums -> bmean.
static __global__ void __launch_bounds__(kBThreads)
kb_join_gather(int n, int R, int CT, int c0, int k, const int *__restrict__ perm,
               const double *__restrict__ B, double *__restrict__ Bs, BCol *col, double *part,
               unsigned *ticket)
{
    __shared__ double tot[256];
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    double acc[1][8];
    for (int j = 0; j < 8; ++j) acc[0][j] = 0.0;
    for (int i = blockIdx.x * S + o; i < n; i += gridDim.x * S) {
        const int src = perm[i];
        for (int j = 0; j < R / CT; ++j) {
            const int c = cl + j * CT;
            if (c < c0 || c >= c0 + k) continue;
            const double v = B[(size_t)(c - c0) * n + src];
            Bs[(size_t)i * R + c] = v;
            acc[0][j] += v;
        }
    }
    if (bcol_reduce<1, 8>(acc, R, CT, part, ticket, tot))
        for (int c = threadIdx.x; c < R; c += kBThreads)
            if (c >= c0 && c < c0 + k) col[c].bmean = tot[c] / (double)n;
}

// Centre the joining columns, r = Bs, x = 0 there (and x64 = 0 if given:
// the FP64 solution of a refined column), and start their CG.
template <typename V>
__global__ void __launch_bounds__(kBThreads)
kb_join_center(int n, int R, int CT, int c0, int k, double *__restrict__ Bs, V *__restrict__ r,
               V *__restrict__ x, BCol *col, double tol, int maxit, double *part, unsigned *ticket,
               double *__restrict__ x64)
{
    __shared__ double tot[512];
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    double acc[2][8];
    for (int j = 0; j < 8; ++j) acc[0][j] = acc[1][j] = 0.0;
    for (int i = blockIdx.x * S + o; i < n; i += gridDim.x * S) {
        for (int j = 0; j < R / CT; ++j) {
            const int c = cl + j * CT;
            if (c < c0 || c >= c0 + k) continue;
            const size_t q = (size_t)i * R + c;
            const double v = Bs[q] - col[c].bmean;
            Bs[q] = v;
            r[q] = (V)v;
            x[q] = V(0);
            if (x64) x64[q] = 0.0;
            acc[0][j] += v * v;
            acc[1][j] += v;
        }
    }
    if (bcol_reduce<2, 8>(acc, R, CT, part, ticket, tot)) {
        for (int c = threadIdx.x; c < R; c += kBThreads) {
            if (c < c0 || c >= c0 + k) continue;
            BCol &C = col[c];
            C.bnorm = sqrt(tot[c]);
            C.rr = tot[c];
            C.rs = tot[R + c];
            C.relres = 1.0;
            C.iter = 0;
            C.first = 1;
            C.tol = tol;
            C.maxit = maxit;
            C.join = 1;
            C.flag = tot[c] > 0.0 ? kRun : kConverged;
        }
    }
}

// First direction of the joining columns only: p = z - zmean.
template <typename V>
__global__ void __launch_bounds__(kBThreads)
kb_pupdate_join(int n, int R, int CT, const V *__restrict__ z, V *__restrict__ p, const BCol *col)
{
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    for (int i = blockIdx.x * S + o; i < n; i += gridDim.x * S)
        for (int jj = 0; jj < R / CT; ++jj) {
            const int c = cl + jj * CT;
            if (col[c].join && col[c].flag == kRun) p[(size_t)i * R + c] = z[(size_t)i * R + c] - (V)col[c].zmean;
        }
}

static __global__ void kb_clear_join(int R, BCol *col)
{
    for (int c = threadIdx.x; c < R; c += blockDim.x) col[c].join = 0;
}

// Stop columns [c0, c0 + k) (cancelled requests): flag := f.
static __global__ void kb_set_flags(int R, int c0, int k, BCol *col, int f)
{
    for (int c = threadIdx.x; c < R; c += blockDim.x)
        if (c >= c0 && c < c0 + k) col[c].flag = f;
}

// X(:, 0..k) = x(:, c0..c0+k) - mean, back in the caller's numbering.
template <typename V>
__global__ void __launch_bounds__(kBThreads)
kb_scatter_range(int n, int R, int CT, int c0, int k, const int *__restrict__ perm,
                 const V *__restrict__ x, const double *__restrict__ means, double *__restrict__ X)
{
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    for (int i = blockIdx.x * S + o; i < n; i += gridDim.x * S) {
        const int dst = perm[i];
        for (int jj = 0; jj < R / CT; ++jj) {
            const int c = cl + jj * CT;
            if (c >= c0 && c < c0 + k) X[(size_t)(c - c0) * n + dst] = (double)x[(size_t)i * R + c] - means[c];
        }
    }
}

// Restart of stopped columns whose true residual missed the tolerance: r =
// the true residual res (FP64, from kb_spmm) for columns c in [c0, c0 + k)
// with flag converged and tres[c] > tol.  The flags are set afterwards by
// kb_restart_flags (one block), so that every block decides alike here.
template <typename V>
__global__ void __launch_bounds__(kBThreads)
kb_restart_copy(int n, int R, int CT, int c0, int k, const double *__restrict__ res, V *__restrict__ r,
                const BCol *col, const double *__restrict__ tres, double tol)
{
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    for (int i = blockIdx.x * S + o; i < n; i += gridDim.x * S)
        for (int jj = 0; jj < R / CT; ++jj) {
            const int c = cl + jj * CT;
            if (c < c0 || c >= c0 + k || col[c].flag != kConverged || !(tres[c] > tol)) continue;
            r[(size_t)i * R + c] = (V)res[(size_t)i * R + c];
        }
}

static __global__ void kb_restart_flags(int R, int c0, int k, BCol *col, const double *__restrict__ tres,
                                        double tol)
{
    for (int c = threadIdx.x; c < R; c += blockDim.x) {
        if (c < c0 || c >= c0 + k || col[c].flag != kConverged || !(tres[c] > tol)) continue;
        col[c].flag = kRun;
        col[c].first = 1;
        col[c].join = 1;
    }
}

// Mixed-precision refinement of served columns.  x64(:, c) += x(:, c), then
// x(:, c) = 0, for the columns c in [c0, c0 + k) (their inner solves ended).
template <typename V>
__global__ void __launch_bounds__(kBThreads)
kb_add_cols(int n, int R, int CT, int c0, int k, double *__restrict__ x64, V *__restrict__ x)
{
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    for (int i = blockIdx.x * S + o; i < n; i += gridDim.x * S)
        for (int jj = 0; jj < R / CT; ++jj) {
            const int c = cl + jj * CT;
            if (c >= c0 && c < c0 + k) {
                const size_t q = (size_t)i * R + c;
                x64[q] += (double)x[q];
                x[q] = V(0);                    // added once: a column not refined again adds nothing
            }
        }
}

// Next inner solve of the columns in range whose true residual tres[c] is
// above tol: r = (V) res (the FP64 true residual), x = 0.
template <typename V>
__global__ void __launch_bounds__(kBThreads)
kb_refine_copy(int n, int R, int CT, int c0, int k, const double *__restrict__ res, V *__restrict__ r,
               V *__restrict__ x, const double *__restrict__ tres, double tol)
{
    const int S = kBThreads / CT, o = threadIdx.x / CT, cl = threadIdx.x % CT;
    for (int i = blockIdx.x * S + o; i < n; i += gridDim.x * S)
        for (int jj = 0; jj < R / CT; ++jj) {
            const int c = cl + jj * CT;
            if (c < c0 || c >= c0 + k || !(tres[c] > tol)) continue;
            const size_t q = (size_t)i * R + c;
            r[q] = (V)res[q];
            x[q] = V(0);
        }
}

// ...and their CG state: running again from a first direction, tolerance
// max(refine_tol, 0.3 tol / tres) relative to ||Pi b|| times tres (the inner
// system's right-hand side is the residual), at most 0.5; maxit per solve.
static __global__ void kb_refine_flags(int R, int c0, int k, BCol *col, const double *__restrict__ tres, double tol,
                                       double refine_tol, int maxit)
{
    for (int c = threadIdx.x; c < R; c += blockDim.x) {
        if (c < c0 || c >= c0 + k || !(tres[c] > tol)) continue;
        BCol &C = col[c];
        const double rel = fmin(0.5, fmax(refine_tol, 0.3 * tol / tres[c]));
        C.flag = kRun;
        C.first = 1;
        C.join = 1;
        C.iter = 0;
        C.maxit = maxit;
        C.tol = rel * tres[c];                 // relative to ||Pi b|| (the column's bnorm)
    }
}

}  // namespace lap
