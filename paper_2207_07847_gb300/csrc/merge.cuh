// Merge-path CSR matvec y = L x in edge-difference form (Merrill & Garland's
// merge-based SpMV decomposition, SC'16): the n row ends and the nnz entries
// form one merged sequence (row r's entries, then its end); every thread takes
// kMergeIpt consecutive items of it, so every thread does the same work
// whatever the row lengths, and a hub row is split over as many threads and
// blocks as its length needs.  A block stages its entries and row ends in
// shared memory (coalesced loads) and each thread finds its start on the
// merge path by binary search there.
//
// Deterministic: a row split across threads is the partial sum of the thread
// where it starts, then the partials of the following threads in order --
// inside a block by the starting thread, across blocks by k_merge_fix -- so
// every row is summed the same way on every run.  The reductions of MODE 0/1
// (p.q and sum q; ||r||^2 and sum r) run as a pass over the finished vector
// (k_merge_reduce), in row order.
#pragma once

#include "kernels.cuh"

namespace lap {

constexpr int kMergeIpt = 8;                        // merged items per thread
constexpr int kMergeTile = kBlock * kMergeIpt;      // items per block
constexpr int kMergeKernel = -2;                    // DevCsr::kernel value of this matvec

// The rows ended before diagonal d of the merged sequence: the smallest r in
// [lo, hi) with end(r) + r + 1 > d (end(r) = one past row r's last entry),
// else hi.
template <typename End>
__device__ __forceinline__ int merge_search(int64_t d, int lo, int hi, End end)
{
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (static_cast<int64_t>(end(mid)) + mid + 1 > d) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

template <typename V, int MODE>
__device__ __forceinline__ void merge_finish(int r, V s, V *y, const double *bs, double *yres)
{
    if (MODE == 1) yres[r] = bs[r] - static_cast<double>(s);
    else y[r] = s;
}

// Per block b: bh (the block's first row when it started in an earlier
// block: its row, the partial over this block, whether it ends here) and bt
// (a row started in this block that goes on past its end: its row and the
// partial so far); rows are -1 where there is none.
template <typename V, int MODE>
__global__ void __launch_bounds__(kBlock)
k_merge(int n, int64_t nnz, const int *__restrict__ rp, const int *__restrict__ ci, const V *__restrict__ w,
        const V *__restrict__ x, V *__restrict__ y, const double *__restrict__ bs, double *__restrict__ yres,
        int *__restrict__ bh_row, V *__restrict__ bh_val, unsigned char *__restrict__ bh_end,
        int *__restrict__ bt_row, V *__restrict__ bt_val, const CgScalars *sc)
{
    if (MODE != 2 && halted(sc)) return;
    __shared__ int s_ci[kMergeTile];
    __shared__ V s_w[kMergeTile];
    __shared__ int s_end[kMergeTile + 1];           // ends of rows I0 .. I1
    __shared__ int s_hrow[kBlock], s_trow[kBlock];
    __shared__ V s_hval[kBlock], s_tval[kBlock];
    __shared__ unsigned char s_has[kBlock], s_hend[kBlock];   // has: 1 head, 2 tail
    __shared__ int s_I0, s_I1, s_start0;
    __shared__ int64_t s_J0;
    const int t = threadIdx.x;
    const int64_t total = static_cast<int64_t>(n) + nnz;
    const int64_t D0 = static_cast<int64_t>(blockIdx.x) * kMergeTile;
    const int64_t D1 = D0 + kMergeTile < total ? D0 + kMergeTile : total;
    if (t == 0) {
        auto gend = [&](int r) { return rp[r + 1]; };
        const int i0 = merge_search(D0, static_cast<int>(D0 - nnz > 0 ? D0 - nnz : 0),
                                    static_cast<int>(D0 < n ? D0 : n), gend);
        const int i1 = merge_search(D1, static_cast<int>(D1 - nnz > 0 ? D1 - nnz : 0),
                                    static_cast<int>(D1 < n ? D1 : n), gend);
        s_I0 = i0;
        s_I1 = i1;
        s_J0 = D0 - i0;
        s_start0 = i0 < n ? rp[i0] : static_cast<int>(nnz);
        bt_row[blockIdx.x] = -1;
    }
    __syncthreads();
    const int I0 = s_I0, I1 = s_I1;
    const int64_t J0 = s_J0, J1 = D1 - I1;
    for (int64_t k = t; k < J1 - J0; k += kBlock) {
        s_ci[k] = ci[J0 + k];
        s_w[k] = w[J0 + k];
    }
    const int nend = (I1 < n ? I1 : n - 1) - I0 + 1;
    for (int k = t; k < nend; k += kBlock) s_end[k] = rp[I0 + k + 1];
    __syncthreads();
    auto end_of = [&](int r) { return s_end[r - I0]; };
    auto start_of = [&](int r) { return r == I0 ? s_start0 : s_end[r - 1 - I0]; };

    unsigned char has = 0, hend = 0;
    int hrow = -1, trow = -1;
    V hval = V(0), tval = V(0);
    const int64_t d0 = D0 + static_cast<int64_t>(t) * kMergeIpt;
    const int64_t d1 = d0 + kMergeIpt < D1 ? d0 + kMergeIpt : D1;
    if (d0 < d1) {
        int i = merge_search(d0, I0, I1, end_of);
        int64_t j = d0 - i;
        bool head_open = !(i < n && j == start_of(i));   // the row began in an earlier thread
        V acc = V(0);
        V xi = i < n ? x[i] : V(0);
        int64_t rend = i < n ? end_of(i) : INT64_MAX;
        for (int64_t d = d0; d < d1; ++d) {
            if (j < rend) {
                const int k = static_cast<int>(j - J0);
                acc += s_w[k] * (xi - x[s_ci[k]]);
                ++j;
            } else {
                if (head_open) {
                    has |= 1;
                    hrow = i;
                    hval = acc;
                    hend = 1;
                    head_open = false;
                } else {
                    merge_finish<V, MODE>(i, acc, y, bs, yres);
                }
                ++i;
                acc = V(0);
                if (i < n) {
                    xi = x[i];
                    rend = end_of(i);
                }
            }
        }
        if (head_open) {                 // the share lies inside one row
            has |= 1;
            hrow = i;
            hval = acc;
            hend = 0;
        } else if (i < n && j > start_of(i)) {   // a row started here goes on
            has |= 2;
            trow = i;
            tval = acc;
        }
    }
    s_has[t] = has;
    s_hend[t] = hend;
    s_hrow[t] = hrow;
    s_hval[t] = hval;
    s_trow[t] = trow;
    s_tval[t] = tval;
    __syncthreads();
    if (has & 2) {
        V s = tval;
        bool done = false;
        for (int u = t + 1; u < kBlock; ++u) {
            if (!(s_has[u] & 1) || s_hrow[u] != trow) break;
            s += s_hval[u];
            if (s_hend[u]) {
                merge_finish<V, MODE>(trow, s, y, bs, yres);
                done = true;
                break;
            }
        }
        if (!done) {
            bt_row[blockIdx.x] = trow;
            bt_val[blockIdx.x] = s;
        }
    }
    if (t == 0) {
        if (s_has[0] & 1) {
            const int r = s_hrow[0];
            V s = s_hval[0];
            bool e = s_hend[0] != 0;
            for (int u = 1; !e && u < kBlock && (s_has[u] & 1) && s_hrow[u] == r; ++u) {
                s += s_hval[u];
                e = s_hend[u] != 0;
            }
            bh_row[blockIdx.x] = r;
            bh_val[blockIdx.x] = s;
            bh_end[blockIdx.x] = e ? 1 : 0;
        } else {
            bh_row[blockIdx.x] = -1;
        }
    }
}

// Rows that run across blocks: the starting block's partial, then the
// following blocks' partials in order, until the row ends.
template <typename V, int MODE>
__global__ void __launch_bounds__(kBlock)
k_merge_fix(int nblocks, V *__restrict__ y, const double *__restrict__ bs, double *__restrict__ yres,
            const int *__restrict__ bh_row, const V *__restrict__ bh_val, const unsigned char *__restrict__ bh_end,
            const int *__restrict__ bt_row, const V *__restrict__ bt_val, const CgScalars *sc)
{
    if (MODE != 2 && halted(sc)) return;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    const int r = bt_row[b];
    if (r < 0) return;
    V s = bt_val[b];
    for (int c = b + 1; c < nblocks && bh_row[c] == r; ++c) {
        s += bh_val[c];
        if (bh_end[c]) {
            merge_finish<V, MODE>(r, s, y, bs, yres);
            return;
        }
    }
}

// The reductions of MODE 0 (p.q, sum q -> alpha) and MODE 1 (||r||^2, sum r
// -> relres) over the finished vector, in row order.
template <typename V, int MODE>
__global__ void __launch_bounds__(kBlock)
k_merge_reduce(int n, const V *__restrict__ x, const V *__restrict__ y, const double *__restrict__ yres,
               CgScalars *sc, double *part, unsigned *ticket)
{
    if (halted(sc)) return;
    double a0 = 0.0, a1 = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (MODE == 1) {
            const double ri = yres[i];
            a0 += ri * ri;
            a1 += ri;
        } else {
            const double q = static_cast<double>(y[i]);
            a0 += static_cast<double>(x[i]) * q;
            a1 += q;
        }
    }
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

}  // namespace lap
