// Device-resident model and workspaces of one solver handle.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <vector>

#include "band.cuh"
#include "kernels.cuh"
#include "lap_internal.h"

namespace lap {

// RAII device buffer from the library allocator.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { reset(); }
    void reset()
    {
        if (p) dev_free(p, nullptr);
        p = nullptr;
        bytes = 0;
    }
    bool alloc(size_t b)
    {
        reset();
        // 16-byte multiple plus 16 bytes: bulk copies of a range may round its
        // end up to the next 16-byte boundary and read that far
        b = (b + 15) / 16 * 16 + 16;
        p = dev_alloc(b, nullptr);
        bytes = p ? b : 0;
        return p != nullptr;
    }
    template <typename T> T *as() const { return static_cast<T *>(p); }
};

// A Laplacian's off-diagonal part on the device, as CSR and as SELL-32 (see
// HostSell); `kernel` selects the matvec: 0 = SELL, t > 0 = CSR with t threads
// per row, kMergeKernel = merge-path CSR (chosen by timing at setup).
template <typename V> struct DevCsr {
    int n = 0;
    int64_t nnz = 0;
    int *rp = nullptr, *ci = nullptr;
    V *w = nullptr, *dg = nullptr;
    int nslices = 0, nlong = 0;
    int64_t *sptr = nullptr;
    unsigned *lmask = nullptr;
    int *rowperm = nullptr;            // row of each SELL slot (-1: none)
    int *eci = nullptr;
    V *ew = nullptr;
    int *lrow = nullptr, *lci = nullptr;
    int64_t *lrp = nullptr;
    V *lw = nullptr;
    int nchunks = 0;
    int *lchunk_ptr = nullptr, *chunk_row = nullptr;
    int64_t *chunk_beg = nullptr;
    V *chunk_part = nullptr;           // per-chunk partial sums (scratch)
    unsigned char *is_long = nullptr;  // per row: 1 if a long row (batched SpMM)
    int *lrow_of = nullptr;            // per row: its index among the long rows
    int64_t ell_entries = 0, long_entries = 0;
    int kernel = 0;
    int vec = 1;                       // SELL lane-group width (1, 2, 4)
    int sell_grid = 0;                 // SELL blocks per launch (0: one per 8 slices, capped)
    int stream_hint = 0;               // 1: SELL and chunk entries loaded evict-first
    // merge-path matvec (merge.cuh): per block, the partials of the rows that
    // run across blocks
    int merge_nb = 0;
    int *mg_hrow = nullptr, *mg_trow = nullptr;
    V *mg_hval = nullptr, *mg_tval = nullptr;
    unsigned char *mg_hend = nullptr;
};

template <typename V> struct DevMspLevel {
    int n = 0, nagg = 0;
    int64_t off = 0;            // expanded offset of this level (tree order)
    int *seg = nullptr;         // shared between precisions
    V *inv = nullptr, *lcf = nullptr;
    int nbig = 0;               // aggregates of more than kBatchBigAgg members ...
    int *big = nullptr;         // ... their indices (batched kernels: a block each)
};

template <typename V> struct DevMsp {
    int levels = 0;
    std::vector<DevMspLevel<V>> lev;   // levels 1..l-1 (index k-1)
    std::vector<int64_t> off;          // expanded offsets, size l+1
    std::vector<V> gamma;              // c_{k+1} / c_k per level k < l
    std::vector<double> c;             // c_k = sum_{i<k} (-mu)^i per level (index k-1)
    double *G = nullptr;               // dense top-level pseudo-inverse (FP64)
    int ntop = 0;
    V mu = V(0);
    // fused coarse tail: levels tail0 .. l-1 (0-based) run in one block
    int tail0 = -1;                    // -1: no tail kernel
    size_t tail_smem = 0;
    TailParams<V> tail_n{};            // n-space MSP (pc = 1, dcoef = c_k)
    TailParams<V> tail_t{};            // expanded-space solve (pc = dcoef = 1, f added)
    // band sweeps of the levels below the tail, bottom band first; the three
    // sets share their tiles and differ in coefficients
    std::vector<BandParams<V>> band_n; // n-space MSP: gamma_k, dcoef c_k, pc 1
    std::vector<BandParams<V>> band_t; // expanded-space solve: gamma 1, dcoef 1, pc 1
    std::vector<BandParams<V>> band_p; // P(mu) by Horner: dcoef 1, pc -mu
    // the expanded-space CG step and its reductions fused into band_t and
    // tail_t (needs bands, a tail and room for the partials): up pairs of
    // all bands, then the tail's down pair at xfuse_slot
    bool xfuse = false;
    int xfuse_fin_n = 0, xfuse_slot = 0;
};

// Reduction scratch + device scalars of one CG.
struct CgState {
    CgScalars *sc = nullptr;
    double *part = nullptr;
    unsigned *ticket = nullptr;
};

// Vectors of one CG on L (n-space), preconditioned by the sweeps.
template <typename V> struct CgVectors {
    V *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr;
    V *A = nullptr, *Y = nullptr, *T = nullptr;   // expanded-space sweep buffers (ntilde)
};

}  // namespace lap
