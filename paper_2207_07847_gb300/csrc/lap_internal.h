// Internal declarations of the GB300 graph-Laplacian solver library.
// Host setup (setup.cpp) builds a HostModel; the CUDA side (solve.cu) uploads
// it into a DeviceModel and runs the preconditioned CG kernels (kernels.cuh).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "lap.h"

namespace lap {

// ---------------------------------------------------------------------------
// Host-side model produced by the setup stage.
//
// Every level is stored in "tree order": the members of each aggregate are
// contiguous (matched pair first, then leftovers by increasing id) and the
// aggregates of level k appear in the tree order of level k+1.  Consequently
// the subtree of any vertex is contiguous on every finer level, restriction is
// a segmented sum over contiguous segments and prolongation a segmented
// broadcast.  The top level keeps its own numbering.
// ---------------------------------------------------------------------------
struct HostLevel {
    int64_t n = 0;
    // adjacency in the hierarchy's own numbering (level 1: the input order)
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    std::vector<double> w;
    std::vector<double> deg;      // weighted degree d_k
    // aggregation to level k+1 (empty on the top level)
    std::vector<int32_t> agg;     // agg_k(u), hierarchy numbering
    std::vector<int32_t> pa, pb;  // matched pair that created each aggregate
    std::vector<double> out;      // out_k(u): weight from u to other aggregates
    // tree order
    std::vector<int32_t> perm;    // storage position -> hierarchy id
    std::vector<int32_t> pos;     // hierarchy id -> storage position
};

struct HostCsr {                  // square CSR, off-diagonal entries + diagonal
    int64_t n = 0;
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    std::vector<double> w;        // positive edge weights (matrix entry is -w)
    std::vector<double> diag;     // row sums of w
};

// Sliced ELL (SELL-32) copy of a Laplacian's off-diagonal part: rows are cut
// into slices of 32 consecutive rows; slice s stores width_s = its longest row
// as width_s x 32 entries, column-major (entry j of row 32 s + lane at
// sptr[s] + 32 j + lane), padded with (own row, weight 0).  Rows longer than
// `long_threshold` are kept out of the slices (their lanes are padding) and
// listed as CSR rows processed by a whole warp each.
struct HostSell {
    int64_t n = 0, nslices = 0;
    int vec = 1;                      // entries per lane group (1, 2 or 4): see make_sell
    std::vector<int64_t> sptr;        // [nslices + 1]
    std::vector<uint32_t> longmask;   // [nslices] lanes whose row is a long row
    std::vector<int32_t> rowperm;     // [nslices * 32] row held by each slot (-1: none); empty: slot = row
    std::vector<int32_t> eci;
    std::vector<double> ew;
    std::vector<int32_t> lrow;        // long rows
    std::vector<int64_t> lrp;         // [nlong + 1]
    std::vector<int32_t> lci;
    std::vector<double> lw;
    // long rows are cut into chunks of at most kChunk entries, summed by
    // separate warps into per-chunk partials; chunk range of long row r:
    // [lchunk_ptr[r], lchunk_ptr[r+1])
    std::vector<int32_t> lchunk_ptr;  // [nlong + 1]
    std::vector<int32_t> chunk_row;   // long-row index of each chunk
    std::vector<int64_t> chunk_beg;   // [nchunks + 1] entry ranges (into lci/lw)
};

// SELL-32 of A: slices of 32 rows, each padded to its longest row (rounded up
// to a multiple of vec) and stored lane-interleaved in groups of vec entries
// (the rows sorted by decreasing length within windows of 8 slices when that
// saves at least 5% of the padded size: slot 32 s + l then holds row
// rowperm[32 s + l]):
// entry j of lane l of slice s at sptr[s] + (j / vec) * 32 * vec + l * vec +
// j % vec, so that a lane loads vec consecutive entries with one vector load.
// Rows longer than long_threshold go to the long-row chunks (threshold 0:
// chosen from the row lengths, see choose_long_threshold).  vec = 0 picks
// the largest of 4, 2, 1 whose padding adds at most 6% to the vec = 1 size.
void make_sell(const HostCsr &A, HostSell &S, int64_t long_threshold, int vec = 0);

struct HostMspLevel {             // elimination data of level k < l (tree order)
    int64_t n = 0, nagg = 0;
    std::vector<int32_t> seg;     // [nagg+1] member ranges in level-k storage
    std::vector<double> inv;      // [4*nagg] pair solve: beta/det, alpha/det, 1/(alpha+beta),
                                  // alpha/(alpha+beta) of the 2x2 Schur complement
    std::vector<double> lcf;      // [3*(n-2*nagg)] leftover (g_a, g_b, 1/d)
};

struct HostModel {
    lap_options opt{};
    double mu = 0.8;
    int levels = 0;
    std::vector<HostLevel> lev;
    std::vector<int64_t> offset;  // expanded offsets, offset[k] = n_1 + .. + n_k
    HostCsr L1;                   // level-1 Laplacian in tree order
    std::vector<HostMspLevel> msp;
    std::vector<double> coarse_pinv;   // dense (mu^(2(l-1)) L_l)^+ , n_l x n_l row-major
    std::vector<double> c;        // c_k = sum_{i<k} (-mu)^i, k = 1..l (index k-1)
    HostCsr LH;                   // L_H over the expanded vertices in tree order (PEGP)
    bool has_LH = false;
    int64_t edges_T = 0;
};

lap_status validate_csr(int64_t n, const int64_t *rp, const int32_t *ci, const double *w,
                        std::string *why);
// The host model of one graph: hierarchy, tree order, sparsifier data and
// (PEGP) L_H.  With opt.setup_device (and a GPU) the hierarchy and L_H come
// from device kernels on `stream` (setup_device.cu), bit-exact with the host's.
lap_status build_model(int64_t n, const int64_t *rp, const int32_t *ci, const double *w,
                       const lap_options &opt, HostModel &m, void *stream = nullptr);
// The parts of build_model (m.opt and m.mu set first).
void build_hierarchy_host(int64_t n, const int64_t *rp, const int32_t *ci, const double *w, HostModel &m);
lap_status finish_model(HostModel &m);
lap_status device_build_model(int64_t n, const int64_t *rp, const int32_t *ci, const double *w, HostModel &m,
                              void *stream);
// edges of H (which = 0) or T (which = 1) in the hierarchy's expanded numbering, i < j
void expanded_edges(const HostModel &m, int which, std::vector<int64_t> &I,
                    std::vector<int64_t> &J, std::vector<double> &W);

// Band sweeps (levels [k0, k1) of the sparsifier solve per launch): band
// tops from level 0 up to kmax, and the tiles of one band (runs of level-k1
// vertices whose descendants on levels k0..k1 need at most `cap` bytes of
// shared memory with values of sv bytes): tab holds ntiles + 1 rows of
// k1 - k0 + 1 first indices, fits one flag per tile (0: the tile needs more
// than cap_fit bytes and runs in global memory).
constexpr int kBandMaxLevels = 16;
std::vector<int> plan_band_tops(const HostModel &m, int kmax, int cap, int sv);
void plan_band_tiles(const HostModel &m, int k0, int k1, int cap, int cap_fit, int sv, std::vector<int> &tab,
                     std::vector<char> &fits, int &ntiles);

// splitmix64 output i (>= 1) for `seed` (Steele, Lea & Flood 2014)
uint64_t splitmix64(uint64_t seed, uint64_t i);

// ---------------------------------------------------------------------------
// Device allocation through an optional caller allocator.
// ---------------------------------------------------------------------------
void *dev_alloc(size_t bytes, void *stream);
void dev_free(void *p, void *stream);

// Tridiagonal (a, b) of CG's Lanczos process from its first k step lengths
// alpha and coefficients beta: a_j = 1/alpha_j + beta_(j-1)/alpha_(j-1),
// b_j = sqrt(beta_j)/alpha_j.  False if a coefficient is not admissible
// (alpha <= 0, beta < 0, or not finite).
bool lanczos_tridiagonal(const double *alpha, const double *beta, int k, std::vector<double> &a,
                         std::vector<double> &b);
// Smallest and largest eigenvalue of the symmetric tridiagonal matrix with
// diagonal a and off-diagonal b, by Sturm-count bisection.
bool tridiag_extremes(const std::vector<double> &a, const std::vector<double> &b, double *lo, double *hi);

}  // namespace lap
