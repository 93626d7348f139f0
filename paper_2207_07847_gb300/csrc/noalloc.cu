// Laplacian residual that allocates no device memory.
//
// For callers that cannot allocate device memory at all -- a process whose
// device-memory quota is already spent (an out-of-memory handler that still
// has to report how good the last iterate is), or code that must not touch an
// allocator it shares with other work -- this entry point needs no handle and
// no allocator: the caller passes the graph (device CSR), x and b, and
// receives r and two norms.  The only scratch it needs, the per-tile partial
// sums of its reductions, lives in a fixed file-scope __device__ array that
// every GPU using this library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "lap.h"

namespace {

constexpr int kTile = 256;                    // rows per block, one partial each
constexpr int kMaxTiles = 65536;              // => at most 16,777,216 rows
constexpr int64_t kMaxRows = int64_t(kTile) * kMaxTiles;

struct NoallocScratch {
    double part[kMaxTiles][2];                // per-tile partial sums
    double mean;                              // mean of b
    double rr, bb;                            // ||r||^2, ||Pi b||^2
    unsigned ticket;                          // blocks finished (must start at 0)
};

// 1 MiB + a few bytes, shared by every call on the device.
static __device__ __align__(256) NoallocScratch g_noalloc;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
NoallocScratch *g_addr[kMaxDevices] = {};

// Per-tile sums of b; the last block adds the partials in tile order.
__global__ void __launch_bounds__(kTile) k_na_mean(int64_t n, const double *__restrict__ b,
                                                   NoallocScratch *S)
{
    __shared__ double sm[kTile / 32];
    __shared__ bool last;
    const int64_t i = int64_t(blockIdx.x) * kTile + threadIdx.x;
    double v = i < n ? b[i] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kTile / 32; ++w) s += sm[w];
        S->part[blockIdx.x][0] = s;
        __threadfence();
        last = atomicAdd(&S->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double s = 0.0;
        for (unsigned t = 0; t < gridDim.x; ++t) s += __ldcg(&S->part[t][0]);
        S->mean = s / static_cast<double>(n);
        S->ticket = 0u;
    }
}

// r_i = (b_i - mean) - sum_j w_ij (x_i - x_j); per-tile ||r||^2, ||Pi b||^2.
__global__ void __launch_bounds__(kTile) k_na_residual(int64_t n, const int64_t *__restrict__ rp,
                                                       const int32_t *__restrict__ ci,
                                                       const double *__restrict__ w,
                                                       const double *__restrict__ x,
                                                       const double *__restrict__ b,
                                                       double *__restrict__ r, NoallocScratch *S)
{
    __shared__ double sm[2][kTile / 32];
    __shared__ bool last;
    const int64_t i = int64_t(blockIdx.x) * kTile + threadIdx.x;
    double rr = 0.0, bb = 0.0;
    if (i < n) {
        const double xi = x[i];
        double s = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s += w[p] * (xi - x[ci[p]]);
        const double bi = b[i] - S->mean;
        const double ri = bi - s;
        r[i] = ri;
        rr = ri * ri;
        bb = bi * bi;
    }
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, o);
        bb += __shfl_down_sync(0xffffffffu, bb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sm[0][threadIdx.x >> 5] = rr;
        sm[1][threadIdx.x >> 5] = bb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int q = 0; q < kTile / 32; ++q) {
            a += sm[0][q];
            c += sm[1][q];
        }
        S->part[blockIdx.x][0] = a;
        S->part[blockIdx.x][1] = c;
        __threadfence();
        last = atomicAdd(&S->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double a = 0.0, c = 0.0;
        for (unsigned t = 0; t < gridDim.x; ++t) {
            a += __ldcg(&S->part[t][0]);
            c += __ldcg(&S->part[t][1]);
        }
        S->rr = a;
        S->bb = c;
        S->ticket = 0u;
    }
}

// Device address of the scratch array on the current device (looked up once).
lap_status scratch_address(NoallocScratch **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        (void)cudaGetLastError();
        return LAP_ERR_CUDA;
    }
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return LAP_ERR_CUDA;
        }
        g_addr[dev] = static_cast<NoallocScratch *>(p);
    }
    *out = g_addr[dev];
    return LAP_OK;
}

}  // namespace

extern "C" lap_status lap_laplacian_residual_noalloc(int64_t n, const int64_t *d_row_ptr,
                                                     const int32_t *d_col_idx, const double *d_w,
                                                     const double *d_x, const double *d_b,
                                                     double *d_r, double *h_norms, void *stream)
{
    if (n < 1 || !d_row_ptr || !d_col_idx || !d_w || !d_x || !d_b || !d_r || !h_norms)
        return LAP_ERR_INVALID_ARG;
    if (n > kMaxRows) return LAP_ERR_UNSUPPORTED;      // scratch holds kMaxTiles partials
    NoallocScratch *S = nullptr;
    lap_status st = scratch_address(&S);
    if (st != LAP_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const unsigned tiles = static_cast<unsigned>((n + kTile - 1) / kTile);
    // a previous call that failed mid-way could have left the counter set
    if (cudaMemsetAsync(&S->ticket, 0, sizeof(unsigned), s) != cudaSuccess) {
        (void)cudaGetLastError();
        return LAP_ERR_CUDA;
    }
    k_na_mean<<<tiles, kTile, 0, s>>>(n, d_b, S);
    if (cudaGetLastError() != cudaSuccess) return LAP_ERR_CUDA;
    k_na_residual<<<tiles, kTile, 0, s>>>(n, d_row_ptr, d_col_idx, d_w, d_x, d_b, d_r, S);
    if (cudaGetLastError() != cudaSuccess) return LAP_ERR_CUDA;
    double tot[2] = {0.0, 0.0};
    if (cudaMemcpyAsync(tot, &S->rr, sizeof(tot), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        (void)cudaGetLastError();
        return LAP_ERR_CUDA;
    }
    h_norms[0] = std::sqrt(tot[0]);
    h_norms[1] = std::sqrt(tot[1]);
    return LAP_OK;
}
