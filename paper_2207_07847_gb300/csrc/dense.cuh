// Dense kernels of the exact PEGP preconditioner M = L_H^+ (Section 3.2) for
// small graphs.
//
// At setup the expanded Laplacian is Jacobi-scaled and its null space lifted,
//
//     A = S L_H S + v v^T / (v^T v),   S = diag(L_H)^(-1/2),  v = diag(L_H)^(1/2),
//
// (v = S^-1 1 spans the null space of S L_H S, and A maps it to itself), A is
// inverted in place by blocked Gauss-Jordan elimination, and G = S A^-1 S.
// For a right-hand side f with zero sum, S f is orthogonal to v, so
// L_H (G f) = f: G applies L_H^+ up to an additive constant, which the
// prolongation's mean projection removes.  The scaling keeps the inverse
// accurate although the level weights mu^(2(k-1)) span many decades: the
// scaled matrix is about as well conditioned as the normalised Laplacian of
// the expanded graph.  Every preconditioner application is then one dense
// matvec y~ = G r~ between the restriction and the prolongation.
//
// Matrices are row-major with a leading dimension np = ntilde rounded up to
// kGjB; the padding rows and columns hold the identity during the inversion.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kernels.cuh"

namespace lap {

constexpr int kGjB = 64;            // pivot block = tile edge
constexpr int kGjK = 32;            // k-chunk of a tile product staged per pass
constexpr int kGjThreads = 256;     // 16 x 16 threads, 4 x 4 outputs each
constexpr int kDenseMaxN = 16384;   // largest expanded size inverted densely

// A[i][j] = v_i v_j / (v^T v) inside, the identity on the padding.
__global__ void __launch_bounds__(kBlock)
k_dense_fill(int np, int nt, const double *__restrict__ v, double vv_inv, double *__restrict__ A)
{
    const int64_t total = static_cast<int64_t>(np) * np;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = static_cast<int>(e / np), j = static_cast<int>(e % np);
        A[e] = (i < nt && j < nt) ? v[i] * v[j] * vv_inv : (i == j ? 1.0 : 0.0);
    }
}

// Adds S L_H S row by row: -w_ij s_i s_j off the diagonal, 1 on it.
__global__ void __launch_bounds__(kBlock)
k_dense_scatter(int nt, int np, const int64_t *__restrict__ rp, const int *__restrict__ ci,
                const double *__restrict__ w, const double *__restrict__ s, double *__restrict__ A)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += gridDim.x * blockDim.x) {
        double *row = A + static_cast<int64_t>(i) * np;
        const double si = s[i];
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) row[ci[p]] -= w[p] * si * s[ci[p]];
        row[i] += 1.0;
    }
}

// Pivot block: B = A_KK^-1 by unblocked Gauss-Jordan in shared memory.  A_KK
// is a principal block of a symmetric positive definite matrix's Schur
// complement, so no pivoting is needed; *bad is set if a pivot is not positive
// and finite (the host then reports a breakdown).
__global__ void __launch_bounds__(kGjThreads)
k_gj_pivot(int np, int k0, const double *__restrict__ A, double *__restrict__ B, int *bad)
{
    __shared__ double M[kGjB][kGjB + 1];
    __shared__ double rowp[kGjB], colp[kGjB];
    for (int e = threadIdx.x; e < kGjB * kGjB; e += blockDim.x) {
        const int i = e / kGjB, j = e % kGjB;
        M[i][j] = A[static_cast<int64_t>(k0 + i) * np + k0 + j];
    }
    __syncthreads();
    for (int p = 0; p < kGjB; ++p) {
        if (threadIdx.x < kGjB) {
            rowp[threadIdx.x] = M[p][threadIdx.x];
            colp[threadIdx.x] = M[threadIdx.x][p];
        }
        __syncthreads();
        const double d = rowp[p];
        if (threadIdx.x == 0 && !(d > 0.0 && isfinite(d))) *bad = 1;
        const double piv = 1.0 / d;
        for (int e = threadIdx.x; e < kGjB * kGjB; e += blockDim.x) {
            const int i = e / kGjB, j = e % kGjB;
            double val;
            if (i == p) val = j == p ? piv : rowp[j] * piv;
            else if (j == p) val = -colp[i] * piv;
            else val = M[i][j] - colp[i] * piv * rowp[j];
            M[i][j] = val;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < kGjB * kGjB; e += blockDim.x) B[e] = M[e / kGjB][e % kGjB];
}

// acc += X Y for one 64 x 64 tile: X is 64 x 64 (row-major, ldx), Y 64 x 64
// (row-major, ldy).  Thread (ty, tx) of the 16 x 16 grid owns rows ty + 16 a
// and columns tx + 16 b, so the tile's stores are coalesced along rows.
__device__ __forceinline__ void gj_tile_product(const double *__restrict__ X, int64_t ldx,
                                                const double *__restrict__ Y, int64_t ldy,
                                                double (&acc)[4][4])
{
    __shared__ double Xs[kGjB][kGjK + 1];
    __shared__ double Ys[kGjK][kGjB];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (int kc = 0; kc < kGjB; kc += kGjK) {
        __syncthreads();
        for (int e = threadIdx.x; e < kGjB * kGjK; e += kGjThreads) {
            const int i = e / kGjK, k = e % kGjK;
            Xs[i][k] = X[i * ldx + kc + k];
            const int k2 = e / kGjB, j = e % kGjB;
            Ys[k2][j] = Y[(kc + k2) * ldy + j];
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kGjK; ++k) {
            double xa[4], yb[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) xa[a] = Xs[ty + 16 * a][k];
#pragma unroll
            for (int b = 0; b < 4; ++b) yb[b] = Ys[k][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(xa[a], yb[b], acc[a][b]);
        }
    }
}

// Panels of pivot step K = [k0, k0 + 64): block t copies the column panel
// C = A[rows of tile t][K] and, for t != K, forms the row panel
// R[:, tile t] = B A[K][tile t].  A is only read here.
__global__ void __launch_bounds__(kGjThreads)
k_gj_panels(int np, int k0, const double *__restrict__ A, const double *__restrict__ B,
            double *__restrict__ C, double *__restrict__ R)
{
    const int t = blockIdx.x;
    const int64_t r0 = static_cast<int64_t>(t) * kGjB;
    for (int e = threadIdx.x; e < kGjB * kGjB; e += blockDim.x) {
        const int i = e / kGjB, c = e % kGjB;
        C[(r0 + i) * kGjB + c] = A[(r0 + i) * np + k0 + c];
    }
    if (t * kGjB == k0) return;
    double acc[4][4] = {};
    gj_tile_product(B, kGjB, A + static_cast<int64_t>(k0) * np + r0, np, acc);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) R[static_cast<int64_t>(ty + 16 * a) * np + r0 + tx + 16 * b] = acc[a][b];
}

// Rank-64 update of pivot step K, tile (I, J) = (blockIdx.y, blockIdx.x):
//   I = K:         A_KJ = R_J (J != K),  A_KK = B
//   I != K, J = K: A_IK = -C_I B
//   otherwise:     A_IJ -= C_I R_J
// (Gauss-Jordan in place: after the last pivot step A holds A^-1.)
__global__ void __launch_bounds__(kGjThreads)
k_gj_update(int np, int k0, double *__restrict__ A, const double *__restrict__ B,
            const double *__restrict__ C, const double *__restrict__ R)
{
    const int64_t i0 = static_cast<int64_t>(blockIdx.y) * kGjB, j0 = static_cast<int64_t>(blockIdx.x) * kGjB;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const bool colK = j0 == k0;
    if (i0 == k0) {
        for (int e = threadIdx.x; e < kGjB * kGjB; e += blockDim.x) {
            const int i = e / kGjB, j = e % kGjB;
            A[(i0 + i) * np + j0 + j] = colK ? B[e] : R[static_cast<int64_t>(i) * np + j0 + j];
        }
        return;
    }
    double acc[4][4] = {};
    if (colK) gj_tile_product(C + i0 * kGjB, kGjB, B, kGjB, acc);
    else gj_tile_product(C + i0 * kGjB, kGjB, R + j0, np, acc);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            double *pa = A + (i0 + ty + 16 * a) * np + j0 + tx + 16 * b;
            *pa = colK ? -acc[a][b] : *pa - acc[a][b];
        }
}

// G = S A^-1 S inside (in place), and its FP32 copy if G32 is given.
__global__ void __launch_bounds__(kBlock)
k_dense_finish(int np, int nt, const double *__restrict__ s, double *__restrict__ G, float *__restrict__ G32)
{
    const int64_t total = static_cast<int64_t>(np) * np;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = static_cast<int>(e / np), j = static_cast<int>(e % np);
        const double g = (i < nt && j < nt) ? G[e] * s[i] * s[j] : 0.0;
        G[e] = g;
        if (G32) G32[e] = static_cast<float>(g);
    }
}

// y = G x over the first nt rows and columns of a row-major matrix with
// leading dimension ld (a multiple of 64, so every row starts 16-byte
// aligned): one warp per row, 16-byte loads of G and x, warp-shuffle sum.
// V = double accumulates in FP64, V = float in FP32.
template <typename V>
__global__ void __launch_bounds__(kBlock)
k_dense_gemv(int nt, int64_t ld, const V *__restrict__ G, const V *__restrict__ x, V *__restrict__ y,
             const CgScalars *sc)
{
    if (halted(sc)) return;
    using V4 = typename std::conditional<std::is_same<V, double>::value, double2, float4>::type;
    constexpr int W = sizeof(V4) / sizeof(V);
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int nv = nt / W;                       // whole vectors per row
    const V4 *xv = reinterpret_cast<const V4 *>(x);
    for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < nt; row += nw) {
        const V4 *gv = reinterpret_cast<const V4 *>(G + row * ld);
        V s = V(0);
#pragma unroll 4
        for (int j = lane; j < nv; j += 32) {
            const V4 g = gv[j], xx = xv[j];
            if constexpr (W == 2) {
                s = fma(g.x, xx.x, s);
                s = fma(g.y, xx.y, s);
            } else {
                s = fmaf(g.x, xx.x, s);
                s = fmaf(g.y, xx.y, s);
                s = fmaf(g.z, xx.z, s);
                s = fmaf(g.w, xx.w, s);
            }
        }
        for (int j = nv * W + lane; j < nt; j += 32) s += G[row * ld + j] * x[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) y[row] = s;
    }
}

}  // namespace lap
