// Kernels of flexible GMRES(m) with right preconditioning (Saad, SIAM J. Sci.
// Comput. 14, 1993), the outer Krylov method of the paper's experiments
// (Section 4), on L x = Pi b in the n-space form (tree order, FP64).
//
// A cycle keeps the orthonormal basis V (m + 1 columns) and the
// preconditioned vectors Z = [B v_1 .. B v_m] (the preconditioner may vary
// from step to step, as the PEGP inner solve does), column after column
// (column j at offset j * n).  Step j: z_j = B v_j, w = L z_j, two passes of
// classical Gram-Schmidt against v_1..v_j (each: the j + 1 dot products in
// one launch, then w -= V h), h_(j+1,j) = ||w||, v_(j+1) = w / h_(j+1,j), and
// one thread applies the Givens rotations to the new Hessenberg column; the
// rotated right-hand side's entry j + 1 is the residual norm.  The cycle
// ends with y = R^-1 g and x += Z y.  Every reduction is a fixed-order sum of
// per-block partials, so results are deterministic.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kernels.cuh"

namespace lap {

constexpr int kGmMax = 128;        // longest cycle (restart length)
constexpr int kGmDotBlocks = 256;  // blocks per column of a multi-column dot

// Device state of one FGMRES cycle.
struct GmState {
    double H[(kGmMax + 1) * kGmMax];   // Hessenberg, column j at j * (kGmMax + 1), rotated
    double cs[kGmMax], sn[kGmMax];     // Givens rotations
    double g[kGmMax + 1];              // rotated right-hand side (beta e_1)
    double y[kGmMax];                  // least-squares solution of the cycle
    double h1[kGmMax + 1], h2[kGmMax + 1];   // Gram-Schmidt coefficients, passes 1 and 2
    double wnorm;                      // ||w|| after the second pass
    int j_done;                        // steps completed in the cycle
};

// Cycle start: v_1 = r / ||r|| (||r||^2 in sc->rr), g = ||r|| e_1.
__global__ void __launch_bounds__(kBlock)
k_gm_start(int n, const double *__restrict__ r, double *__restrict__ V, CgScalars *sc, GmState *gm)
{
    const double beta = sqrt(sc->rr);
    const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) V[i] = r[i] * inv;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        gm->g[0] = beta;
        gm->j_done = 0;
    }
}

// Z_j = z - mean (the preconditioned vector, projected; mean in *zmean) or a
// plain copy (zmean == nullptr).
__global__ void __launch_bounds__(kBlock)
k_gm_store_z(int n, const double *__restrict__ z, const double *zmean, double *__restrict__ Zj,
             const CgScalars *sc)
{
    if (halted(sc)) return;
    const double m = zmean ? *zmean : 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) Zj[i] = z[i] - m;
}

// Partial dot products of w with the columns 0..gridDim.y-1 of V: block
// (b, c) writes its sum to part[c * gridDim.x + b].
__global__ void __launch_bounds__(kBlock)
k_gm_dots(int n, const double *__restrict__ V, const double *__restrict__ w, double *__restrict__ part,
          const CgScalars *sc)
{
    if (halted(sc)) return;
    const int c = blockIdx.y;
    const double *v = V + static_cast<int64_t>(c) * n;
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s += v[i] * w[i];
    double t[1] = {s};
    block_sum<1>(t);
    if (threadIdx.x == 0) part[c * gridDim.x + blockIdx.x] = t[0];
}

// h[c] = sum of the nb partials of column c, in block order (one block per column).
__global__ void __launch_bounds__(kBlock)
k_gm_dots_sum(int nb, const double *__restrict__ part, double *__restrict__ h, const CgScalars *sc)
{
    if (halted(sc)) return;
    const int c = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[c * nb + b];
    double t[1] = {s};
    block_sum<1>(t);
    if (threadIdx.x == 0) h[c] = t[0];
}

// w -= V[:, 0..ncols) h, and ||w|| of the result into gm->wnorm.
__global__ void __launch_bounds__(kBlock)
k_gm_orth(int n, int ncols, const double *__restrict__ V, const double *__restrict__ h,
          double *__restrict__ w, GmState *gm, const CgScalars *sc, double *part, unsigned *ticket)
{
    if (halted(sc)) return;
    __shared__ double hs[kGmMax + 1];
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) hs[c] = h[c];
    __syncthreads();
    double s2 = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double v = w[i];
        for (int c = 0; c < ncols; ++c) v -= hs[c] * V[static_cast<int64_t>(c) * n + i];
        w[i] = v;
        s2 += v * v;
    }
    double t[1] = {s2};
    if (grid_sum<1>(t, part, ticket) && threadIdx.x == 0) gm->wnorm = sqrt(t[0]);
}

// v_(j+1) = w / ||w|| (a zero w, an exact solution in the space, leaves zeros).
__global__ void __launch_bounds__(kBlock)
k_gm_scale(int n, const double *__restrict__ w, double *__restrict__ vnext, const GmState *gm,
           const CgScalars *sc)
{
    if (halted(sc)) return;
    const double inv = gm->wnorm > 0.0 ? 1.0 / gm->wnorm : 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) vnext[i] = w[i] * inv;
}

// Column j of the Hessenberg matrix (h1 + h2, ||w||), the earlier rotations
// applied to it, a new rotation zeroing its subdiagonal entry, the rotated
// right-hand side, and the step's book-keeping: residual norm |g_(j+1)|
// relative to ||Pi b||, history, convergence (a zero ||w|| means the space
// holds the exact solution: converged).  One thread.
__global__ void k_gm_givens(int j, GmState *gm, CgScalars *sc)
{
    if (halted(sc)) return;
    double *h = gm->H + j * (kGmMax + 1);
    for (int i = 0; i <= j; ++i) h[i] = gm->h1[i] + gm->h2[i];
    const double hn = gm->wnorm;
    h[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
        const double t = gm->cs[i] * h[i] + gm->sn[i] * h[i + 1];
        h[i + 1] = -gm->sn[i] * h[i] + gm->cs[i] * h[i + 1];
        h[i] = t;
    }
    const double d = hypot(h[j], h[j + 1]);
    sc->alpha = 0.0;
    if (!(d > 0.0) || !isfinite(d)) {
        // B v_j = 0 (or not finite): the step adds nothing; keep the others
        finish_step(sc, gm->g[j] * gm->g[j]);
        gm->j_done = j;
        sc->flag = kBreakdown;
        return;
    }
    const double c = h[j] / d, s = h[j + 1] / d;
    gm->cs[j] = c;
    gm->sn[j] = s;
    h[j] = d;
    h[j + 1] = 0.0;
    gm->g[j + 1] = -s * gm->g[j];
    gm->g[j] = c * gm->g[j];
    finish_step(sc, gm->g[j + 1] * gm->g[j + 1]);
    gm->j_done = j + 1;
    if (sc->flag == kRun && hn == 0.0) sc->flag = kConverged;
}

// End of a cycle: y = R^-1 g over the completed steps (back-substitution),
// then the flag is reset so that the true residual can be formed (the host
// keeps the step's stop reason).  One thread.
__global__ void k_gm_solve(GmState *gm, CgScalars *sc)
{
    const int k = gm->j_done;
    for (int i = k - 1; i >= 0; --i) {
        double s = gm->g[i];
        for (int c = i + 1; c < k; ++c) s -= gm->H[c * (kGmMax + 1) + i] * gm->y[c];
        gm->y[i] = s / gm->H[i * (kGmMax + 1) + i];
    }
    sc->stop = sc->flag;
    sc->flag = kRun;
}

// x += Z[:, 0..k) y, k = the cycle's completed steps.
__global__ void __launch_bounds__(kBlock)
k_gm_xupdate(int n, const double *__restrict__ Z, const GmState *gm, double *__restrict__ x)
{
    __shared__ double ys[kGmMax];
    const int k = gm->j_done;
    for (int c = threadIdx.x; c < k; c += blockDim.x) ys[c] = gm->y[c];
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double v = x[i];
        for (int c = 0; c < k; ++c) v += ys[c] * Z[static_cast<int64_t>(c) * n + i];
        x[i] = v;
    }
}

}  // namespace lap
