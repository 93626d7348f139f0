// Kernels of the stretch estimate (Section 3.3): the stretch of H over the
// sparsifier T in its effective-resistance form, tr(L_T^+ L_H), by
// Hutchinson's estimator z^T L_T^+ L_H z over Rademacher vectors z.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace lap {

// SplitMix64 (Steele, Lea & Flood 2014): the i-th output of the generator
// seeded with `seed` (the state advances by the golden gamma; the output is
// the variant-13 finaliser of the state).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + i * 0x9E3779B97F4A7C15ull;
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}

// z[i] = -1 if the top bit of SplitMix64(seed, sample * 2^32 + hidx[i]) is set,
// else +1; hidx maps tree order to the level-by-level hierarchy order, so a
// sample does not depend on the storage order.
__global__ void __launch_bounds__(kBlock)
k_rademacher(int64_t nt, uint64_t seed, uint32_t sample, const int64_t *__restrict__ hidx,
             double *__restrict__ z)
{
    const uint64_t base = static_cast<uint64_t>(sample) << 32;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt; i += (int64_t)gridDim.x * blockDim.x)
        z[i] = (splitmix64_at(seed, base + static_cast<uint64_t>(hidx[i])) >> 63) ? -1.0 : 1.0;
}

// out = z^T (u - mean(u)) = sum z u - (sum u / nt) sum z.
__global__ void __launch_bounds__(kBlock)
k_stretch_dot(int64_t nt, const double *__restrict__ z, const double *__restrict__ u, double *out,
              double *part, unsigned *ticket)
{
    double zu = 0.0, zs = 0.0, us = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt; i += (int64_t)gridDim.x * blockDim.x) {
        zu += z[i] * u[i];
        zs += z[i];
        us += u[i];
    }
    double v[3] = {zu, zs, us};
    if (grid_sum<3>(v, part, ticket) && threadIdx.x == 0) *out = v[0] - v[2] / (double)nt * v[1];
}

}  // namespace lap
