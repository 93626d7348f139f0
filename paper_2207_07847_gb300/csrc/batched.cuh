// Batched solve entry points shared by the C ABI and the server.
#pragma once

#include <cuda_runtime.h>

#include "lap.h"

struct lap_handle_s;

namespace lap {

#define LAP_LTRY(x)                       \
    do {                                  \
        lap_status s_ = (x);              \
        if (s_ != LAP_OK) return s_;      \
    } while (0)

// Solve nr <= 256 columns of one graph (column-major device B/X, column j at
// offset j * n) on the handle's private stream; writes nr infos.
lap_status batched_solve_chunk(lap_handle_s &h, int nr, const double *B, double *X,
                               lap_solve_info *infos);
lap_status batched_enter(lap_handle_s &h, cudaStream_t user);
lap_status batched_leave(lap_handle_s &h, cudaStream_t user);

}  // namespace lap
