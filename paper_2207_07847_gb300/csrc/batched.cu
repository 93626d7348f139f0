// Batched solves: many (graph, right-hand side) pairs per launch.
#include "solver.cuh"

extern "C" lap_status lap_pcg_solve_batched(int32_t ng, const lap_handle *hs, const int32_t *nrhs,
                                            const double *const *d_B, double *const *d_X,
                                            void *stream, lap_solve_info *infos)
{
    (void)ng; (void)hs; (void)nrhs; (void)d_B; (void)d_X; (void)stream; (void)infos;
    return LAP_ERR_UNSUPPORTED;
}
