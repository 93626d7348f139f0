// Solver handle and the host-side entry points shared by the C ABI files.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <vector>

#include "device_model.cuh"
#include "lap_internal.h"

namespace lap {
struct BatchWork;   // batched-solve workspace (batched.cu)
struct GmState;     // FGMRES cycle state (fgmres.cuh)
}

struct lap_handle_s {
    lap::HostModel m;
    bool host_only = false;
    int device = 0;
    int sms = 0;
    int grid_cap = 0;                 // resident 256-thread blocks on the device
    cudaStream_t s = nullptr;         // private stream (graphs are captured on it)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<std::unique_ptr<lap::DevBuf>> bufs;
    int64_t device_bytes = 0;

    lap::DevCsr<double> L64;
    lap::DevCsr<float> L32;
    lap::DevMsp<double> M64;
    lap::DevMsp<float> M32;
    lap::DevCsr<double> H64;          // L_H (PEGP), expanded tree order
    lap::DevCsr<float> H32;
    double *G64 = nullptr;            // exact PEGP: dense L_H^+ (up to a constant), tree order
    float *G32 = nullptr;             // its FP32 copy (mixed precision)
    int64_t g_ld = 0;                 // leading dimension of G64 / G32
    int tpr = 8, tprH = 8;            // threads per CSR row

    int *perm1 = nullptr;             // tree position -> input vertex id
    int64_t *xmap = nullptr;          // tree expanded index -> hierarchy expanded index
    double *bs = nullptr;             // centred right-hand side (tree order)
    double *bin = nullptr, *xout = nullptr;   // staging for host-vector solves

    lap::CgVectors<double> w64;       // FP64 CG on L
    lap::CgVectors<float> w32;        // FP32 inner CG of mixed precision
    lap::CgVectors<double> e64;       // expanded-space CG (PEGP inner solve)
    lap::CgVectors<float> e32;
    lap::CgState st64, st32, ste64, ste32, stb;   // scalars + reduction scratch
    lap::CgScalars *hsc = nullptr;    // pinned host mirror of one CgScalars

    cudaGraphExec_t g_iter64 = nullptr, g_iter32 = nullptr;
    cudaGraphExec_t g_in64 = nullptr, g_in32 = nullptr;   // PEGP inner-iteration chunks
    int64_t nodes_iter64 = 0, nodes_iter32 = 0, nodes_in64 = 0, nodes_in32 = 0;
    mutable int64_t launches = 0;     // kernels launched (graph replays add their nodes)
    double *hist = nullptr;           // device history of the last solve (maxit entries)
    int hist_count = 0;
    int hist_capacity = 0;
    double *lz = nullptr;             // (alpha, beta) per outer step, 2 * hist_capacity
    int lz_run = 0;                   // steps of the last solve's first CG run
    // FGMRES (allocated by the first FGMRES solve): basis V (m + 1 columns),
    // preconditioned vectors Z (m columns), cycle state, dot partials, and
    // the captured cycle
    double *gm_V = nullptr, *gm_Z = nullptr, *gm_part = nullptr;
    lap::GmState *gm = nullptr;
    int gm_m = 0;
    cudaGraphExec_t g_gm = nullptr;
    int64_t nodes_gm = 0;
    std::shared_ptr<lap::BatchWork> batch;   // allocated by the first batched solve
    int batch_ct[6] = {0, 0, 0, 0, 0, 0};   // tuned column tile per batch width 8..256
};

namespace lap {

lap_status upload_model(lap_handle_s &h, cudaStream_t user);
void destroy_handle(lap_handle_s &h);

lap_status block_laplacian(lap_handle_s &h, const double *x, double *y, cudaStream_t user);
lap_status block_precond(lap_handle_s &h, const double *r, double *z, cudaStream_t user);
lap_status block_restrict(lap_handle_s &h, const double *r, double *rt, cudaStream_t user);
lap_status block_prolong(lap_handle_s &h, const double *yt, double *z, cudaStream_t user);
lap_status block_msp_solve(lap_handle_s &h, const double *rt, double *yt, cudaStream_t user);
lap_status block_pegp(lap_handle_s &h, const double *xt, double *yt, cudaStream_t user);

lap_status solve_device(lap_handle_s &h, const double *b, double *x, cudaStream_t user,
                        lap_solve_info &info);
lap_status solve_host(lap_handle_s &h, const double *b, double *x, cudaStream_t user,
                      lap_solve_info &info);
lap_status update_options(lap_handle_s &h, const lap_options &o);
lap_status get_history(lap_handle_s &h, double *out, int cap, int *count);
lap_status get_lanczos(lap_handle_s &h, double *alpha, double *beta, int cap, int *count);
lap_status estimate_stretch(lap_handle_s &h, int samples, uint64_t seed, double *vals);
lap_status kernel_bench(lap_handle_s &h, int kernel, int precision, int reps, double *ms,
                        double *bytes);

}  // namespace lap
