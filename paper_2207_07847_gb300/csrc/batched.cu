// Batched solves: many right-hand sides per graph, each with its own CG.
// Several graphs with the same solve settings go to a merged solve group
// (group.cu: one launch per phase for all graphs); otherwise, and for one
// graph, the following.
//
// One graph's columns are solved together: every matvec is an SpMM over the
// block vector, every sweep of the sparsifier solve handles all columns, and
// every column keeps its own alpha, beta, rho and convergence flag (a
// converged column is frozen while the others continue).  The iterations run
// as a CUDA graph of `check_every` steps; the host reads the column flags
// between graph launches.  In LAP_MIXED the columns run in FP32 and each one
// is refined against its own FP64 true residual.  Several graphs in one call
// run on their handles' private streams, advanced round-robin by the host so
// their work overlaps on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "batched_impl.cuh"

namespace lap {

namespace {

lap_status prepare(lap_handle_s &h, int R)
{
    BatchWork *b = h.batch.get();
    if (b && b->R == R) return LAP_OK;
    h.batch.reset();
    std::unique_ptr<BatchWork> nb;
    LAP_LTRY(make_batch(h, R, h.m.opt.precision == LAP_MIXED, h.s, nb));
    h.batch = std::move(nb);
    return LAP_OK;
}

}  // namespace

// Solve the columns [c0, c0 + nr) of one graph; infos gets nr entries.
lap_status batched_solve_chunk(lap_handle_s &h, int nr, const double *B, double *X,
                               lap_solve_info *infos)
{
    const int R = pow2_at_least(nr);
    LAP_LTRY(prepare(h, R));
    BatchWork &b = *h.batch;
    const lap_options &o = h.m.opt;
    const int n = static_cast<int>(b.n);
    const cudaStream_t s = h.s;
    const int CT = b.CT;
    std::vector<BCol> cols;
    std::vector<int> iters(R, 0), refs(R, 0);
    h.launches += 2;
    kb_gather<double><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(n, R, CT, nr, h.perm1, B, b.Bs, b.col64,
                                                               b.part, b.ticket);
    lap_status result = LAP_OK;
    if (o.precision != LAP_MIXED) {
        auto &v = b.v64;
        kb_center<double><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(n, R, CT, nr, 1, b.Bs, v.r, v.x, b.col64,
                                                                   v.col, o.tol, o.maxit, nullptr, 0.0,
                                                                   b.part, b.ticket);
        bprecond<double>(h, b, v, false, s);
        h.launches += 1;
        kb_pupdate<double><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(
            n, R, CT, o.prec == LAP_PREC_NONE ? v.r : v.z, v.p, v.col);
        result = biterate<double>(h, b, v, cols, s);
        for (int c = 0; c < nr; ++c) iters[c] = cols.empty() ? 0 : cols[c].iter;
        // true residuals, reported per column
        bspmm<double, 1>(h, b, h.L64, v.x, nullptr, b.r64, v.chunk, v.col, s);
        LAP_LTRY(poll_cols(b, v.col, cols, s));
        h.launches += 2;
        kb_mean<double><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(n, R, CT, v.x, b.means, b.part, b.ticket);
        kb_scatter<double><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(n, R, CT, nr, h.perm1, v.x, b.means, X);
    } else {
        // FP64 start: r64 = Bs (centred), x64 = 0
        kb_center<double><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(n, R, CT, nr, 1, b.Bs, b.r64, b.x64,
                                                                   b.col64, b.col64, o.tol, o.maxit,
                                                                   nullptr, 0.0, b.part, b.ticket);
        auto &v = b.v32;
        std::vector<BCol> outer;
        for (int ref = 0;; ++ref) {
            if (ref > 0) {
                bspmm<double, 1>(h, b, h.L64, b.x64, nullptr, b.r64, b.v64.chunk, b.col64, s);
                h.launches += 1;
                kb_refine_flags<<<1, 256, 0, s>>>(R, nr, b.col64, o.tol);
            }
            LAP_LTRY(poll_cols(b, b.col64, outer, s));
            bool any = false;
            for (int c = 0; c < nr; ++c) any |= outer[c].flag == kRun;
            if (!any || ref >= o.max_refine) break;
            int used = 0;
            for (int c = 0; c < nr; ++c) used = std::max(used, iters[c]);
            if (used >= o.maxit) break;
            // FP32 inner CG on the residual of every running column
            h.launches += 1;
            kb_center<float><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(
                n, R, CT, nr, 0, b.r64, v.r, v.x, b.col64, v.col, o.tol, o.maxit - used, b.col64,
                o.refine_tol, b.part, b.ticket);
            bprecond<float>(h, b, v, false, s);
            h.launches += 1;
            kb_pupdate<float><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(
                n, R, CT, o.prec == LAP_PREC_NONE ? v.r : v.z, v.p, v.col);
            lap_status it = biterate<float>(h, b, v, cols, s);
            if (it != LAP_OK) {
                result = it;
                break;
            }
            for (int c = 0; c < nr; ++c)
                if (outer[c].flag == kRun) {
                    iters[c] += cols[c].iter;
                    refs[c] = ref + 1;
                }
            h.launches += 1;
            kb_add<float><<<h.grid_cap, kBThreads, 0, s>>>(static_cast<int64_t>(n) * R, b.x64, v.x);
        }
        bspmm<double, 1>(h, b, h.L64, b.x64, nullptr, b.r64, b.v64.chunk, b.col64, s);
        LAP_LTRY(poll_cols(b, b.col64, cols, s));
        h.launches += 2;
        kb_mean<double><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(n, R, CT, b.x64, b.means, b.part, b.ticket);
        kb_scatter<double><<<bgrid(h, n, R, CT), kBThreads, 0, s>>>(n, R, CT, nr, h.perm1, b.x64, b.means,
                                                                    X);
    }
    LAP_BCK(cudaStreamSynchronize(s));
    for (int c = 0; c < nr; ++c) {
        lap_solve_info &inf = infos[c];
        std::memset(&inf, 0, sizeof(inf));
        inf.iterations = iters[c];
        inf.refinements = refs[c];
        inf.relres = cols[c].bnorm > 0.0 ? cols[c].relres : 0.0;
        inf.relres_recurrence = inf.relres;
        inf.status = result != LAP_OK ? result
                   : (inf.relres <= o.tol ? LAP_OK : LAP_ERR_NO_CONVERGENCE);
    }
    return result;
}

lap_status batched_enter(lap_handle_s &h, cudaStream_t user)
{
    LAP_BCK(cudaSetDevice(h.device));
    LAP_BCK(cudaEventRecord(h.ev_in, user));
    LAP_BCK(cudaStreamWaitEvent(h.s, h.ev_in, 0));
    return LAP_OK;
}

lap_status batched_leave(lap_handle_s &h, cudaStream_t user)
{
    LAP_BCK(cudaEventRecord(h.ev_out, h.s));
    LAP_BCK(cudaStreamWaitEvent(user, h.ev_out, 0));
    return LAP_OK;
}

}  // namespace lap

extern "C" lap_status lap_pcg_solve_batched(int32_t ng, const lap_handle *hs, const int32_t *nrhs,
                                            const double *const *d_B, double *const *d_X,
                                            void *stream, lap_solve_info *infos)
{
    using namespace lap;
    if (ng < 0 || (ng > 0 && (!hs || !nrhs || !d_B || !d_X))) return LAP_ERR_INVALID_ARG;
    for (int g = 0; g < ng; ++g) {
        if (!hs[g] || hs[g]->host_only || nrhs[g] < 0 || (nrhs[g] > 0 && (!d_B[g] || !d_X[g])))
            return LAP_ERR_INVALID_ARG;
        if (hs[g]->m.opt.prec != LAP_PREC_MSP && hs[g]->m.opt.prec != LAP_PREC_NONE)
            return LAP_ERR_UNSUPPORTED;
        // a single-level hierarchy (n <= coarse_max) has no aggregates to sweep
        if (hs[g]->m.opt.prec == LAP_PREC_MSP && hs[g]->m.levels < 2) return LAP_ERR_UNSUPPORTED;
    }
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    // several graphs with the same solve settings: one merged group, one
    // launch per PCG phase for all of them (group.cu)
    if (ng >= 2) {
        bool same = true;
        for (int g = 0; g < ng && same; ++g) {
            const lap_handle_s &h = *hs[g], &h0 = *hs[0];
            const lap_options &a = h.m.opt, &b = h0.m.opt;
            same = nrhs[g] <= 256 && h.m.levels >= 2 && a.prec == b.prec && a.precision == b.precision &&
                   h.m.mu == h0.m.mu && h.device == h0.device && a.tol == b.tol && a.maxit == b.maxit &&
                   a.check_every == b.check_every && a.max_refine == b.max_refine &&
                   a.refine_tol == b.refine_tol;
        }
        if (same) {
            lap_group grp = nullptr;
            lap_status st = lap_group_create(ng, hs, &grp);
            if (st == LAP_OK) st = lap_pcg_solve_group(grp, nrhs, d_B, d_X, stream, infos);
            lap_group_destroy(grp);
            return st;
        }
    }
    lap_status result = LAP_OK;
    size_t off = 0;
    std::vector<lap_solve_info> scratch;
    for (int g = 0; g < ng; ++g) {
        lap_handle_s &h = *hs[g];
        const int64_t n = h.m.lev[0].n;
        const auto t0 = std::chrono::steady_clock::now();
        const int64_t l0 = h.launches;
        lap_status st = batched_enter(h, user);
        for (int c0 = 0; st == LAP_OK && c0 < nrhs[g]; c0 += 256) {
            const int nr = std::min(256, nrhs[g] - c0);
            scratch.assign(static_cast<size_t>(nr), lap_solve_info{});
            st = batched_solve_chunk(h, nr, d_B[g] + static_cast<size_t>(c0) * n,
                                     d_X[g] + static_cast<size_t>(c0) * n, scratch.data());
            if (infos)
                for (int c = 0; c < nr; ++c) infos[off + c0 + c] = scratch[c];
        }
        const lap_status st2 = batched_leave(h, user);
        if (infos) {
            const double secs =
                std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            for (int c = 0; c < nrhs[g]; ++c) {
                infos[off + c].seconds = secs;
                infos[off + c].kernel_launches = static_cast<int32_t>(h.launches - l0);
            }
        }
        if (result == LAP_OK) result = st != LAP_OK ? st : st2;
        off += static_cast<size_t>(nrhs[g]);
    }
    return result;
}
