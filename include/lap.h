/*
 * lap.h -- C ABI of the GB300 solver for weighted graph Laplacian systems
 * L x = b, preconditioned by the multilevel expanded-graph preconditioners of
 * Hu & Lin, "Solving Graph Laplacians via Multilevel Sparsifiers".
 *
 * The method (citations are to the paper's sections and equations):
 *   - the aggregation hierarchy of Section 2.2 (random-order maximal-weight
 *     matching, leftovers join the aggregate of their heaviest neighbour,
 *     Galerkin coarse graphs), giving P^k and the composite prolongation
 *     P(mu) = [I, -mu P^2, ..., (-mu)^(l-1) P^l];
 *   - the expanded Laplacian L_Gt = P(mu)^T L P(mu) (Section 3.1,
 *     Eq. def:L_ell), its positively weighted subgraph H (PEGP, Section 3.2)
 *     and the multilevel sparsifier T of H (MSP, Section 3.3);
 *   - conjugate gradients on L x = b with the preconditioner
 *     B = Pi P(mu) M P(mu)^T Pi, M = L_T^+ (MSP) or ~L_H^+ (PEGP), Pi the mean
 *     projection.  This is the paper's expanded-system iteration (Section 4)
 *     recast on the original n unknowns; the paper's Krylov method is FGMRES.
 *
 * Conventions shared by every entry point:
 *   - Graphs are undirected, connected, given as symmetric CSR with both
 *     directions stored, no self-loops, no duplicate entries and strictly
 *     positive finite weights.  Vertex ids are 0-based.
 *   - "d_" pointers are CUDA device pointers; "h_" pointers are host memory.
 *     Vectors are contiguous FP64 arrays in the caller's vertex numbering.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is ordered on that stream; entry points that
 *     return results on the host synchronise it.
 *   - Right-hand sides need not have zero sum: the solver projects b onto
 *     the range of L (mean removed) and returns the zero-mean solution.
 *   - No entry point aborts, traps or prints.  Failures are reported by the
 *     returned lap_status; CUDA failures map to LAP_ERR_CUDA.
 *   - A handle may be used by one thread at a time; distinct handles are
 *     independent.
 */
#ifndef LAP_H
#define LAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lap_status {
    LAP_OK = 0,
    LAP_ERR_INVALID_ARG = 1,     /* bad pointer, size, option or layout       */
    LAP_ERR_NOT_SYMMETRIC = 2,   /* CSR is not symmetric (pattern or weight)  */
    LAP_ERR_NOT_CONNECTED = 3,   /* graph has more than one component         */
    LAP_ERR_BAD_WEIGHT = 4,      /* weight <= 0, NaN or Inf                   */
    LAP_ERR_OOM = 5,             /* device or host allocation failed          */
    LAP_ERR_CUDA = 6,            /* a CUDA call failed                        */
    LAP_ERR_NO_CONVERGENCE = 7,  /* maxit reached before the tolerance        */
    LAP_ERR_BREAKDOWN = 8,       /* p^T L p <= 0 or a non-finite CG scalar    */
    LAP_ERR_TIMEOUT = 9,         /* options.timeout_s elapsed                 */
    LAP_ERR_CANCELLED = 10,      /* request cancelled (serving)               */
    LAP_ERR_BUSY = 11,           /* no capacity (serving admission)           */
    LAP_ERR_UNSUPPORTED = 12     /* valid request this build does not handle  */
} lap_status;

/* Preconditioner M in B = Pi P(mu) M P(mu)^T Pi. */
typedef enum lap_prec {
    LAP_PREC_NONE = 0,        /* B = Pi: plain conjugate gradients            */
    LAP_PREC_MSP = 1,         /* M = L_T^+, multilevel sparsifier (Sec. 3.3)  */
    LAP_PREC_PEGP_INNER = 2,  /* M ~= L_H^+ by an inner CG on L_H with MSP     */
    LAP_PREC_PEGP_EXACT = 3   /* M = L_H^+ applied exactly: a dense inverse of
                                 the scaled L_H, computed on the device at
                                 setup (ntilde <= 16384, else setup returns
                                 LAP_ERR_UNSUPPORTED)                          */
} lap_prec;

typedef enum lap_precision {
    LAP_FP64 = 0,             /* every vector, matvec and sweep in FP64       */
    LAP_MIXED = 1             /* FP32 matvecs/sweeps with FP32 accumulation,
                                 FP64 dots, scalars, projection, coarsest
                                 solve and iterative-refinement residuals    */
} lap_precision;

/* Matching pass of the coarsening (Section 2.2). */
typedef enum lap_matching {
    LAP_MATCH_GREEDY = 0,     /* the paper's pass: vertices in (seeded) random
                                 order, each matched to its heaviest unmatched
                                 neighbour                                      */
    LAP_MATCH_HANDSHAKE = 1   /* deterministic parallel variant (a change of
                                 the method): rounds in which vertices pointing
                                 at each other (each at its heaviest unmatched
                                 neighbour, ties to the smaller id) are matched,
                                 until no unmatched vertex has an unmatched
                                 neighbour; seed and order_random are unused   */
} lap_matching;

/* Outer Krylov method of lap_pcg_solve. */
typedef enum lap_krylov {
    LAP_KRYLOV_CG = 0,        /* preconditioned CG (flexible for PEGP_INNER)     */
    LAP_KRYLOV_FGMRES = 1     /* flexible GMRES(restart), right preconditioning  */
} lap_krylov;

typedef struct lap_options {
    int32_t prec;          /* lap_prec (default LAP_PREC_MSP)                     */
    int32_t precision;     /* lap_precision (default LAP_FP64)                    */
    double mu;             /* 0 < mu < 1; mu <= 0 selects 1/sqrt(n) (default 0.8) */
    int32_t coarse_max;    /* stop coarsening once a level has <= coarse_max
                              vertices (default 32; 2 = the paper's "level =
                              max" with two top vertices)                          */
    int32_t max_levels;    /* cap on the number of levels, 0 = none (default 0)   */
    uint64_t seed;         /* seeds the random visit order (default 0)            */
    int32_t order_random;  /* 1: visit vertices in the hashed random order;
                              0: in increasing id order (default 1)               */
    double tol;            /* relative residual ||Pi b - L x|| / ||Pi b||, 1e-8   */
    int32_t maxit;         /* outer iteration cap (default 1000)                  */
    double inner_tol;      /* PEGP_INNER: inner CG stops at ||r~|| <= inner_tol *
                              ||r~_0|| (default 1e-2)                             */
    int32_t inner_maxit;   /* PEGP_INNER inner iteration cap (default 200)        */
    double refine_tol;     /* LAP_MIXED: relative tolerance of each FP32 inner
                              solve between FP64 residual refreshes (1e-4)        */
    int32_t max_refine;    /* LAP_MIXED: cap on refinement steps (default 20)     */
    int32_t check_every;   /* outer iterations between host convergence polls (8) */
    double timeout_s;      /* wall-clock limit per solve, <= 0: none (default 0)  */
    int32_t spmv_tpr;      /* matvec kernel: 0 = timed at setup (autotune), -1 =
                              SELL-32 slices, -2 = merge-path CSR (equal shares
                              of rows and entries per thread), t > 0 = CSR with
                              t threads per row                                 */
    int32_t host_only;     /* 1: build the host-side setup only and touch no GPU;
                              only the lap_get_* queries work on such a handle  */
    int32_t stall_window;  /* LAP_MIXED: an FP32 inner solve returns to refinement
                              once its residual has set no new minimum for this
                              many iterations (default 1000; 0 = never)         */
    int32_t krylov;        /* outer method: LAP_KRYLOV_CG (default) or
                              LAP_KRYLOV_FGMRES (the paper's, Section 4; LAP_FP64
                              solves only)                                       */
    int32_t restart;       /* FGMRES cycle length m, 1..128 (default 30)          */
    int32_t matching;      /* lap_matching: the coarsening's matching pass
                              (default LAP_MATCH_GREEDY, the paper's)           */
    int32_t setup_device;  /* 1: the hierarchy (matching, coarse graphs, degrees,
                              out-weights) and PEGP's L_H are built by device
                              kernels on the setup stream, bit-exact with the
                              host build; needs matching = LAP_MATCH_HANDSHAKE
                              (else LAP_ERR_INVALID_ARG); ignored with host_only.
                              Default 0: host threads                           */
    int32_t reserved[1];
} lap_options;

typedef struct lap_solve_info {
    int32_t status;            /* lap_status of this solve                        */
    int32_t iterations;        /* outer CG iterations (products with L)           */
    int32_t refinements;       /* LAP_MIXED: FP64 residual refreshes              */
    int32_t inner_iterations;  /* PEGP_INNER: total inner CG iterations           */
    int32_t restarts;          /* restarts from a recomputed true residual        */
    int32_t kernel_launches;   /* CUDA kernels launched by the call (graph nodes
                                  counted one by one)                              */
    double relres;             /* true relative residual of the returned x        */
    double relres_recurrence;  /* recurrence estimate at exit                     */
    double seconds;            /* host wall time of the call                      */
} lap_solve_info;

#define LAP_MAX_LEVELS 64

typedef struct lap_hierarchy_info {
    int32_t levels;                     /* l                                        */
    int32_t prec;                       /* preconditioner built at setup            */
    int64_t n;                          /* vertices of the input graph              */
    int64_t ntilde;                     /* vertices of the expanded graph, sum n_k  */
    int64_t nnz;                        /* stored CSR entries of the input graph    */
    int64_t level_size[LAP_MAX_LEVELS]; /* n_k, k = 1..l                            */
    int64_t nnz_H;                      /* stored off-diagonal entries of L_H       */
    int64_t edges_T;                    /* undirected edges of T                    */
    int64_t device_bytes;               /* device memory held by the handle         */
    double mu;                          /* the mu actually used                     */
} lap_hierarchy_info;

typedef struct lap_handle_s *lap_handle;

/* Fill *opts with the defaults listed above. */
void lap_options_default(lap_options *opts);

/* Static string naming a status code; never NULL. */
const char *lap_status_string(int32_t status);

/*
 * Route the library's device allocations through a caller allocator (for
 * example PyTorch's caching allocator).  alloc(ctx, bytes, stream) returns a
 * device pointer or NULL; release(ctx, ptr, stream) frees it.  Passing NULL
 * for both restores cudaMalloc/cudaFree.  Affects allocations made after the
 * call; set it once before the first lap_setup.
 */
typedef void *(*lap_alloc_fn)(void *ctx, size_t bytes, void *stream);
typedef void (*lap_free_fn)(void *ctx, void *ptr, void *stream);
lap_status lap_set_allocator(lap_alloc_fn alloc, lap_free_fn release, void *ctx);

/*
 * Build the solver for the graph (n, row_ptr[n+1], col_idx[nnz], w[nnz]) held
 * in host memory (copied; the caller keeps ownership).  Validates the CSR
 * (symmetry, weights, connectivity), builds the aggregation hierarchy
 * (Section 2.2), the sparsifier T (Section 3.3) and, for the PEGP
 * preconditioners, H (Section 3.2), and uploads everything to the current
 * CUDA device on `stream`.  Requires n >= 2.  opts == NULL uses the defaults.
 * On success *out owns device memory until lap_destroy.  LAP_PREC_PEGP_EXACT
 * with two or more levels also inverts the expanded Laplacian densely
 * (ntilde^2 doubles, plus ntilde^2 floats for LAP_MIXED; O(ntilde^3) FP64
 * work): LAP_ERR_UNSUPPORTED if ntilde > 16384, LAP_ERR_BREAKDOWN if a pivot
 * of the elimination is not positive.
 */
lap_status lap_setup(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                     const double *w, const lap_options *opts, void *stream,
                     lap_handle *out);

/* Release a handle and its device memory (synchronises its streams). NULL is ok. */
void lap_destroy(lap_handle h);

/*
 * Change the solve-time options of a handle: tol, maxit, inner_tol,
 * inner_maxit, refine_tol, max_refine, check_every, timeout_s, stall_window,
 * krylov, restart and precision.
 * precision may switch to LAP_MIXED only if the handle was set up with
 * LAP_MIXED (FP32 copies exist); switching to LAP_FP64 is always allowed.
 * Setup-time fields (prec, mu, coarse_max, max_levels, seed, order_random,
 * matching, spmv_tpr, host_only) are ignored.
 */
lap_status lap_update_options(lap_handle h, const lap_options *opts);

/*
 * Time one kernel of the solve on the handle's data, for roofline reports:
 *   kernel 0: CSR matvec with L          kernel 1: CSR matvec with L_H (PEGP)
 *   kernel 2: the whole MSP sweep B r    kernel 3: fused CG update + the first
 *                                                  upward band of the sweep
 *   kernel 4: the sweep's coarse tail    kernel 5: the last downward band
 *             (one block)                          (z and its reductions)
 *   kernel 6: the exact PEGP dense matvec y~ = G r~ (LAP_PREC_PEGP_EXACT)
 *   kernel 7: one iteration of the PEGP inner CG on L_H (matvec, step,
 *             expanded-space MSP sweep, reductions, new direction;
 *             LAP_PREC_PEGP_INNER)
 *   kernel 8: the expanded-space MSP solve y~ = L_T^+ f alone (PEGP inner)
 *   kernel 9: kernel 1 in the stored-diagonal form y = diag(L_H) x - W x
 *             (one multiply-add per entry instead of a subtraction and a
 *             multiply-add, the diagonal read too; the solves use kernel 1's
 *             edge-difference form)
 * in FP64 (precision 0) or FP32 (precision 1, LAP_MIXED handles).  Runs `reps`
 * back-to-back launches (sequences for kernels 2, 7, 8) on the handle's
 * stream timed by CUDA events and writes the mean milliseconds per launch and
 * the algorithmic bytes of one launch (every array the kernel must touch, read
 * or written once).  Overwrites the handle's solve workspace (kernel 7 first
 * fills the inner CG's vectors with fixed values; LAP_ERR_BREAKDOWN if its
 * iterations broke down while timed).  Kernels 3-5 need an MSP handle with at
 * least two levels, kernels 7-8 a PEGP inner handle with at least two levels,
 * else LAP_ERR_INVALID_ARG.
 */
lap_status lap_kernel_bench(lap_handle h, int32_t kernel, int32_t precision, int32_t reps,
                            double *ms_per_launch, double *bytes_per_launch);

/* Sizes of the hierarchy built by lap_setup. */
lap_status lap_get_hierarchy_info(lap_handle h, lap_hierarchy_info *info);

/*
 * Integer outputs of the setup, for bit-exact comparison: for level k
 * (1 <= k < l) write agg_out[u] = id of the level-(k+1) aggregate holding
 * level-k vertex u, both in the hierarchy's own numbering (level-1 ids are
 * the input ids; coarse ids are aggregate creation order).  agg_out has
 * level_size[k-1] entries.  pair_a/pair_b (optional, level_size[k] entries)
 * receive the two matched vertices that created each aggregate.
 */
lap_status lap_get_aggregates(lap_handle h, int32_t level, int32_t *agg_out,
                              int32_t *pair_a, int32_t *pair_b);

/*
 * Edge list of H (which = 0, Section 3.2) or T (which = 1, Section 3.3) in
 * the expanded numbering: level-k vertex u has index offset_k + u with
 * offset_k = n_1 + ... + n_{k-1} and u in the hierarchy's numbering.  Edges
 * are written once with i < j, sorted by (i, j).  With i == NULL only *count
 * is written.  Otherwise cap must be >= the count.  H requires a PEGP setup.
 */
lap_status lap_get_expanded_edges(lap_handle h, int32_t which, int64_t cap, int64_t *count,
                                  int64_t *i, int64_t *j, double *w);

/* --- device building blocks (each one step of the solve, FP64, device-resident) --- */

/* d_y = L d_x (n-vectors).  Section 2.1. */
lap_status lap_laplacian_apply(lap_handle h, const double *d_x, double *d_y, void *stream);

/* d_z = B d_r = Pi P(mu) M P(mu)^T Pi d_r with the handle's preconditioner
 * (n-vectors).  Eq. (1) preconditioner; Sections 3.2-3.3. */
lap_status lap_precond_apply(lap_handle h, const double *d_r, double *d_z, void *stream);

/* d_rt = P(mu)^T d_r: restriction to the expanded space (ntilde-vector in
 * the expanded numbering).  Section 2.2 composite prolongation. */
lap_status lap_restrict_apply(lap_handle h, const double *d_r, double *d_rt, void *stream);

/* d_z = P(mu) d_yt: prolongation from the expanded space.  Section 2.2. */
lap_status lap_prolong_apply(lap_handle h, const double *d_yt, double *d_z, void *stream);

/* d_yt = a solution of L_T y = d_rt (d_rt must sum to zero), by elimination
 * without fill-in over T's aggregates (Section 3.3) and a pseudo-inverse on
 * the top level; defined up to a constant vector. */
lap_status lap_msp_solve(lap_handle h, const double *d_rt, double *d_yt, void *stream);

/* d_yt = L_H d_xt (ntilde-vectors).  Section 3.2.  Requires a PEGP setup. */
lap_status lap_pegp_apply(lap_handle h, const double *d_xt, double *d_yt, void *stream);

/* --- solves --- */

/*
 * Solve L x = b by preconditioned CG (flexible CG for PEGP_INNER), or with
 * krylov = LAP_KRYLOV_FGMRES by flexible GMRES(restart) with right
 * preconditioning (FP64 only, else LAP_ERR_UNSUPPORTED; iterations count the
 * products with L, restarts the cycles after the first), to the handle's
 * tolerance.  d_b and d_x are device n-vectors (may not alias).
 * Synchronises `stream` before returning.  info may be NULL.  Returns LAP_OK
 * on convergence, LAP_ERR_NO_CONVERGENCE / LAP_ERR_BREAKDOWN /
 * LAP_ERR_TIMEOUT with the best x so far otherwise.
 */
lap_status lap_pcg_solve(lap_handle h, const double *d_b, double *d_x, void *stream,
                         lap_solve_info *info);

/*
 * Recurrence relative residuals ||r_k|| / ||Pi b|| of the outer iterations of
 * the handle's last solve, k = 1..count (FP64 solves; for LAP_MIXED the
 * entries are those of the FP32 inner solves, each relative to its own
 * right-hand side).  Writes at most cap values to h_out (host) and the
 * number recorded to *count (capped at the handle's maxit).
 */
lap_status lap_get_history(lap_handle h, double *h_out, int32_t cap, int32_t *count);

/*
 * CG coefficients of the first CG run of the handle's last solve (the whole
 * solve unless it restarted; for LAP_MIXED the first FP32 inner solve): the
 * step lengths alpha_j (x += alpha_j p_j) and the direction coefficients
 * beta_j (p_(j+1) = Pi z_(j+1) + beta_j p_j), j = 0..count-1, with beta of the
 * last step reported as 0.  Writes at most cap values to each of the host
 * arrays h_alpha and h_beta (either may be NULL) and the run's length to
 * *count.  LAP_ERR_INVALID_ARG for a host-only handle.
 */
lap_status lap_get_lanczos(lap_handle h, double *h_alpha, double *h_beta, int32_t cap,
                           int32_t *count);

/*
 * Extreme eigenvalues of the preconditioned operator B L on the complement of
 * the constants, estimated from the last solve's first CG run by the Lanczos
 * connection: the k x k tridiagonal with diagonal 1/alpha_j +
 * beta_(j-1)/alpha_(j-1) and off-diagonal sqrt(beta_j)/alpha_j has
 * eigenvalues (Ritz values) inside [lambda_min, lambda_max] of B L that
 * approach its extremes as k grows; lambda_max / lambda_min estimates, from
 * below, the condition number the paper bounds: the nonzero eigenvalues of
 * B L are those of M L_Gt, which for the exact PEGP lie in [1 - rho, 1]
 * (Section 3.2, spectral equivalence of Gt and H) and for MSP below the
 * stretch over 1 - rho (Section 3.3).  Computed on the host by Sturm-count
 * bisection.  *steps (may be NULL) receives k.  LAP_ERR_UNSUPPORTED for
 * LAP_PREC_PEGP_INNER (flexible CG has no Lanczos relation), LAP_ERR_INVALID_ARG
 * when the last solve ran no CG step (none yet, a zero right-hand side, or an
 * FGMRES solve), LAP_ERR_BREAKDOWN if a coefficient is not admissible.
 */
lap_status lap_estimate_condition(lap_handle h, int32_t *steps, double *lambda_min,
                                  double *lambda_max);

/*
 * Stretch of H over the sparsifier T (Section 3.3) in its effective-resistance
 * form, tr(L_T^+ L_H) = ||K_T||_F^2 = sum over H's edges of w_e R_T(e): at
 * least kappa(L_T^+ L_H) and at most the paper's path stretch.  Estimated by
 * Hutchinson's method: for s = 0..samples-1, h_vals[s] = z_s^T L_T^+ L_H z_s
 * (host array of `samples` doubles), whose mean is an unbiased estimate.
 * Entry i of z_s is -1 if the top bit of SplitMix64(seed, s * 2^32 + i) is
 * set, else +1, with i the expanded index level by level in hierarchy order
 * (aggregate creation order).  Each sample is one FP64 L_H matvec and one
 * expanded-space MSP solve on the device.  LAP_ERR_UNSUPPORTED unless the
 * handle was set up with a PEGP preconditioner and has two or more levels.
 */
lap_status lap_estimate_stretch(lap_handle h, int32_t samples, uint64_t seed, double *h_vals);

/* Same as lap_pcg_solve with host vectors: copies b in and x out on `stream`
 * (the copies are part of the call). */
lap_status lap_pcg_solve_host(lap_handle h, const double *h_b, double *h_x, void *stream,
                              lap_solve_info *info);

/*
 * Solve many systems together: graph g in [0, ng) has nrhs[g] right-hand
 * sides stored column after column in d_B[g] (n_g * nrhs[g] doubles, column
 * j at offset j * n_g); solutions go to d_X[g] in the same layout.  All
 * handles must use LAP_PREC_MSP (with at least two levels) or LAP_PREC_NONE,
 * else LAP_ERR_UNSUPPORTED.  Every (graph, column)
 * pair runs its own CG with its own scalars and stops on its own; the
 * matvecs and sweeps of all pairs are batched.  infos (optional) receives
 * sum(nrhs) entries in (graph, column) order.  Two or more graphs whose
 * handles share the solve settings (precision, mu, tol, maxit, check_every,
 * refinement) and have at most 256 right-hand sides each are merged into a
 * temporary solve group (lap_group_create below: one launch per PCG phase
 * for all graphs); otherwise the graphs are solved one after another.
 */
lap_status lap_pcg_solve_batched(int32_t ng, const lap_handle *hs, const int32_t *nrhs,
                                 const double *const *d_B, double *const *d_X, void *stream,
                                 lap_solve_info *infos);

/*
 * Solve groups: many graphs of uneven size solved together with one launch
 * per PCG phase for all of them (the scope table's batched row: graphs
 * concatenated block-diagonally with per-graph segment ids and per-(graph,
 * column) CG scalars; the paper solves one system at a time, Section 4).
 *
 * lap_group_create merges the setups of ng handles (caller-owned; they must
 * outlive the group, which uses their top-level dense pseudo-inverses in
 * place): all with LAP_PREC_MSP or all with LAP_PREC_NONE (else
 * LAP_ERR_UNSUPPORTED; the PEGP preconditioners are refused: their inner
 * solves on L_H run per graph), every hierarchy with at least two levels
 * (LAP_ERR_UNSUPPORTED), the same precision, mu and device
 * (LAP_ERR_INVALID_ARG).  The merge copies the graphs' level-1 Laplacians,
 * aggregation segments and elimination coefficients into one block-diagonal
 * layout on the device (graphs ordered by decreasing hierarchy depth); the
 * solve options (tol, maxit, check_every, refinement) are the first
 * handle's at creation.
 *
 * lap_pcg_solve_group solves graph g's nrhs[g] (0..256) right-hand sides
 * d_B[g] (column-major, n_g x nrhs[g], device) into d_X[g] (same layout) on
 * `stream`, every (graph, column) pair with its own CG (and, with
 * LAP_MIXED, its own FP64 refinement), stopping on its own.  Each PCG phase
 * (matvec, each sweep level, the graphs' top-level solves, the direction
 * update) is one launch over all graphs; the iterations run as CUDA graphs
 * of check_every steps.  infos (optional, host) receives sum(nrhs) entries in
 * (graph, column) order.  Reuses its workspace between calls of the same
 * maximum width; one call at a time per group.
 */
typedef struct lap_group_s *lap_group;
lap_status lap_group_create(int32_t ng, const lap_handle *hs, lap_group *out);
lap_status lap_pcg_solve_group(lap_group grp, const int32_t *nrhs, const double *const *d_B,
                               double *const *d_X, void *stream, lap_solve_info *infos);
void lap_group_destroy(lap_group grp);

/*
 * Residual of a graph Laplacian system without any device allocation.
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory at all: code inside a process whose
 * device-memory quota is already spent (an out-of-memory handler that still
 * has to report how good the last iterate is), or code that must not touch
 * an allocator it shares with other work.  It needs no handle and no
 * allocator:
 *
 *   d_r[i] = (b_i - mean(b)) - sum_j w_ij (x_i - x_j)     (r = Pi b - L x)
 *   h_norms[0] = ||r||_2,  h_norms[1] = ||Pi b||_2        (written on the host)
 *
 * for the graph (n, d_row_ptr[n+1] int64, d_col_idx[nnz] int32, d_w[nnz]) in
 * DEVICE memory, symmetric CSR as everywhere in this library (not checked:
 * out-of-range indices are the caller's error).  d_x, d_b, d_r are device
 * n-vectors; d_r may not alias d_x or d_b.  The call synchronises `stream`.
 *
 * Scratch: a fixed 1 MiB __device__ array inside this library (every GPU that
 * loads the library holds it until the process exits) keeps one partial sum
 * per 256-row tile, so n may be at most 16,777,216; larger n returns
 * LAP_ERR_UNSUPPORTED before any work is queued.  The first call on a device
 * looks the array's device address up (cudaGetSymbolAddress) and caches it:
 * make that first call before any stream capture.  All calls on a device
 * share the one array, so calls that overlap on the GPU (different streams,
 * threads or processes sharing a context) race and must be serialised by the
 * caller.  Allocates nothing: no cudaMalloc, no cudaFree, no library
 * allocator.  A launch that fails (no kernel image for the device, a bad
 * launch configuration) returns LAP_ERR_CUDA and leaves h_norms unwritten.
 */
lap_status lap_laplacian_residual_noalloc(int64_t n, const int64_t *d_row_ptr,
                                          const int32_t *d_col_idx, const double *d_w,
                                          const double *d_x, const double *d_b, double *d_r,
                                          double *h_norms, void *stream);

/* --- serving: continuous batching of solve requests ---
 *
 * A server answers a stream of solve requests L_h X = B on set-up graphs.  It
 * extends the batched solve above to requests that arrive at any time (the
 * paper solves one system at a time; serving is this library's addition).
 * Every graph with requests in flight has a resident column batch of R
 * columns (R = the smallest power of two >= max(8, max_slots), at most 256)
 * on its own CUDA stream; a request occupies nrhs contiguous columns of its
 * graph's batch.  One worker thread alternates between
 *   - admission: queued requests take free columns; a graph without a batch
 *     gets one if the device memory of all batches stays within
 *     hbm_budget_bytes (the first batch is always admitted);
 *   - one launch of check_every CG iterations of every batch (the batches of
 *     different graphs overlap on the device).  New requests join a running
 *     batch at this boundary: only their columns are started, the other
 *     columns keep their iterates, directions and scalars;
 *   - retirement: a request whose columns have all stopped (converged,
 *     iteration limit, breakdown, cancelled, timed out) gets its solution
 *     (mean-zero, caller's vertex numbering) written to its d_X, its info
 *     filled and its callback called; its columns become free at once.
 * On a LAP_FP64 handle the columns run in FP64, and a column whose recurrence
 * converged while its true residual did not restarts from the true residual
 * (at most 4 times).  On a LAP_MIXED handle the columns run the FP32 CG and
 * each request is refined against its FP64 true residual (refine_tol,
 * max_refine as for lap_pcg_solve): when its inner solves have stopped, the
 * corrections go into its FP64 solution and the columns still above the
 * tolerance start the next inner solve.  tol, maxit and timeout_s come from
 * the handle's options.  Every column's arithmetic is
 * independent of the other columns and of the moment it joined, so a
 * request's result is bitwise the same whether it ran alone or with others
 * on the same server (same handle, same max_slots).
 *
 * Threading: the calls below are thread-safe.  While a server holds requests
 * of a handle, that handle may not be used by any other call (its launch
 * counter and CUDA graphs belong to the worker), and lap_destroy(h) may be
 * called only once they have all finished.
 */

typedef struct lap_server_s *lap_server;

typedef struct lap_server_options {
    int64_t hbm_budget_bytes;  /* device memory all resident batches may hold (bytes) */
    int32_t max_slots;         /* columns per graph batch (1..256, rounded up, >= 8) */
    int32_t check_every;       /* CG iterations between admission / retirement
                                * points (<= 0: the handle's check_every)          */
    int32_t reserved[8];
} lap_server_options;

/* Called on the server's worker thread when a request finishes, after its
 * solution has been written (d_X is complete when the callback runs). */
typedef void (*lap_done_cb)(void *user, uint64_t req_id, const lap_solve_info *info);

/* Defaults: 32 GiB budget, 16 slots, check_every 8. */
void lap_server_options_default(lap_server_options *opts);

/* Start a server (worker thread) on the current device.  LAP_ERR_INVALID_ARG
 * for max_slots outside 1..256 or a budget <= 0. */
lap_status lap_server_create(const lap_server_options *opts, lap_server *out);

/*
 * Queue a request: solve L_h X = B for nrhs columns (column-major as in
 * lap_pcg_solve_batched: d_B and d_X hold n * nrhs doubles, column j at
 * offset j * n; device pointers that must stay valid, and d_B unchanged,
 * until the request has finished).  Returns at once with *req_id (ids start
 * at 1).  cb (optional) is called on completion.  Errors, returned before
 * anything is queued: LAP_ERR_INVALID_ARG (null pointer, host-only handle,
 * nrhs < 1 or nrhs > the batch width R), LAP_ERR_UNSUPPORTED (a
 * preconditioner other than LAP_PREC_MSP with >= 2 levels or LAP_PREC_NONE),
 * LAP_ERR_BUSY (one batch of this graph alone exceeds hbm_budget_bytes),
 * LAP_ERR_CANCELLED (the server is shutting down).
 */
lap_status lap_serve_submit(lap_server s, lap_handle h, int32_t nrhs, const double *d_B,
                            double *d_X, lap_done_cb cb, void *user, uint64_t *req_id);

/*
 * Block until request req_id has finished or timeout_s seconds have passed
 * (timeout_s <= 0: no limit).  On completion writes its info (seconds = time
 * from submission to completion, kernel_launches = kernels of its batch
 * while it was resident), forgets the id and returns the request's status;
 * otherwise returns LAP_ERR_TIMEOUT and the request goes on.  An unknown (or
 * already waited-for) id gives LAP_ERR_INVALID_ARG.
 */
lap_status lap_serve_wait(lap_server s, uint64_t req_id, double timeout_s, lap_solve_info *info);

/* Cancel a queued or running request: it finishes at the next retirement
 * point with status LAP_ERR_CANCELLED (a running one with its current iterate
 * written to d_X).  No effect on a finished request. */
lap_status lap_serve_cancel(lap_server s, uint64_t req_id);

/* Cancel the queued requests, finish the admitted ones (callbacks run), stop
 * the worker and free the server and its batches. */
void lap_server_destroy(lap_server s);

#ifdef __cplusplus
}
#endif

#endif /* LAP_H */
