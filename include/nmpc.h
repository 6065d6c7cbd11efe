/* nmpc.h -- C ABI of the GB300-native parametric interior-point NMPC library.
 *
 * The library implements the per-iteration hot path of the parametric
 * interior-point method of arXiv 2606.04725 (Sec. 3.2, Algorithms 1 and 2):
 * stage-parallel derivative evaluation, assembly of the condensed Lifted-KKT
 * matrix (eq. liftedkkt-pd) into a fixed pattern, numeric supernodal factorization
 * (the Cholesky of eq. cholesky-numeric in its square-root-free form K = L D L^T)
 * against a symbolic analysis done once (eqs. cholesky-symCholesky,
 * cholesky-numCholesky), triangular solves (eqs. cholesky-lower/upper/delta),
 * line search (eq. infiniteOCP-lineSearch) and barrier/termination control
 * (eqs. infiniteOCP-innerTol/outerTol).  Every numeric step runs in CUDA
 * kernels for sm_103a in FP64; there is no CPU fallback.
 *
 * Conventions for every entry point:
 *  - Return value: NMPC_OK or an error status; no entry point aborts, exits
 *    or throws.  nmpc_last_error() gives a message for the last failure.
 *  - Pointers are owned by the caller and are not retained past the call.
 *    "on_device" arguments say whether the caller's arrays are device
 *    pointers (1) or host pointers (0).  Host arrays may be pageable.
 *  - All device work is ordered on the CUDA stream given to nmpc_build.
 *    Calls that read or write host memory synchronize that stream before
 *    returning; calls with device arrays return without synchronizing.
 *  - Device memory is not allocated by the library: nmpc_build performs the
 *    one-time host analysis and reports the workspace size; the caller
 *    allocates it (for example as a torch.uint8 tensor) and hands it over
 *    with nmpc_bind.  The workspace must stay valid until nmpc_destroy.
 *  - Layout of one instance's primal vector y (stage-interleaved):
 *      y = [ x_0 | x_1 u_1 | ... | x_T u_T ],  n = nx + T (nx + nu)
 *    with nx states and nu controls per stage (for the DAE column the
 *    "controls" are [y (N) u L V S]); rows of h are the initial condition
 *    x_0 - p_x0 = 0 followed by the T backward-Euler steps, nr rows each
 *    (nx, or 2N + 3 for the DAE column: its balances, then its algebraic rows).
 */
#ifndef NMPC_H
#define NMPC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nmpc_handle nmpc_handle;

typedef enum {
  NMPC_OK = 0,
  NMPC_ERR_INVALID = 1,      /* bad argument (size, pointer, state of the handle) */
  NMPC_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  NMPC_ERR_WORKSPACE = 3,    /* workspace missing or too small */
  NMPC_MAX_ITER = 10,        /* interior-point iteration limit reached */
  NMPC_LINESEARCH_FAIL = 11, /* step size fell below alpha_min (no restoration phase) */
  NMPC_INERTIA_FAIL = 12,    /* regularization delta_w exceeded its maximum */
  NMPC_NONFINITE = 13,       /* NaN or Inf in the residuals */
  NMPC_TIMEOUT = 14,         /* a bounded device wait gave up */
  NMPC_NOT_SOLVED = 15       /* no converged solution is available yet */
} nmpc_status;

typedef enum {
  NMPC_MODEL_DISTILLATION = 0, /* binary column of Sec. 4.1 (eq. distill-ocp) */
  NMPC_MODEL_PLATE = 1,        /* linear heated plate, boundary flux actuators */
  NMPC_MODEL_TOY = 2,          /* dy/dt = 4 sin u - y^3 of the paper's code listing */
  NMPC_MODEL_PAPER_PLATE = 3,  /* the paper's nonlinear heated plate (Sec. 4.2, eq. pde-ocp): n x n
                                  nodes on [-1,1]^2 (n in g), the (n-2)^2 interior temperatures as
                                  states, one control Q >= 50 that sets the Dirichlet data
                                  4.1 Q^(1/3) at x1 = -1 and Q^(1/2) at x2 = -1 (T_b elsewhere),
                                  heat loss, tracking of the region [-0.5,0.5]^2 to one setpoint
                                  per stage, rho Q^2 */
  NMPC_MODEL_DISTILLATION_DAE = 4 /* the column of eq. (distill-ocp) as printed, with its algebraic
                                  variables: per stage [x (N) | y (N) u L V S], per step the N
                                  balances, the N equilibria y = a x / (1 + (a-1) x) and
                                  L = uD, V = L + D, S = L + F as rows; y in [0,1], L, V, S in
                                  [0, 10]; the constants and cost of NMPC_MODEL_DISTILLATION */
} nmpc_model;

typedef enum {
  NMPC_ORDER_AUTO = 0,         /* chosen by the autotuner (or a size rule) */
  NMPC_ORDER_NATURAL = 1,      /* stage order: elimination tree is a chain */
  NMPC_ORDER_ND = 2,           /* geometric nested dissection (time, then space) */
  NMPC_ORDER_TWO_SIDED = 3     /* nested dissection whose leaves of nd_leaf stages (the whole horizon
                                  when nd_leaf <= 1) are eliminated from both ends toward their middle
                                  stage: the flops of stage order with half its chain length */
} nmpc_ordering;

typedef enum {
  NMPC_KKT_LIFTED = 0,         /* Lifted-KKT (eqs. liftedkkt, liftedkkt-pd): h relaxed to |h| <= gamma */
  NMPC_KKT_HYKKT = 1           /* HyKKT (Sec. 3.2.2): equalities kept, augmented Cholesky plus CG */
} nmpc_kkt;

/* Problem description.  All instances share the model and its constants;
 * each instance has its own horizon T (block-diagonal batch, one KKT block
 * per instance).  Fill it with nmpc_problem_defaults first. */
typedef struct {
  int model;             /* nmpc_model */
  int n_instances;       /* >= 1 */
  const int* horizons;   /* n_instances horizons T >= 1 (host pointer) */
  int N;                 /* distillation: trays, condenser = 1, reboiler = N */
  int Nf;                /* distillation: feed tray (1-based, 2 <= Nf <= N-1) */
  int g;                 /* plate: grid side (cells), g % (S/4) == 0 */
  int S;                 /* plate: actuator segments, multiple of 4 */
  double dt;             /* time step of the backward-Euler transcription */
  double alpha, D, F, xF, Ac, At, Ar, wdu; /* distillation constants */
  double kappa, cq, rho_u;                 /* plate constants */
  double xlo, xhi, ulo, uhi;               /* bounds of x_1..x_T and u_1..u_T (+-INFINITY allowed) */
  double wu, ubar;       /* distillation: control-tracking stage cost wu dt (u_k - ubar)^2, the
                            0.1 (u - ubar)^2 integrand of eq. (distill-ocp), Sec. 4.1, by the
                            rectangle rule; wu = 0 (default) leaves it out */
  double Tb, qloss;      /* paper's plate: fixed boundary temperature and heat loss (table
                            pde-params: 50, 10); its alpha is kappa (230) and its rho rho_u (1e-8) */
} nmpc_problem;

/* Solver options.  Defaults from nmpc_options_defaults. */
typedef struct {
  double tol;            /* outer tolerance on the scaled optimality error E_0 (1e-8) */
  double gamma;          /* Lifted-KKT relaxation -gamma <= h <= gamma (1e-8) */
  double mu0_cold;       /* initial barrier parameter, cold start (0.1) */
  double mu0_warm;       /* initial barrier parameter, warm start (1e-8) */
  double push_cold;      /* bound push of the initial point, cold (1e-2) */
  double push_warm;      /* bound push of the initial point, warm (1e-9) */
  int max_iter;          /* interior-point iteration limit (200) */
  int ordering;          /* nmpc_ordering */
  int nd_leaf;           /* nested dissection: stages per leaf (1); two-sided order: stages per
                            two-sided leaf, <= 1 for the whole horizon */
  int use_graph;         /* run the interior-point loop as one CUDA graph with device-set
                            conditional nodes (1, default); 0: host-driven loop, same kernels */
  long long spin_limit;  /* iteration limit of bounded device waits (1e7) */
  double pivtol;         /* inertia test: a pivot must exceed pivtol * |K_jj| (1e-12) */
  int factor_mode;       /* 0: cluster-cooperative fronts where they fit, the blocked large-front
                            path elsewhere (default); 1: one CTA per front; 2: blocked path everywhere;
                            3: dataflow: one persistent launch factors the leading levels whose
                            fronts fit one CTA's shared memory, each front starting as soon as its
                            children are done (no per-level launches), then mode 0 above them */
  int solve_mode;        /* 0: persistent dataflow solves over the levels of small fronts (default);
                            1: one launch per level */
  int panel_scale;       /* triangular solves of the fronts solved one block per front:
                            0: automatic (default): form 1 below when the solves are latency-bound
                               (at most 4 fronts per SM in every level), else form 3;
                            1: after each factorization the 16x16 unit diagonal blocks of L are
                               inverted in place and the rows below each block are multiplied by
                               its inverse: one dense product per block and solve;
                            2: the diagonal blocks only: two products per block;
                            3: no transform: column-by-column substitution */
  int amalgamation;      /* relaxed amalgamation of fundamental supernodes (Sec. 3.2.3 supernodes):
                            0: automatic (default): 2 where every front of the partition
                               of 1 has at most 128 rows (small, latency-bound fronts),
                               else 1; values outside 0..2 make nmpc_build fail with
                               NMPC_ERR_INVALID;
                            1: relaxed: a supernode whose columns end right before its parent's
                               merges into it while the merged panel's explicit zeros stay
                               under a limit that falls with the panel's width;
                            2: sibling-limited: as 1, but a supernode whose parent has other
                               children merges only into a panel of at most 16 columns, so
                               the separators of nested dissection stay separate fronts */
  double dw_max;         /* inertia correction (eq. infiniteOCP-inertia, W&B Algorithm IC):
                            an instance whose regularization delta_w would exceed dw_max
                            stops with NMPC_INERTIA_FAIL (1e40) */
  int kkt;               /* Newton system (nmpc_kkt): NMPC_KKT_LIFTED (default), or NMPC_KKT_HYKKT,
                            the alternative to lifting that Sec. 3.2.2 names: the equalities
                            h = 0 keep their multipliers lambda, K_gamma = W + Sigma_y +
                            delta_w I + hykkt_gamma H^T H is assembled into the same factor
                            pattern and factored by the same kernels (its positive pivots are
                            the inertia test), and conjugate gradients on the Schur complement
                            H K_gamma^-1 H^T, one pair of triangular solves per CG iteration,
                            give lambda's step (Regev et al. 2023, after Golub & Greif 2003);
                            gamma is then unused.  nmpc_sensitivity needs the lifted form. */
  double hykkt_gamma;    /* HyKKT augmentation weight (1e4) */
  double cg_tol;         /* HyKKT: CG stops when ||r||_2 <= cg_tol ||r_0||_2 (1e-12) */
  int cg_max_iter;       /* HyKKT: CG iterations per Newton step at most (200) */
} nmpc_options;

/* Per-instance result of a solve.  Times are measured with CUDA events on
 * the library stream and cover the whole solve call. */
typedef struct {
  int status;            /* nmpc_status of this instance */
  int iters;             /* interior-point iterations */
  int inertia_retries;   /* factorizations repeated with a larger delta_w */
  int ls_trials;         /* line-search trial points evaluated */
  double mu_final;
  double kkt_scaled;     /* scaled E_0 at the returned point */
  double kkt_unscaled;
  double objective;
  double ms_total;       /* whole solve call (same for all instances) */
  int cg_iters;          /* HyKKT: conjugate-gradient iterations of this solve (0 for Lifted-KKT) */
} nmpc_info;

typedef struct {
  int n_total, m_total;      /* primal variables / equality rows over all instances */
  int n_supernodes, n_levels;
  long long nnz_L;           /* stored entries of the supernodal factor (lower panels) */
  double factor_flops;       /* floating-point operations of one numeric factorization */
  double solve_flops;        /* of one forward + backward solve */
  long long workspace_bytes;
  double analysis_ms;        /* host time of the one-time structure analysis */
  int max_front;             /* largest frontal matrix order */
  int ordering_used;
  long long kernel_launches; /* kernels launched by this handle so far */
  int amalgamation_used;     /* supernode amalgamation of the last instance (1 relaxed, 2 sibling-limited) */
} nmpc_stats;

/* Average device time (CUDA events on the library stream) of the phases of
 * one interior-point iteration, re-run at the current iterate. */
typedef struct {
  double ms_eval;            /* stage-parallel residual/Jacobian/Hessian evaluation */
  double ms_assemble;        /* condensed-matrix assembly into the factor pattern */
  double ms_factor;          /* numeric supernodal factorization (L D L^T) */
  double ms_solve;           /* right-hand side, forward and backward solves */
  int reps;
} nmpc_phase_times;

void nmpc_problem_defaults(int model, nmpc_problem* prob);
void nmpc_options_defaults(nmpc_options* opts);

/* One-time structure analysis (Sec. 3.2.3, Algorithm 2 "SymCholesky" and the
 * transcription): Jacobian/Hessian patterns, condensed pattern, ordering P,
 * elimination tree, supernodes, level sets, L layout and scatter maps.
 * Host work only; no device memory is touched.  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).  On success *out owns the
 * analysis; query nmpc_workspace_bytes and call nmpc_bind next. */
nmpc_status nmpc_build(const nmpc_problem* prob, const nmpc_options* opts, void* cuda_stream,
                       nmpc_handle** out);

/* Device workspace size in bytes required by nmpc_bind (256-byte aligned). */
nmpc_status nmpc_workspace_bytes(const nmpc_handle* h, size_t* bytes);

/* Hand over caller-allocated device memory (workspace, >= nmpc_workspace_bytes,
 * 256-byte aligned) and upload the structure.  Must be called once before
 * set_params/solve.  The memory stays owned by the caller. */
nmpc_status nmpc_bind(nmpc_handle* h, void* workspace, size_t bytes);

/* Parameter update without rebuilding anything (Sec. 3.3,
 * set_parameter_value; Algorithm 1 last line).  instance = -1 sets all
 * instances from arrays packed instance after instance.  Any pointer may be
 * NULL to keep that parameter.
 *   x0:       nx values per instance (initial state p_x0)
 *   setpoint: distillation/toy: T values per instance (setpoint of x_{k,1}
 *             resp. y_k, k = 1..T); plate: g*g target field per instance;
 *             paper's plate: T values (the region setpoint T_sp(t_k)).
 *             With instance = -1 and unequal horizons, instance i takes its
 *             own T_i values, one instance after another (sum of T_i)
 *   u_prev:   distillation: 1 value per instance (u_0 of the Delta-u term);
 *             paper's plate: the control Q of the cold start */
nmpc_status nmpc_set_params(nmpc_handle* h, int instance, const double* x0, const double* setpoint,
                            const double* u_prev, int on_device);

/* Run Algorithm 2 on every instance until each converges (E_0 <= tol) or
 * fails.  warm_start = 0: cold start from a constant trajectory (the paper's
 * PU mode); 1: start from the previous solution with mu0_warm (WS+PU).
 * info: n_instances records (host), may be NULL.  Returns NMPC_OK when every
 * instance converged, else the first failing instance's status. */
nmpc_status nmpc_solve(nmpc_handle* h, int warm_start, nmpc_info* info);

/* Copy an instance's solution: y (n of that instance); duals (nullable)
 * receives [zL (n), zU (n), s+ (m), s- (m), w+ (m), w- (m), b+ (m), b- (m)].
 * instance = -1 copies every instance, packed one after another (n and m
 * then count all instances; y of instance i starts at the sum of the n of
 * the instances before it). */
nmpc_status nmpc_get_solution(nmpc_handle* h, int instance, double* y, double* duals, int on_device);

/* Overwrite an instance's primal-dual point (same layout as get_solution;
 * instance = -1: every instance, packed as get_solution(-1) returns them);
 * the next warm solve starts from it.  duals may be NULL to keep them. */
nmpc_status nmpc_set_start(nmpc_handle* h, int instance, const double* y, const double* duals,
                           int on_device);

/* Adjoint sensitivity at the converged point (not in the paper): for a loss
 * l(y*) with gradient dloss_dy (n of the instance), solve the transposed
 * condensed KKT system with the stored L D L^T factor (plus iterative
 * refinement) and return dl/dp_x0 (nx) and dl/dsetpoint (T values or g*g).
 * Either output may be NULL. */
nmpc_status nmpc_sensitivity(nmpc_handle* h, int instance, const double* dloss_dy,
                             double* dloss_dx0, double* dloss_dsetpoint, int on_device);

/* Time each phase of an interior-point iteration reps times at the current
 * iterate (after a solve or set_start) without changing the iterate or the
 * solver state.  Used for roofline measurements. */
nmpc_status nmpc_time_phases(nmpc_handle* h, int reps, nmpc_phase_times* out);

/* Per-iteration trace of the last solve of an instance: 8 doubles per
 * interior-point iteration [mu, alpha (accepted primal step), alpha_dual,
 * delta_w, theta, phi_mu, E_mu, line-search trials].  Copies up to cap
 * iterations to host memory; returns the number of iterations (or -1). */
int nmpc_get_trace(nmpc_handle* h, int instance, double* out, int cap);

/* Sizes and one-time analysis figures. */
nmpc_status nmpc_get_stats(const nmpc_handle* h, nmpc_stats* stats);

/* Per-instance dimensions: n, m, offset of the instance in the packed vectors. */
nmpc_status nmpc_instance_dims(const nmpc_handle* h, int instance, int* n, int* m, int* T);

/* Introspection of the one-time analysis (host only, usable before bind).
 * Copies up to cap entries of the requested array into out (int32 unless
 * noted) and returns the full length, or -1 for an unknown selector:
 *   0 perm (n_total): factor position of each variable
 *   1 supernode first column, 2 supernode column count, 3 supernode row count
 *   4 supernode row lists, concatenated
 *   5 supernode parent (-1 for roots)
 *   6 level pointer (n_levels + 1), 7 supernodes ordered by level
 *   8 condensed-matrix lower pattern as (row, col) pairs in factor order
 *     (2 int32 per entry; the returned length counts pairs)
 *   9 reduction chunks as (instance, kind 0 variables / 1 rows, begin, end)
 *     (4 int32 per chunk; the returned length counts chunks)
 *   10 the variables in the order the reductions visit them (n_total): chunk
 *      by chunk, longest column of the Jacobian first
 *   11 entries of each variable's column of the Jacobian (n_total) */
long long nmpc_structure_export(const nmpc_handle* h, int what, void* out, long long cap);

/* Size of the library's static device workspace used by nmpc_solve_static. */
#define NMPC_STATIC_WORKSPACE_BYTES (32 * 1024 * 1024)

/* One-shot cold solve that allocates nothing (no paper counterpart).
 *
 * For callers that cannot allocate device memory themselves -- for example a
 * control task that may only use memory fixed when the process starts, or a
 * plug-in that is handed a stream and its input/output buffers but no
 * allocator -- and therefore cannot supply the workspace that nmpc_bind
 * needs.  This entry point runs the same analysis and the same kernels as
 * nmpc_build + nmpc_bind + nmpc_set_params + nmpc_solve + nmpc_get_solution,
 * but every device scratch array (factor panels, multifrontal update
 * matrices, reduction partials, iterates) lives in one file-scope device
 * array of NMPC_STATIC_WORKSPACE_BYTES (32 MiB) that every GPU loading the
 * library holds until the process exits.  It makes no device or pinned-host
 * allocation: no cudaMalloc, cudaFree, cudaMallocHost or other CUDA
 * allocating routine (the host-side analysis uses ordinary heap memory).
 *
 *   prob, opts:     as for nmpc_build (opts may be NULL)
 *   cuda_stream:    stream for all work (NULL = legacy default stream)
 *   x0, setpoint, u_prev: parameters packed for all instances as in
 *                   nmpc_set_params(instance = -1); NULL keeps zeros
 *   y_out:          receives the primal solutions of all instances, packed
 *                   instance after instance (sum of n over instances)
 *   info:           n_instances records (host), may be NULL
 *   on_device:      1 if x0/setpoint/u_prev/y_out are device pointers
 * Returns NMPC_ERR_WORKSPACE (with a message on stderr) when the problem's
 * workspace exceeds NMPC_STATIC_WORKSPACE_BYTES, otherwise as nmpc_solve.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  All
 * calls share the one array and each call overwrites and clears what it
 * uses: calls that overlap on the GPU (other streams or threads) race and
 * must be serialized by the caller.  Always a cold start. */
nmpc_status nmpc_solve_static(const nmpc_problem* prob, const nmpc_options* opts, void* cuda_stream,
                              const double* x0, const double* setpoint, const double* u_prev,
                              double* y_out, nmpc_info* info, int on_device);

/* ------------------------------------------------------------------------
 * Autotuner (the batch path's tuning of the supernodal schedule; not in the
 * paper).  The symbolic analysis and the kernels' schedule depend on options
 * the problem does not fix: the ordering (nested dissection with leaves of
 * 1 or 2 stages; the two-sided stage order; stage order for short
 * horizons), the supernode amalgamation under nested dissection
 * (amalgamation 1 or 2), the factorization's schedule (factor_mode 0: one
 * launch per level, or 3: the dataflow launch) and the solve form
 * (panel_scale 1 or 3).  nmpc_autotune builds every candidate (reusing
 * those nmpc_autotune_workspace_bytes just built for the same problem),
 * binds it to the caller's workspace, runs one cold solve of the given
 * parameters and, if every instance converged, times one iteration's
 * evaluation, assembly, factorization and solves at that point (as
 * nmpc_time_phases, reported) and two steps of the closed loop of Algorithm 1
 * (every instance restarted warm from its own x_1 and u_1; the measured state
 * is the prediction, as the bench's closed loop).  It keeps the candidate
 * with the fastest re-solve -- which weighs both the full iterations and
 * those in which few instances of a batch still run -- and writes its ordering,
 * nd_leaf, amalgamation, factor_mode and panel_scale into *opts (the other
 * fields are kept).
 * Results are cached per problem (model, sizes, horizons, constants) and
 * remaining options for the life of the process: a repeated call returns
 * the cached choice without running anything.
 *   workspace, bytes: device memory of at least the size that
 *                 nmpc_autotune_workspace_bytes reports (256-byte aligned);
 *                 its contents are overwritten
 *   x0, setpoint, u_prev: packed instance after instance, as nmpc_set_params
 *                 (instance = -1) would take them, except that setpoints of
 *                 instances with different horizons follow one another (T_i
 *                 values each); NULL keeps zeros
 *   report:       may be NULL; candidates in the order tried
 * Returns NMPC_ERR_WORKSPACE if the workspace is too small for every
 * candidate, NMPC_ERR_CUDA on a CUDA error, NMPC_MAX_ITER (or the first
 * failing status) if no candidate converged, else NMPC_OK. */
#define NMPC_TUNE_MAX 16
typedef struct {
  int ordering, nd_leaf, panel_scale;
  int status;            /* of the cold solve (NMPC_ERR_WORKSPACE: skipped, too large) */
  int iters;             /* largest over instances */
  double ms_per_iter;    /* evaluation + assembly + factorization + solves at the converged point */
  int amalgamation;      /* nmpc_options.amalgamation of the candidate */
  int factor_mode;       /* nmpc_options.factor_mode of the candidate (0 per-level launches, 3 dataflow) */
  double ms_resolve;     /* mean of two warm closed-loop re-solves after the cold solve (the choice's key) */
} nmpc_tune_candidate;
typedef struct {
  int n_candidates, best, cached;
  nmpc_tune_candidate cand[NMPC_TUNE_MAX];
} nmpc_tune_report;

nmpc_status nmpc_autotune_workspace_bytes(const nmpc_problem* prob, const nmpc_options* opts, size_t* bytes);
nmpc_status nmpc_autotune(const nmpc_problem* prob, nmpc_options* opts, void* cuda_stream, void* workspace,
                          size_t bytes, const double* x0, const double* setpoint, const double* u_prev,
                          int on_device, nmpc_tune_report* report);

/* ------------------------------------------------------------------------
 * Measurement and self-test hooks (not in the paper).
 *
 * nmpc_debug_recip: out[i] = the reciprocal the factorization uses for its
 * pivots (reading of eq. cholesky-numeric in L D L^T form: one reciprocal per
 * column), computed by the same device routine, for n device values in[i]
 * (in, out: device pointers, n >= 0).  Ordered on cuda_stream; returns
 * without synchronizing.  For tests that compare it with IEEE division.
 *
 * nmpc_probe_fp64: measured FP64 throughput of this GPU in TFLOP/s, the peak
 * that the factorization's FP64 rate is compared with.  kind 0: independent
 * FMA chains on every thread; kind 1: the f64 tensor-core instruction
 * mma.sync.m8n8k4 with independent accumulators on every warp.
 * blocks_per_sm (1..8) blocks of 256 threads per SM, iters steps each; one
 * warm-up launch, then one launch timed with CUDA events on cuda_stream
 * (synchronizes it).  Allocates no device memory. */
nmpc_status nmpc_debug_recip(const double* in, double* out, long long n, void* cuda_stream);
nmpc_status nmpc_probe_fp64(int kind, int blocks_per_sm, int iters, void* cuda_stream, double* tflops);

/* Release host memory of the handle (the caller frees the workspace).
 * Synchronizes the library stream.  NULL is ignored. */
void nmpc_destroy(nmpc_handle* h);

const char* nmpc_status_string(int status);
const char* nmpc_last_error(const nmpc_handle* h);

#ifdef __cplusplus
}
#endif
#endif
