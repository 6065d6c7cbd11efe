/* Oracle for the parametric interior-point NMPC hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, FP64 CPU implementation
 * written from the paper (arXiv 2606.04725, Sec. 3.2 and Algorithm 2) and the
 * interior-point method it cites (Wachter & Biegler 2006).  Only the tests,
 * __graft_entry__.smoke() and bench.py's CPU-baseline leg may load it.  It
 * shares no code with the CUDA library: no headers, helpers or tables.
 *
 * Parity status of each part (pins live in tests/test_oracle_*.py):
 *   model residuals/derivatives  pinned (complex step, conservation laws,
 *                                steady state of Sec. 4.1, stencil exactness)
 *   banded Cholesky              pinned (numpy.linalg.cholesky, Laplacian)
 *   sparse Cholesky, ND order    pinned (fill against numpy.linalg.cholesky of
 *                                the permuted matrix, solves, the failing pivot
 *                                against Schur-complement pivots, fill on grids
 *                                below the natural order's, Newton step and
 *                                IPM solutions equal to the band path's)
 *   SymCholesky                  pinned (Fig. cholesky-symExample, brute force)
 *   Newton step / condensation   pinned (uncondensed primal-dual Newton system)
 *   optimality error E_mu, E_0   pinned (lifted KKT residual from the dense
 *                                Jacobian, scaled and unscaled)
 *   line search, step update     pinned (step by step against the Newton
 *                                direction, merits recomputed from the model,
 *                                fraction to the boundary, filter tests)
 *   barrier update               pinned (the mu chain and its E_mu tests, per
 *                                iteration)
 *   inertia correction           pinned (delta_w sequence of W&B Algorithm IC,
 *                                definiteness by dense eigenvalues where they
 *                                can decide it)
 *   converged solutions          pinned (dense KKT solve of LQ cases,
 *                                brute-force active sets, FD stationarity)
 *   HyKKT Newton step            pinned (dense primal-dual Newton system of the
 *                                unlifted barrier problem; independent of the
 *                                augmentation weight)
 *   HyKKT converged solutions    pinned (equality QP incl. its multipliers,
 *                                brute-force active sets, FD stationarity)
 *   iteration counts             parity unpinned (no external count exists)
 */
#ifndef NMPC_ORACLE_H
#define NMPC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_DISTILL = 0, OR_PLATE = 1, OR_TOY = 2, OR_PPLATE = 3, OR_DDAE = 4 };

typedef struct {
  int model;
  int nx, nu, T;      /* states per stage, controls per stage, intervals */
  int n, m;           /* filled by or_setup */
  int N, Nf;          /* distillation: trays (condenser = 1, reboiler = N), feed tray */
  int g, S;           /* plate: grid side, actuator segments */
  double dt;
  double alpha, D, F, xF, Ac, At, Ar, wdu; /* distillation constants */
  double wu, ubar;    /* distillation: weight of the control-tracking cost (u - ubar)^2 per unit time */
  double kappa, cq, rho_u;                 /* plate constants */
  double xlo, xhi, ulo, uhi;               /* bounds on x_1..x_T, u_1..u_T (+-inf allowed) */
  const double* x0;   /* nx: initial state parameter */
  const double* sp;   /* distillation/toy: T setpoints; plate: g*g target field */
  double uprev;       /* distillation: u_0; paper's plate: the control of the cold start */
  double Tb, qloss;   /* paper's plate (Sec. 4.2): fixed boundary temperature, heat loss */
  int nr;             /* filled by or_setup: rows per backward-Euler step (nx except for OR_DDAE) */
} or_problem;

typedef struct {
  double tol;        /* outer tolerance on the scaled E_0 */
  double gamma;      /* Lifted-KKT relaxation of the equalities */
  double mu0_cold, mu0_warm;
  double push_cold, push_warm;
  int max_iter;
  double pivtol;     /* relative pivot tolerance of the inertia test */
  double dw_max;     /* largest regularization delta_w of the inertia correction (W&B Algorithm IC: 1e40) */
  int kkt;           /* Newton system: 0 Lifted-KKT (eq. liftedkkt-pd), 1 HyKKT (Sec. 3.2.2's alternative) */
  double hy_gamma;   /* HyKKT: augmented-Lagrangian weight of H^T H */
  double cg_tol;     /* HyKKT: CG stops when ||r||^2 <= cg_tol^2 ||r_0||^2 */
  int cg_max_iter;   /* HyKKT: CG iterations per Newton step at most */
  int linsolve;      /* factorization of K: 0 band Cholesky in stage order, 1 sparse Cholesky
                        after the oracle's nested-dissection ordering (or_sparse.inc) */
} or_options;

typedef struct {
  int status;        /* 0 converged, 10 max iter, 11 line search, 12 inertia, 13 non-finite */
  int iters;
  int inertia_retries;
  int ls_trials;
  double mu_final, E0_scaled, E0_unscaled, objective, delta_w_last;
  int cg_iters;      /* HyKKT: CG iterations over the whole solve */
} or_info;

/* Primal-dual state.  All arrays are caller-owned.
 *   y, zL, zU: n     s_p, s_m, w_p, w_m, b_p, b_m: m
 * (s = slacks, w = omega multipliers, b = beta slack-bound multipliers, for the
 * lifted rows  h - gamma + s_p = 0  and  -h - gamma + s_m = 0).
 * With kkt = 1 (HyKKT) the equalities h = 0 stay and w_p holds their
 * multipliers lambda; s_p, s_m, w_m, b_p and b_m are not used. */
typedef struct {
  double *y, *zL, *zU;
  double *s_p, *s_m, *w_p, *w_m, *b_p, *b_m;
} or_state;

int or_setup(or_problem* p);
int or_jac_nnz(const or_problem* p);
void or_bounds(const or_problem* p, double* yL, double* yU);
void or_eval(const or_problem* p, const double* y, double* f, double* grad, double* h,
             int* rowptr, int* colidx, double* Hvals);
void or_eval_complex(const or_problem* p, const double* y_re, const double* y_im,
                     double* f_re_im, double* grad_re_im, double* h_re_im, double* Hvals_re_im);
int or_hessian(const or_problem* p, const double* y, const double* lam,
               int* rows, int* cols, double* vals, int cap);
int or_steady_state(const or_problem* p, double u, double* x);
int or_solve(const or_problem* p, const or_options* o, or_state* z, int warm,
             or_info* info, double* trace, int trace_cap);
void or_kkt_error(const or_problem* p, const or_options* o, const or_state* z, double mu,
                  double* E_scaled, double* E_unscaled);
int or_newton_step(const or_problem* p, const or_options* o, const or_state* z, double mu,
                   double delta_w, or_state* d);
int or_band_cholesky(int n, int b, double* band);
int or_symbolic(int n, const int* colptr, const int* rowidx, int* parent,
                int* Lcolptr, int* Lrowidx, int cap);
int or_nd_order(int n, const int* xadj, const int* adj, int leaf, int* perm);
int or_sparse_cholesky(int n, const int* colptr, const int* rowidx, const double* vals,
                       int use_nd, double tol, int* perm, double* b, long* nnzL);

#ifdef __cplusplus
}
#endif
#endif
