// Internal layout shared by the host structure builder and the CUDA kernels.
//
// Slot conventions (the builder and the kernels must agree):
//   H (Jacobian of the equality rows) is stored ELL-style, WH slots per row:
//     distillation (WH=5): [x_k,i | x_{k+1},i-1 | x_{k+1},i | x_{k+1},i+1 | u_{k+1}]
//     plate        (WH=8): [x_k,c | x_{k+1},c-g | c-1 | c | c+1 | c+g | v_a | v_b]
//     toy          (WH=3): [y_k | y_{k+1} | u_{k+1}]
//     paper plate  (WH=7): [T_k,c | T_{k+1},c-m | c-1 | c | c+1 | c+m | Q_{k+1}] (m = g - 2
//                          interior nodes per row; the Q slot only next to x1 = -1 or x2 = -1)
//     DAE column   (WH=8): balance of tray i [x_k,i | x_{k+1},i-1 | x_{k+1},i | y_{k+1},i |
//                          y_{k+1},i+1 | L | V | S]; equilibrium i [x_{k+1},i | y_{k+1},i];
//                          L - uD [u | L]; V - L - D [L | V]; S - L - F [L | S]
//   Rows per step: nr = nx, except the DAE column (2N + 3: N balances, N equilibria,
//   3 flow equations); the rows of step k start at nx + nr k.
//   Initial-condition rows use slot 0 only (coefficient 1).  Unused slots
//   carry column -1 and value 0.
//   W (Hessian of the Lagrangian, lower triangle) is stored per stage
//   k = 1..T, WS slots per stage:
//     distillation (WS=2N+2): [x_k,i diag (N) | (u_k, x_k,i) (N) | u_k diag | (u_k, u_{k-1})]
//     plate        (WS=g*g+S): [x_k,c diag | v_k,s diag]
//     toy          (WS=2): [y_k diag | u_k diag]
//     paper plate  (WS=(g-2)^2+1): [T_k,c diag | Q_k diag]
//     DAE column   (WS=3N+1): [x_j diag (N) | (L or S, x_j), j < N (N-1: L above the feed,
//                  S from it down) | (V, x_1) | (V, y_j), j >= 2 (N-1) | u diag | (u_k, u_{k-1})]
#pragma once
#include <cstdint>

namespace nmpc {

enum Model { MODEL_DISTILL = 0, MODEL_PLATE = 1, MODEL_TOY = 2, MODEL_PPLATE = 3, MODEL_DDAE = 4 };

// Per-instance control state of the interior-point method (device resident).
// One record per instance; the control kernels run one thread per instance.
struct Ctl {
  double mu, tau, dw, dw_last;
  double theta_max, theta_min;
  double f, logsum, theta, phi;       // at the current iterate
  double gphi;                        // directional derivative of phi_mu
  double alpha, alpha_min, alpha_pri, alpha_dual;
  double E0, E0u, Emu;
  double ft, logsum_t, theta_t;       // at the trial point
  double sw_gphi, sw_theta;           // (-gphi)^s_phi and delta theta^s_theta of this iteration
  int status;                         // 0 running, else nmpc_status (1 = converged)
  int iter;
  int phase;                          // see PH_* below
  int need_factor;                    // 1 while this instance still needs a factorization
  int factor_fail;                    // set by the factor kernels
  int ls_active;                      // 1 while the line search is running
  int nf;                             // filter entries
  int inertia_retries, ls_trials, augment;
  int first;                          // first iteration of a solve
  int ls_trials0;                     // ls_trials at the start of this iteration's search
  // HyKKT form: conjugate gradients on S dlam = t (S = H K^-1 H^T) of this iteration
  double cg_rr, cg_stop, cg_alpha, cg_beta;  // r^T r, cg_tol^2 r_0^T r_0, step, p-update weight
  int cg_active;                      // 1 while this instance's CG runs
  int cg_it, cg_total;                // CG iterations of this Newton step / of the solve
  int solve_skip;                     // 1: the triangular solves skip this instance (CG done)
};

constexpr int FILTER_CAP = 256;
constexpr int ST_RUNNING = 0;
constexpr int ST_CONVERGED = 1;  // mapped to NMPC_OK at the API

// Constants of the interior-point method (Wachter & Biegler 2006 defaults).
constexpr double KAPPA_EPS = 10.0, KAPPA_MU = 0.2, THETA_MU = 1.5, TAU_MIN = 0.99, S_MAX = 100.0;
constexpr double KAPPA_SIGMA = 1e10, GAMMA_THETA = 1e-5, GAMMA_PHI = 1e-5, DELTA_SW = 1.0;
constexpr double S_THETA = 1.1, S_PHI = 2.3, ETA_PHI = 1e-4, GAMMA_ALPHA = 0.05;
constexpr double DELTA_W0 = 1e-4, DELTA_WMIN = 1e-20;
constexpr double KAPPA_W_MINUS = 1.0 / 3.0, KAPPA_W_PLUS = 8.0, KAPPA_W_PLUS_BAR = 100.0;

struct ModelConst {
  int model, nx, nu, N, Nf, g, S, WH, WS;
  int nr;                             // rows per backward-Euler step: nx, or 2N + 3 for the DAE column
  double dt, alpha, D, F, xF, Ac, At, Ar, wdu, kappa, cq, rho_u;
  double xlo, xhi, ulo, uhi;
  double wu, ubar;                    // control-tracking cost wu dt (u - ubar)^2 (distillation)
  double inv_Ac, inv_At, inv_Ar;      // 1/holdups (distillation), computed once on the host
  double gamma, tol, pivtol;
  double dw_max;                      // largest delta_w of the inertia correction
  double Tb, qloss;                   // paper's plate: boundary temperature, heat loss
  int kkt;                            // 0 Lifted-KKT, 1 HyKKT
  int cg_max_iter;                    // HyKKT: CG iterations per Newton step at most
  double hy_gamma, cg_tol;            // HyKKT: augmentation weight, CG relative tolerance
};

// Reduction chunks never straddle an instance.  kind 0: variables, 1: rows.
// One chunk is reduced by one block of RED_CHUNK threads (one element per
// thread): small chunks spread the FP64 work of a reduction over many SMs.
constexpr int RED_CHUNK = 128;
// Blocks a reduction should give at least, when the problem allows (152 SMs x 8).
constexpr int RED_TARGET_BLOCKS = 1216;
struct Chunk {
  int inst, kind, begin, end;
};

// Partial sums/extrema of one chunk (deterministic two-pass reductions).
// Sums of logarithms are carried as a product of mantissas in [1, 2) and a
// sum of binary exponents (one log per chunk instead of one per element).
struct RedEval {       // at the current iterate
  double dual, prim, cmax, cmin, sum_l, sum_z, f, lgm, lge, theta;
  double nonfinite;     // count of non-finite residual/gradient entries
};
struct RedDir {        // after the Newton direction
  double ap, ad, gphi;
  double pad;
};
struct RedTrial {      // at a trial point
  double f, lgm, lge, theta, nonfinite;
};

// Device view of everything the kernels touch.  Passed by value.
struct Dev {
  ModelConst mc;
  int n_inst, n, m, nW;
  // per instance
  const int* inst_T; const int* inst_voff; const int* inst_roff; const int* inst_woff;
  const int* inst_n; const int* inst_m; const int* inst_nz;
  // per variable / row
  const int* var_inst; const int* row_inst;
  const double* yL; const double* yU;
  // parameters
  double* p_x0; double* p_sp; double* p_uprev;
  int sp_stride;        // setpoint values per instance
  // iterate.  In the HyKKT form wp holds the equality multipliers lambda and
  // wm stays 0 (so wp - wm is the rows' multiplier in either form); sp, sm, bp
  // and bm are not used.
  double *y, *zL, *zU, *sp, *sm, *wp, *wm, *bp, *bm;
  // evaluation
  double *grad, *h, *Hv, *Wv, *fvar;
  // reciprocals at the current iterate: bound gaps, bound duals (n); slacks, slack duals (m)
  double *igL, *igU, *izL, *izU, *isp, *ism, *ibp, *ibm;
  const int* Hcol;
  const int* Hpos;      // per H slot: factor position of its column (perm[Hcol]), -1 for an empty slot
  const int* Hcsc_ptr; const int* Hcsc_slot;
  const int* Wadj_ptr; const int* Wadj_slot; const int* Wadj_other;
  // direction (HyKKT: dwp is lambda's step, the CG iterate)
  double *dy, *dzL, *dzU, *dsp, *dsm, *dwp, *dwm, *dbp, *dbm;
  // HyKKT CG residual, search direction and S p (m each; the storage of dsp,
  // dsm and dbp, which that form does not use)
  double *cg_r, *cg_p, *cg_q;
  double* red_cg;       // per reduction chunk: partial sum of a CG dot product
  double* rowv;         // per-row scratch (H^T v products)
  double* lam;          // per row: w+ - w- at the current iterate (set with the Jacobian)
  double* HD;           // per H slot: H_rs D_r, set with the rows' weights D_r before each assembly
  // trial
  double *yt, *spt, *smt, *ht, *fvart;
  // permutation / solve
  const int* perm;      // perm[i] = position of variable i in the factor ordering
  const int* iperm;
  double* b;            // permuted right-hand side / solution
  // control
  Ctl* ctl;
  double* filt_th; double* filt_ph;
  // reductions
  const Chunk* chunks; int n_chunks;
  const int* inst_chunk_ptr; const int* inst_chunk_list;
  const int* red_var;   // variables chunk by chunk, longest H column first (a permutation)
  RedEval* red_eval; RedDir* red_dir; RedTrial* red_trial;
  // assembly map
  int n_tgt;
  const long long* tgt_L;
  const int* tgt_diag;
  const int* tw_ptr; const int* tw_idx;
  const int* th_ptr; const int* th_a; const int* th_b;
  double* Lval;
  double* Kdiag;        // assembled diagonal of K_c in factor order (pivot tolerance)
  long long nnzL;
  // instance of each supernode (factor kernels)
  const int* sn_inst;
  int max_iter;
  double* trace;        // per instance: (max_iter + 2) x 8 doubles
  int* red_cnt;         // n_inst + 1 arrival counters of the fused reduction kernels (zero between launches)
};

// Conditions of the graph-driven loop, set by the kernels that end each step
// (handles are cudaGraphConditionalHandle values; on = 0 in the host-driven
// loop, which reads the control state itself).  counters: [0] outer steps,
// [1] factorization attempts, [2] line-search trials; cap_*: trip limits.
struct CondArgs {
  unsigned long long h_run, h_if, h_fac, h_ls, h_cg;
  int* counters;        // [3]: CG iterations (HyKKT)
  int cap_iter, cap_inner, cap_cg, on;
};

// One record per supernode, stored in level order, with everything a factor
// or solve block needs about its front and (up to DESC_CH of) its children:
// a block reads it with one round of independent loads instead of a chain
// of dependent index lookups.
constexpr int DESC_CH = 4;
struct alignas(8) IdxPair {
  int src, dst;
};
struct FrontDesc {
  long long Lptr, Uptr, uvptr, rowptr;
  long long abase;                                      // extend-add ranges of the cluster kernel (-1: none)
  long long Wptr;                                       // unscaled-panel scratch of the cluster kernel
  int J, m, c, first, inst, nchild;
  int pos, par_pos;                                     // own and parent's level-order position (-1: root)
  int ch_pos[DESC_CH];                                  // children's level-order positions
  int ch_mc[DESC_CH];                                   // m - c of each child
  long long ch_relptr[DESC_CH], ch_Uptr[DESC_CH], ch_uvptr[DESC_CH];
};

// The triangular solves of the fronts solved one block per front work on a
// transformed panel, written over the factor after each factorization (the
// pivots 1/d_j on the diagonal are kept).  For each block K of IB columns
// (s0 .. e-1, e = s0 + bk):
//   diagonal block: X_K = T_K^{-1} below its diagonal, T_K the unit lower
//                   triangular diagonal block of L;
//   rows e .. m-1:  M_K = L_{e..m-1,K} X_K.
// One InvItem per block with at least two columns: offset of its first entry
// (s0, s0) in L, leading dimension (m of the front), order bk <= IB,
// instance and the number m - e of rows below it.  One ScaleUnit per 32 of
// those rows when the rows are scaled (SnDev::solve_form 2; with form 1 they
// keep L and the solves take two products per block; form 0 transforms
// nothing).
constexpr int IB = 16;
struct alignas(8) InvItem {
  long long off;
  int ld, bk, inst, rows;
};
struct alignas(8) ScaleUnit {
  int item, r0;
};

// Supernodal structure for the factor and solve kernels.
struct SnDev {
  int ns;
  const int* sn_first;        // first (permuted) column
  const int* sn_ncol;         // c_s
  const int* sn_nrow;         // m_s (including the c_s pivot rows)
  const long long* sn_Lptr;   // offset of the m_s x c_s column-major panel
  const long long* sn_Uptr;   // offset of the (m_s-c_s)^2 update matrix
  const long long* sn_rowptr; // offset into sn_rows
  const int* sn_rows;         // sorted row indices of each supernode
  const int* sn_child_ptr; const int* sn_child; // children (CSR, ascending)
  const long long* sn_relptr; const int* sn_rel; // update-row positions in the parent
  const int* sn_inst;
  const int* level_ptr; const int* level_sn;    // supernodes by level (height)
  const FrontDesc* desc;      // descriptors in level_sn order
  const int* pos_of_sn;       // level-order position of each supernode
  const int* front_inst;      // instance of each front, level order
  const IdxPair* amap;        // extend-add pairs (source in child U, destination in own columns)
  const long long* amap_ptr;  // per (front, CTA, child) ranges, from FrontDesc::abase
  const long long* sn_uvptr;  // offset of the (m_s-c_s) update vector (solves)
  double* L;
  double* W;                  // unscaled factor panels W = L D of the cluster-factored fronts
  double* dpiv;               // pivots d_j of the large-front path, factor order
  double* U;
  double* uv;                 // update vectors of the forward solve
  double* fvec;               // front vectors of large-front solves (offset: the front's row list)
  const InvItem* inv;         // diagonal blocks transformed after each factorization
  const ScaleUnit* scale;     // 32-row slices of the rows below them
  int n_inv, n_scale;
  int solve_form;             // solves of small fronts: 0 column substitution on L (no transform);
                              // 1 X_K on the diagonal blocks; 2 X_K and M_K (one product per block)
  const double* Kdiag;        // assembled diagonal in factor order
  double pivtol;
  long long spin_limit;       // polls of a bounded wait between CTAs
  int* timeout;               // set to 1 when a bounded wait ran out
};

}  // namespace nmpc
