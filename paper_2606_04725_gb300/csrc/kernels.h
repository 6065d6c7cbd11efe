// Kernel declarations of the NMPC library (all FP64, sm_103a).
#pragma once
#include <cuda_runtime.h>

#include "nmpc_internal.h"

namespace nmpc {

// 1/d in double precision.  Seed: the PTX approximate reciprocal (relative
// error below 2^-20).  Refinement: one third-order Newton-Raphson step for
// f(y) = 1/y - d, i.e. with e = 1 - d*y the truncated series
// 1/d = y/(1 - e) = y (1 + e + e^2 + ...), y <- y + y (e + e^2), which leaves
// a relative error of order e^3 < 2^-60 plus the rounding of the last FMA.
// Near the ends of the exponent range (and for zero, subnormal, infinite or
// NaN input) the plain division is used.
__device__ __forceinline__ double recip_nr(double d) {
  const int ex = (__double2hiint(d) >> 20) & 0x7ff;
  if (ex < 3 || ex > 2044) return 1.0 / d;
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
  const double e = fma(-d, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

// The triangular solves work on an instance while it runs, except during a
// HyKKT conjugate-gradient loop once that instance's CG has ended.
__device__ __forceinline__ bool solve_on(const Ctl& c) { return c.status == ST_RUNNING && !c.solve_skip; }

constexpr int TPB = 256;  // generic element-wise and per-instance launches
constexpr int EW = 128;   // element-wise kernels: smaller blocks spread FP64 work over more SMs

// model_kernels.cu
__global__ void k_eval_rows(Dev d, int use_trial, int with_jac);
__global__ void k_eval_vars(Dev d, int use_trial);
__global__ void k_eval(Dev d, int use_trial, int with_jac, int nbr);
__global__ void k_set_params(Dev d, int i0, int i1, const double* x0, const double* sp, const double* up, int sp_len);
__global__ void k_set_params_packed(Dev d, const int* spoff, const double* x0, const double* sp, const double* up);
__global__ void k_shift_params(Dev d);
__global__ void k_init_vars(Dev d, int warm, double push);
__global__ void k_init_rows(Dev d, int warm, double push);

// ipm_kernels.cu
__global__ void k_ctl_init(Dev d, double mu0);
__global__ void k_red_eval(Dev d, int max_iter, CondArgs ca);
__global__ void k_zero_L(Dev d, const long long* inst_Lbeg, const long long* inst_Lend);
__global__ void k_rows_pre(Dev d, double* Drow);
__global__ void k_zero_rows(Dev d, const long long* inst_Lbeg, const long long* inst_Lend, double* Drow, int zx);
__global__ void k_assemble(Dev d, const int* tgt_inst, const double* Drow);
__global__ void k_ctl_factor(Dev d, CondArgs ca);
__global__ void k_rhs(Dev d);
__global__ void k_red_dir(Dev d, CondArgs ca);
__global__ void k_trial_point(Dev d);
__global__ void k_red_trial(Dev d, CondArgs ca);
__global__ void k_update(Dev d);
__global__ void k_summary(Dev d, int* flags, int cg);
__global__ void k_red_cg0(Dev d, CondArgs ca);
__global__ void k_cg_apply(Dev d);
__global__ void k_red_cg1(Dev d);
__global__ void k_red_cg2(Dev d, CondArgs ca);
__global__ void k_hy_rhs(Dev d);

// factor_kernels.cu
__global__ void k_factor_level(Dev d, SnDev s, const FrontDesc* dl, int smem_cap);
__global__ void k_factor_cluster(Dev d, SnDev s, const FrontDesc* dl);
__global__ void k_factor_flow(Dev d, SnDev s, const FrontDesc* dl, int nf, int* flags, const int* list,
                              const int* count);
__global__ void k_fwd_level(Dev d, SnDev s, const FrontDesc* dl, int smem_cap);
__global__ void k_bwd_level(Dev d, SnDev s, const FrontDesc* dl, int smem_cap);
__global__ void k_fwd_persist(Dev d, SnDev s, const FrontDesc* dl, int nf, int smem_cap, int* flags, const int* list,
                              const int* count);
__global__ void k_bwd_persist(Dev d, SnDev s, const FrontDesc* dl, int nf, int smem_cap, int* flags, const int* list,
                              const int* count);
// level-ordered list of the fronts [0, nf) of the instances that take part in
// a persistent launch (mode 0: need a factorization; 1: are being solved)
constexpr int FL_THREADS = 1024;
constexpr int FL_MAX_INST = 32768;  // one byte of shared memory per instance
constexpr int PERSIST_STAGE_CAP = 21 * 1024;  // bytes: largest panel a batch's persistent solves stage
__global__ void k_front_list(Dev d, SnDev s, int nf, int mode, int* list, int* count);
__global__ void k_diag_inv(Dev d, SnDev s, int i0);
__global__ void k_panel_scale(Dev d, SnDev s, int u0);
__global__ void k_big_zero(Dev d, SnDev s, const FrontDesc* dl);
__global__ void k_big_extend(Dev d, SnDev s, const FrontDesc* dl, int k);
__global__ void k_big_diag(Dev d, SnDev s, const FrontDesc* dl, int p);
__global__ void k_big_trsm(Dev d, SnDev s, const FrontDesc* dl, int p);
__global__ void k_big_update(Dev d, SnDev s, const FrontDesc* dl, int p);
__global__ void k_bigs_fwd_pre(Dev d, SnDev s, const FrontDesc* dl);
__global__ void k_bigs_fwd_diag(Dev d, SnDev s, const FrontDesc* dl, int jb);
__global__ void k_bigs_fwd_rows(Dev d, SnDev s, const FrontDesc* dl, int jb);
__global__ void k_bigs_fwd_post(Dev d, SnDev s, const FrontDesc* dl);
__global__ void k_bigs_bwd_pre(Dev d, SnDev s, const FrontDesc* dl);
__global__ void k_bigs_bwd_anc(Dev d, SnDev s, const FrontDesc* dl);
__global__ void k_bigs_bwd_diag(Dev d, SnDev s, const FrontDesc* dl, int jb);
__global__ void k_bigs_bwd_cols(Dev d, SnDev s, const FrontDesc* dl, int jb);
__global__ void k_bigs_bwd_post(Dev d, SnDev s, const FrontDesc* dl);
constexpr int BIG_SBW = 128, BIG_SBT = 256;  // SBW, SBT in factor_kernels.cu
constexpr int BIG_NB = 32, BIG_TILE = 64, BIG_ROWS = 256;  // BNB, BT, BROWS in factor_kernels.cu

// adjoint_kernels.cu
__global__ void k_kmat_rows(Dev d, const double* Drow, const double* x, double* t, double* ta, int inst);
__global__ void k_kmat_vars_residual(Dev d, const double* x, const double* t, const double* ta, const double* g,
                                     double* out, double* scale, int inst);
__global__ void k_to_factor_order(Dev d, const double* src, int inst);
__global__ void k_from_factor_order(Dev d, double* x, int accumulate, int inst);
__global__ void k_sens_out(Dev d, const double* v, const double* Drow, int inst, double* dx0, double* dsp);
__global__ void k_ctl_select(Ctl* ctl, int n, int inst, int refactor);
__global__ void k_resid_norms(Dev d, const double* r, const double* scale, int inst, unsigned long long* out);

inline unsigned blocks_for(long long n, int tpb = TPB) { return (unsigned)((n + tpb - 1) / tpb); }

}  // namespace nmpc
