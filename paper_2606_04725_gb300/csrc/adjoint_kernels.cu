// Adjoint sensitivity at the converged point (not in the paper).
//
// With the barrier weights of the converged point held fixed, differentiating
// the condensed Newton system (eq. liftedkkt-pd) gives dy*/dp = -K^{-1} dr_c/dp,
// K = W + Sigma_y + H^T (Q+ + Q-) H.  K is symmetric, so for a loss l(y*) one
// solve v = K^{-1} dl/dy serves every parameter:
//   setpoint sp_k (tracking of x_{k,1}):   dl/dsp_k = 2 dt v_{x_k,1}
//   plate target c:                        dl/dt_c  = sum_k 2 dt h^2 v_{x_k,c}
//   initial state (rows x_0 - p_x0 = 0):   dl/dp_x0,i = D_i v_{x_0,i},
//                                          D_i = Q+_i + Q-_i of that row.
// v comes from the stored Cholesky factor (factored one step before the
// converged point, possibly regularized) and iterative refinement against
// K(z*) applied matrix-free.
#include "kernels.h"

namespace nmpc {

// t_r = D_r (H x)_r for the rows of the selected instance, and the same with
// absolute values (ta_r = D_r (|H| |x|)_r) for the backward error
__global__ void k_kmat_rows(Dev d, const double* Drow, const double* x, double* t, double* ta, int inst) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= d.m || d.row_inst[r] != inst) return;
  const int WH = d.mc.WH;
  double a = 0.0, aa = 0.0;
  for (int s = 0; s < WH; ++s) {
    const int col = d.Hcol[(size_t)r * WH + s];
    if (col >= 0) {
      const double p = d.Hv[(size_t)r * WH + s] * x[col];
      a += p;
      aa += fabs(p);
    }
  }
  t[r] = Drow[r] * a;
  ta[r] = fabs(Drow[r]) * aa;
}

// out = g - K x with K x = W x + Sigma_y x + H^T t (t from k_kmat_rows), and
// scale = (|K| |x|)_v + |g_v|, the denominator of the componentwise backward error
__global__ void k_kmat_vars_residual(Dev d, const double* x, const double* t, const double* ta, const double* g,
                                     double* out, double* scale, int inst) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.n || d.var_inst[v] != inst) return;
  const int WH = d.mc.WH;
  double kx = (d.zL[v] * d.igL[v] + d.zU[v] * d.igU[v]) * x[v];
  double ab = fabs(kx);
  for (int q = d.Wadj_ptr[v]; q < d.Wadj_ptr[v + 1]; ++q) {
    const double p = d.Wv[d.Wadj_slot[q]] * x[d.Wadj_other[q]];
    kx += p;
    ab += fabs(p);
  }
  for (int q = d.Hcsc_ptr[v]; q < d.Hcsc_ptr[v + 1]; ++q) {
    const int s = d.Hcsc_slot[q];
    kx += d.Hv[s] * t[s / WH];
    ab += fabs(d.Hv[s]) * ta[s / WH];
  }
  out[v] = g[v] - kx;
  scale[v] = ab + fabs(g[v]);
}

// scatter an instance's natural-order vector into the factor order (zero elsewhere)
__global__ void k_to_factor_order(Dev d, const double* src, int inst) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.n) return;
  d.b[d.perm[v]] = (d.var_inst[v] == inst) ? src[v] : 0.0;
}

// x (natural order) = [x +] solution held in b (factor order)
__global__ void k_from_factor_order(Dev d, double* x, int accumulate, int inst) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.n || d.var_inst[v] != inst) return;
  const double s = d.b[d.perm[v]];
  x[v] = accumulate ? x[v] + s : s;
}

// parameter gradients from v (natural order) for instance inst
__global__ void k_sens_out(Dev d, const double* v, const double* Drow, int inst, double* dx0, double* dsp) {
  const ModelConst& mc = d.mc;
  const int nx = mc.nx, nu = mc.nu;
  const int vo = d.inst_voff[inst], ro = d.inst_roff[inst], T = d.inst_T[inst];
  const double* vi = v + vo;
  auto offx = [&](int k) { return k == 0 ? 0 : nx + (k - 1) * (nx + nu); };
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  if (dx0)
    for (int i = tid; i < nx; i += nt) dx0[i] = Drow[ro + i] * vi[i];
  if (!dsp) return;
  if (mc.model == MODEL_PLATE) {
    const double hh = 1.0 / mc.g;
    for (int c = tid; c < nx; c += nt) {
      double a = 0.0;
      for (int k = 1; k <= T; ++k) a += vi[offx(k) + c];
      dsp[c] = 2.0 * mc.dt * hh * hh * a;
    }
  } else if (mc.model == MODEL_PPLATE) {
    // the setpoint of stage k enters the gradient of the region term:
    // d(grad_{T_k,c} f)/d sp_k = -2 dt w_c
    const int n = mc.g, mm = n - 2;
    const double hh = 2.0 / (n - 1);
    for (int k = 1 + tid; k <= T; k += nt) {
      double a = 0.0;
      for (int c = 0; c < nx; ++c) {
        const int ci = c % mm + 1, cj = c / mm + 1;
        const int ai = 2 * abs(2 * ci - (n - 1)), aj = 2 * abs(2 * cj - (n - 1));
        if (ai > n - 1 || aj > n - 1) continue;
        a += hh * hh * (ai == n - 1 ? 0.5 : 1.0) * (aj == n - 1 ? 0.5 : 1.0) * vi[offx(k) + c];
      }
      dsp[k - 1] = 2.0 * mc.dt * a;
    }
  } else {
    for (int k = 1 + tid; k <= T; k += nt) dsp[k - 1] = 2.0 * mc.dt * vi[offx(k)];
  }
}

__global__ void k_ctl_select(Ctl* ctl, int n, int inst, int refactor) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  ctl[i].status = (i == inst) ? ST_RUNNING : ST_CONVERGED;
  ctl[i].need_factor = (i == inst) ? refactor : 0;
  ctl[i].factor_fail = 0;
  ctl[i].dw = 0.0;
  ctl[i].ls_active = 0;
}

// out[0] = max_v |r_v| / scale_v (componentwise backward error of K x = g).
// Bit patterns of non-negative doubles order like the values, so an
// integer max is exact and independent of the order of the updates.
__global__ void k_resid_norms(Dev d, const double* r, const double* scale, int inst, unsigned long long* out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.n || d.var_inst[v] != inst) return;
  const double w = scale[v] > 0.0 ? fabs(r[v]) / scale[v] : fabs(r[v]);
  atomicMax(out, (unsigned long long)__double_as_longlong(w));
}

}  // namespace nmpc
