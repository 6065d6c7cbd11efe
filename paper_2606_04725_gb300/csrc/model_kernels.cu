// Stage-parallel model evaluation (hand-derived residuals, Jacobians and
// Hessians of the Lagrangian) and the parameter-update kernel.
//
// One thread per equality row computes h_r and the WH Jacobian slots of the
// row; one thread per primal variable computes the objective gradient, its
// share of the objective and the Hessian slots it owns (Sec. 3.2.2: W, H and
// the residuals of eq. infiniteOCP-augmentedRHS).  Rows and variables are laid
// out stage after stage, so neighbouring threads read neighbouring stages.
#include "kernels.h"

namespace nmpc {

struct Loc {  // position of an element inside its instance
  int inst, T, vo, ro;
};

__device__ __forceinline__ int offx(const ModelConst& mc, int k) { return k == 0 ? 0 : mc.nx + (k - 1) * (mc.nx + mc.nu); }
__device__ __forceinline__ int offu(const ModelConst& mc, int k) { return offx(mc, k) + mc.nx; }

// ------------------------------------------------------------ distillation

// Equilibrium y = a x / (1 + (a-1) x) and its first two derivatives
// a / d^2 and -2 a (a-1) / d^3 (d = 1 + (a-1) x), all from one reciprocal
// of d: every FP64 division costs tens of instructions on this GPU.
struct Vle { double y, d1, d2; };
__device__ __forceinline__ Vle vle_all(double a, double x) {
  const double r = recip_nr(fma(a - 1.0, x, 1.0));
  const double ar = a * r;
  return {ar * x, ar * r, -2.0 * (a - 1.0) * ar * r * r};
}

// Tray i (1-based) balance f_i(x, u) with L = uD, V = L + D, S = L + F, and its
// partial derivatives w.r.t. x_{i-1}, x_i, x_{i+1}, u (eq. distill-ocp).
struct TrayEval { double f, dm, d0, dp, du; };

__device__ TrayEval tray_eval(const ModelConst& mc, const double* x, double u, int i) {
  const int N = mc.N, Nf = mc.Nf;
  const double a = mc.alpha, D = mc.D;
  const double L = u * D, V = L + D, S = L + mc.F;
  TrayEval e{0, 0, 0, 0, 0};
  const double xi = x[i - 1];
  if (i == 1) {  // total condenser
    const Vle v2 = vle_all(a, x[1]);
    const double ic = mc.inv_Ac;
    e.f = V * (v2.y - xi) * ic;
    e.d0 = -V * ic;
    e.dp = V * v2.d1 * ic;
    e.du = D * (v2.y - xi) * ic;
    return e;
  }
  if (i == N) {  // reboiler
    const double xm = x[N - 2];
    const Vle vN = vle_all(a, xi);
    const double ir = mc.inv_Ar;
    e.f = (S * xm - (mc.F - D) * xi - V * vN.y) * ir;
    e.dm = S * ir;
    e.d0 = (-(mc.F - D) - V * vN.d1) * ir;
    e.du = D * (xm - vN.y) * ir;
    return e;
  }
  const double xm = x[i - 2], xp = x[i];
  const Vle vi = vle_all(a, xi), vp = vle_all(a, xp);
  const double yi = vi.y, yp = vp.y, it = mc.inv_At;
  // liquid entering from above: L above the feed tray, L onto the feed tray,
  // S below it; liquid leaving: L above the feed, S from the feed tray down
  const double lin = (i <= Nf) ? L : S;
  const double lout = (i < Nf) ? L : S;
  const double feed = (i == Nf) ? mc.F * mc.xF : 0.0;
  e.f = (feed + lin * xm - lout * xi - V * (yi - yp)) * it;
  e.dm = lin * it;
  e.d0 = (-lout - V * vi.d1) * it;
  e.dp = V * vp.d1 * it;
  e.du = D * (xm - xi - (yi - yp)) * it;
  return e;
}

// ------------------------------------------------------------------ plate

__device__ __forceinline__ int plate_seg_of(const ModelConst& mc, int ci, int cj, int* segs) {
  const int per = mc.S / 4, run = mc.g / per;
  int k = 0;
  if (cj == 0) segs[k++] = ci / run;
  if (ci == mc.g - 1) segs[k++] = per + cj / run;
  if (cj == mc.g - 1) segs[k++] = 2 * per + ci / run;
  if (ci == 0) segs[k++] = 3 * per + cj / run;
  if (k == 2 && segs[1] < segs[0]) { int t = segs[0]; segs[0] = segs[1]; segs[1] = t; }
  return k;
}

// ------------------------------------------------------- the paper's plate
// Sec. 4.2, eq. (pde-ocp): n x n nodes on [-1, 1]^2 (n = mc.g, h = 2/(n-1)),
// interior node q = cj m + ci (m = n - 2) at x1 = -1 + (ci + 1) h,
// x2 = -1 + (cj + 1) h.  Boundary data: 4.1 Q^(1/3) at x1 = -1, Q^(1/2) at
// x2 = -1, T_b at x1 = 1 and x2 = 1; dT/dt = alpha (Laplacian - 5 q_loss^2).

// The step rows x_{k+1} - x_k - dt f are divided by their diagonal coefficient
// 1 + 4 dt alpha / h^2 (7361 at n = 21), so that every row has a unit
// diagonal as the other models' rows do.
__device__ __forceinline__ double pplate_row_scale(const ModelConst& mc) {
  const double hh = 2.0 / (mc.g - 1);
  return 1.0 / (1.0 + 4.0 * mc.dt * mc.kappa / (hh * hh));
}

// Trapezoidal weight of node q in the tracking integral over [-0.5, 0.5]^2
// (h^2 inside, halved on each edge of the region, 0 outside).
__device__ __forceinline__ double pplate_weight(const ModelConst& mc, int q) {
  const int n = mc.g, mm = n - 2;
  const int i = q % mm + 1, j = q / mm + 1;
  const int ai = 2 * abs(2 * i - (n - 1)), aj = 2 * abs(2 * j - (n - 1));
  if (ai > n - 1 || aj > n - 1) return 0.0;
  const double hh = 2.0 / (n - 1);
  return hh * hh * (ai == n - 1 ? 0.5 : 1.0) * (aj == n - 1 ? 0.5 : 1.0);
}

// ------------------------------------------------------------------ rows

// h and H for every row (at iterate y, or at the trial point when only the
// residual is wanted: Hv == nullptr).
__device__ void eval_row(const Dev& d, const double* y, int r, double* hout, double* Hv) {
  const ModelConst& mc = d.mc;
  const int i = d.row_inst[r];
  const int vo = d.inst_voff[i], ro = d.inst_roff[i];
  const int lr = r - ro;
  const int nx = mc.nx;
  const int WH = mc.WH;
  const double* yi = y + vo;
  if (lr < nx) {  // initial condition x_0 - p_x0
    hout[r] = yi[lr] - d.p_x0[(size_t)i * nx + lr];
    if (Hv) {
      Hv[(size_t)r * WH] = 1.0;
      for (int s = 1; s < WH; ++s) Hv[(size_t)r * WH + s] = 0.0;
    }
    return;
  }
  const int k = (lr - nx) / mc.nr, q = (lr - nx) % mc.nr;  // row q of step k -> k+1
  const double* xk = yi + offx(mc, k);
  const double* xn = yi + offx(mc, k + 1);
  const double* un = yi + offu(mc, k + 1);
  const double dt = mc.dt;
  if (mc.model == MODEL_DDAE) {
    double* H = Hv ? Hv + (size_t)r * WH : nullptr;
    const int N = mc.N, Nf = mc.Nf;
    const double* yn = un;  // y_{k+1}
    const double L = un[N + 1], V = un[N + 2], S = un[N + 3];
    if (q < N) {  // balance of tray i
      const int i = q + 1;
      double f, d1 = 0, d2, d3 = 0, d4 = 0, dL = 0, dV, dS = 0;  // d/d x_{i-1}, x_i, y_i, y_{i+1}, L, V, S
      if (i == 1) {
        const double ic = mc.inv_Ac;
        f = V * (yn[1] - xn[0]) * ic;
        d2 = -V * ic; d4 = V * ic; dV = (yn[1] - xn[0]) * ic;
      } else if (i == N) {
        const double ir = mc.inv_Ar;
        f = (S * xn[N - 2] - (mc.F - mc.D) * xn[N - 1] - V * yn[N - 1]) * ir;
        d1 = S * ir; d2 = -(mc.F - mc.D) * ir; d3 = -V * ir; dV = -yn[N - 1] * ir; dS = xn[N - 2] * ir;
      } else {
        const double it = mc.inv_At;
        const double lin = (i <= Nf) ? L : S, lout = (i < Nf) ? L : S;
        const double feed = (i == Nf) ? mc.F * mc.xF : 0.0;
        f = (feed + lin * xn[i - 2] - lout * xn[i - 1] - V * (yn[i - 1] - yn[i])) * it;
        d1 = lin * it; d2 = -lout * it; d3 = -V * it; d4 = V * it; dV = -(yn[i - 1] - yn[i]) * it;
        if (i < Nf) dL = (xn[i - 2] - xn[i - 1]) * it;
        else if (i == Nf) { dL = xn[i - 2] * it; dS = -xn[i - 1] * it; }
        else dS = (xn[i - 2] - xn[i - 1]) * it;
      }
      hout[r] = xn[q] - xk[q] - dt * f;
      if (H) {
        H[0] = -1.0; H[1] = -dt * d1; H[2] = 1.0 - dt * d2; H[3] = -dt * d3; H[4] = -dt * d4;
        H[5] = -dt * dL; H[6] = -dt * dV; H[7] = -dt * dS;
      }
    } else if (q < 2 * N) {  // equilibrium y_i - a x_i / (1 + (a - 1) x_i)
      const int i = q - N;
      const Vle v = vle_all(mc.alpha, xn[i]);
      hout[r] = yn[i] - v.y;
      if (H) {
        H[0] = -v.d1; H[1] = 1.0;
        for (int t = 2; t < WH; ++t) H[t] = 0.0;
      }
    } else {  // flows: L - u D, V - L - D, S - L - F
      const int e = q - 2 * N;
      hout[r] = (e == 0) ? L - un[N] * mc.D : (e == 1) ? V - L - mc.D : S - L - mc.F;
      if (H) {
        H[0] = (e == 0) ? -mc.D : -1.0; H[1] = 1.0;
        for (int t = 2; t < WH; ++t) H[t] = 0.0;
      }
    }
  } else if (mc.model == MODEL_DISTILL) {
    TrayEval e = tray_eval(mc, xn, un[0], q + 1);
    hout[r] = xn[q] - xk[q] - dt * e.f;
    if (Hv) {
      double* H = Hv + (size_t)r * WH;
      H[0] = -1.0;
      H[1] = -dt * e.dm;
      H[2] = 1.0 - dt * e.d0;
      H[3] = -dt * e.dp;
      H[4] = -dt * e.du;
    }
  } else if (mc.model == MODEL_PLATE) {
    const int g = mc.g, ci = q % g, cj = q / g;
    const double hh = 1.0 / g, c = mc.kappa / (hh * hh);
    double lap = 0.0;
    int nb = 0;
    if (cj > 0) { lap += xn[q - g]; ++nb; }
    if (ci > 0) { lap += xn[q - 1]; ++nb; }
    if (ci < g - 1) { lap += xn[q + 1]; ++nb; }
    if (cj < g - 1) { lap += xn[q + g]; ++nb; }
    lap -= nb * xn[q];
    int segs[2];
    const int nsg = plate_seg_of(mc, ci, cj, segs);
    double flux = 0.0;
    for (int t = 0; t < nsg; ++t) flux += un[segs[t]];
    hout[r] = xn[q] - xk[q] - dt * (c * lap + mc.cq / hh * flux);
    if (Hv) {
      double* H = Hv + (size_t)r * WH;
      H[0] = -1.0;
      H[1] = (cj > 0) ? -dt * c : 0.0;
      H[2] = (ci > 0) ? -dt * c : 0.0;
      H[3] = 1.0 + dt * c * nb;
      H[4] = (ci < g - 1) ? -dt * c : 0.0;
      H[5] = (cj < g - 1) ? -dt * c : 0.0;
      H[6] = (nsg > 0) ? -dt * mc.cq / hh : 0.0;
      H[7] = (nsg > 1) ? -dt * mc.cq / hh : 0.0;
    }
  } else if (mc.model == MODEL_PPLATE) {
    const int mm = mc.g - 2, ci = q % mm, cj = q / mm;
    const double hh = 2.0 / (mc.g - 1), c = mc.kappa / (hh * hh);
    const double Q = un[0];
    double sum = -4.0 * xn[q], dq = 0.0;
    if (ci > 0) sum += xn[q - 1];
    else {
      const double cb = cbrt(Q);
      sum += 4.1 * cb;
      dq += 4.1 / 3.0 / (cb * cb);  // d/dQ 4.1 Q^(1/3)
    }
    sum += (ci < mm - 1) ? xn[q + 1] : mc.Tb;
    if (cj > 0) sum += xn[q - mm];
    else {
      const double sq = sqrt(Q);
      sum += sq;
      dq += 0.5 / sq;  // d/dQ Q^(1/2)
    }
    sum += (cj < mm - 1) ? xn[q + mm] : mc.Tb;
    const double s = pplate_row_scale(mc);
    hout[r] = (xn[q] - xk[q] - dt * mc.kappa * (sum / (hh * hh) - 5.0 * mc.qloss * mc.qloss)) * s;
    if (Hv) {
      double* H = Hv + (size_t)r * WH;
      H[0] = -1.0 * s;
      H[1] = (cj > 0) ? -dt * c * s : 0.0;
      H[2] = (ci > 0) ? -dt * c * s : 0.0;
      H[3] = (1.0 + 4.0 * dt * c) * s;
      H[4] = (ci < mm - 1) ? -dt * c * s : 0.0;
      H[5] = (cj < mm - 1) ? -dt * c * s : 0.0;
      H[6] = -dt * c * dq * s;  // 0 away from the controlled sides
    }
  } else {
    const double yn = xn[0], u = un[0];
    hout[r] = yn - xk[0] - dt * (4.0 * sin(u) - yn * yn * yn);
    if (Hv) {
      double* H = Hv + (size_t)r * WH;
      H[0] = -1.0;
      H[1] = 1.0 + 3.0 * dt * yn * yn;
      H[2] = -4.0 * dt * cos(u);
    }
  }
}

__device__ void eval_row_at(const Dev& d, int r, int use_trial, int with_jac) {
  const Ctl& c = d.ctl[d.row_inst[r]];
  if (use_trial) {
    if (!c.ls_active) return;
    eval_row(d, d.yt, r, d.ht, nullptr);
  } else {
    if (c.status != ST_RUNNING) return;
    eval_row(d, d.y, r, d.h, with_jac ? d.Hv : nullptr);
    if (with_jac) d.lam[r] = d.wp[r] - d.wm[r];  // the row's multiplier, for the H^T products
    if (with_jac && d.mc.kkt != 1) {  // reciprocals of the slacks and their duals, reused by every later kernel
      d.isp[r] = recip_nr(d.sp[r]);
      d.ism[r] = recip_nr(d.sm[r]);
      d.ibp[r] = recip_nr(d.bp[r]);
      d.ibm[r] = recip_nr(d.bm[r]);
    }
  }
}

__global__ void k_eval_rows(Dev d, int use_trial, int with_jac) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < d.m) eval_row_at(d, r, use_trial, with_jac);
}

// --------------------------------------------------------------- variables

// Objective share owned by variable v (tracking and control terms are
// attributed to the stage-k variable they penalize) and its gradient.
__device__ void eval_var_obj(const Dev& d, const double* y, int v, double* fshare, double* grad) {
  const ModelConst& mc = d.mc;
  const int i = d.var_inst[v];
  const int vo = d.inst_voff[i], T = d.inst_T[i];
  const int lv = v - vo;
  const int nx = mc.nx, nu = mc.nu;
  double f = 0.0, gr = 0.0;
  if (lv >= nx) {
    const int k = (lv - nx) / (nx + nu) + 1;
    const int q = (lv - nx) % (nx + nu);
    const double* yi = y + vo;
    const double dt = mc.dt;
    if (mc.model == MODEL_DISTILL || mc.model == MODEL_DDAE) {
      const int cu = (mc.model == MODEL_DDAE) ? mc.N : 0;  // u within the control block
      if (q == 0) {
        const double e = yi[lv] - d.p_sp[(size_t)i * d.sp_stride + k - 1];
        f = dt * e * e;
        gr = 2.0 * dt * e;
      } else if (q == nx + cu) {
        const double up = (k == 1) ? d.p_uprev[i] : yi[offu(mc, k - 1) + cu];
        const double du = yi[lv] - up, eu = yi[lv] - mc.ubar;
        f = mc.wdu * du * du + mc.wu * dt * eu * eu;
        gr = 2.0 * mc.wdu * du + 2.0 * mc.wu * dt * eu;
        if (k < T) gr -= 2.0 * mc.wdu * (yi[offu(mc, k + 1) + cu] - yi[lv]);
      }
    } else if (mc.model == MODEL_PLATE) {
      const double hh = 1.0 / mc.g;
      if (q < nx) {
        const double e = yi[lv] - d.p_sp[(size_t)i * d.sp_stride + q];
        f = dt * hh * hh * e * e;
        gr = 2.0 * dt * hh * hh * e;
      } else {
        f = mc.rho_u * dt * yi[lv] * yi[lv];
        gr = 2.0 * mc.rho_u * dt * yi[lv];
      }
    } else if (mc.model == MODEL_PPLATE) {
      if (q < nx) {
        const double w = pplate_weight(mc, q);
        const double e = yi[lv] - d.p_sp[(size_t)i * d.sp_stride + k - 1];
        f = dt * w * e * e;
        gr = 2.0 * dt * w * e;
      } else {
        f = mc.rho_u * dt * yi[lv] * yi[lv];
        gr = 2.0 * mc.rho_u * dt * yi[lv];
      }
    } else {
      if (q == 0) {
        const double e = yi[lv] - d.p_sp[(size_t)i * d.sp_stride + k - 1];
        f = dt * e * e;
        gr = 2.0 * dt * e;
      }
    }
  }
  if (fshare) *fshare = f;
  if (grad) *grad = gr;
}

// Hessian slots owned by variable v of stage k >= 1.  lam = w+ - w- of the
// rows of the backward-Euler step that ends at stage k (rows of stage k-1).
__device__ void eval_var_hess(const Dev& d, int v) {
  const ModelConst& mc = d.mc;
  const int i = d.var_inst[v];
  const int vo = d.inst_voff[i], ro = d.inst_roff[i], T = d.inst_T[i];
  const int lv = v - vo;
  const int nx = mc.nx, nu = mc.nu;
  if (lv < nx) return;
  const int k = (lv - nx) / (nx + nu) + 1;
  const int q = (lv - nx) % (nx + nu);
  double* W = d.Wv + d.inst_woff[i] + (size_t)(k - 1) * mc.WS;
  const double* yi = d.y + vo;
  const int rbase = ro + nx + mc.nr * (k - 1);  // rows of step k-1 -> k
  const double dt = mc.dt;
  if (mc.model == MODEL_PLATE) {
    const double hh = 1.0 / mc.g;
    W[q] = (q < nx) ? 2.0 * dt * hh * hh : 2.0 * mc.rho_u * dt;
    return;
  }
  if (mc.model == MODEL_DDAE) {
    // W slots of stage k (see the slot conventions): the balances are
    // bilinear in (flow, composition), the equilibria carry -vle(x_j)
    const int N = mc.N, Nf = mc.Nf;
    auto c = [&](int tray) { const int rr = rbase + tray - 1; return -dt * (d.wp[rr] - d.wm[rr]); };
    auto mu = [&](int j) { const int rr = rbase + N + j - 1; return d.wp[rr] - d.wm[rr]; };
    if (q < N) {  // x_j: its diagonal and its (flow, x_j) pair
      const int j = q + 1;
      const Vle v = vle_all(mc.alpha, yi[lv]);
      W[q] = (j == 1 ? 2.0 * dt : 0.0) - mu(j) * v.d2;
      if (j <= N - 1) {
        // x_j enters the tray below (x_{(j+1)-1}, inflow) and its own tray (outflow)
        double w = c(j + 1) * (j + 1 == N ? mc.inv_Ar : mc.inv_At);
        if (j >= 2) w -= c(j) * mc.inv_At;
        W[N + j - 1] = w;
      }
    } else if (q < 2 * N) {  // y_j, j >= 2: (V, y_j) from tray j-1 (y_{(j-1)+1}) and tray j (own)
      const int j = q - N + 1;
      if (j >= 2) {
        double w = c(j - 1) * (j - 1 == 1 ? mc.inv_Ac : mc.inv_At);
        w -= c(j) * (j == N ? mc.inv_Ar : mc.inv_At);
        W[2 * N + j - 2] = w;
      }
    } else if (q == 2 * N) {  // u: diagonal and (u_k, u_{k-1})
      W[3 * N - 1] = 2.0 * mc.wdu * (k < T ? 2.0 : 1.0) + 2.0 * mc.wu * dt;
      W[3 * N] = (k >= 2) ? -2.0 * mc.wdu : 0.0;
    } else if (q == 2 * N + 2) {  // V: (V, x_1) from the condenser
      W[2 * N - 1] = -c(1) * mc.inv_Ac;
    }
    return;
  }
  if (mc.model == MODEL_PPLATE) {
    if (q < nx) {
      W[q] = 2.0 * dt * pplate_weight(mc, q);
      return;
    }
    // the boundary data's curvature in Q, weighted by the multipliers of the
    // rows next to the controlled sides (the scaled constraint carries -s dt f):
    // d2/dQ2 4.1 Q^(1/3) = -(8.2/9) Q^(-5/3), d2/dQ2 Q^(1/2) = -Q^(-3/2) / 4
    const int mm = mc.g - 2;
    const double hh = 2.0 / (mc.g - 1), c = mc.kappa / (hh * hh);
    double sl = 0.0, sb = 0.0;
    for (int t = 0; t < mm; ++t) {
      sl += d.wp[rbase + t * mm] - d.wm[rbase + t * mm];  // x1 = -1 side: nodes (0, t)
      sb += d.wp[rbase + t] - d.wm[rbase + t];            // x2 = -1 side: nodes (t, 0)
    }
    const double Q = yi[lv], cb = cbrt(Q), sq = sqrt(Q);
    const double d2l = -(8.2 / 9.0) / (Q * cb * cb), d2b = -0.25 / (Q * sq);
    W[nx] = 2.0 * mc.rho_u * dt - pplate_row_scale(mc) * dt * c * (sl * d2l + sb * d2b);
    return;
  }
  if (mc.model == MODEL_TOY) {
    const double lam = d.wp[rbase] - d.wm[rbase];
    if (q == 0) W[0] = 2.0 * dt + lam * 6.0 * dt * yi[lv];
    else W[1] = lam * 4.0 * dt * sin(yi[lv]);
    return;
  }
  // distillation
  const int N = nx;
  const double a = mc.alpha, D = mc.D;
  const double* x = yi + offx(mc, k);
  const double u = yi[offu(mc, k)];
  const double V = (u + 1.0) * D;
  auto coef = [&](int tray) { const int r = rbase + tray - 1; return -dt * (d.wp[r] - d.wm[r]); };
  auto ihold = [&](int tray) { return tray == 1 ? mc.inv_Ac : (tray == N ? mc.inv_Ar : mc.inv_At); };
  if (q < N) {
    const int j = q + 1;  // tray
    const double xj = x[j - 1];
    const Vle vj = vle_all(a, xj);
    const double y1 = vj.d1, y2 = vj.d2;
    double wdiag = (j == 1) ? 2.0 * dt : 0.0;
    if (j >= 2) wdiag += coef(j) * (-V * y2) * ihold(j);           // own row: -V y''(x_j)
    if (j >= 2) wdiag += coef(j - 1) * (V * y2) * ihold(j - 1);    // row above: +V y''(x_{i+1})
    double wux = 0.0;
    if (j >= 2) wux += coef(j - 1) * (D * y1) * ihold(j - 1);      // row j-1: D y'(x_{i+1})
    if (j == 1) wux += coef(1) * (-D) * mc.inv_Ac;
    else if (j < N) wux += coef(j) * (-D * (1.0 + y1)) * mc.inv_At;
    else wux += coef(N) * (-D * y1) * mc.inv_Ar;
    if (j + 1 <= N) wux += coef(j + 1) * D * ihold(j + 1);         // row j+1: D from x_{i-1}
    W[q] = wdiag;
    W[N + q] = wux;
  } else {
    W[2 * N] = 2.0 * mc.wdu * (k < T ? 2.0 : 1.0) + 2.0 * mc.wu * dt;
    W[2 * N + 1] = (k >= 2) ? -2.0 * mc.wdu : 0.0;
  }
}

__device__ void eval_var_at(const Dev& d, int v, int use_trial) {
  const Ctl& c = d.ctl[d.var_inst[v]];
  if (use_trial) {
    if (!c.ls_active) return;
    eval_var_obj(d, d.yt, v, &d.fvart[v], nullptr);
  } else {
    if (c.status != ST_RUNNING) return;
    eval_var_obj(d, d.y, v, &d.fvar[v], &d.grad[v]);
    eval_var_hess(d, v);
    // reciprocals of the bound gaps and bound duals (0 where the bound is absent)
    const double y = d.y[v], lo = d.yL[v], hi = d.yU[v];
    d.igL[v] = isfinite(lo) ? recip_nr(y - lo) : 0.0;
    d.igU[v] = isfinite(hi) ? recip_nr(hi - y) : 0.0;
    d.izL[v] = isfinite(lo) ? recip_nr(d.zL[v]) : 0.0;
    d.izU[v] = isfinite(hi) ? recip_nr(d.zU[v]) : 0.0;
  }
}

__global__ void k_eval_vars(Dev d, int use_trial) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < d.n) eval_var_at(d, v, use_trial);
}

// rows (blocks 0 .. nbr-1) and variables (the rest) in one launch; the two
// are independent (the Hessian terms read the multipliers, not the rows' values)
__global__ void k_eval(Dev d, int use_trial, int with_jac, int nbr) {
  if ((int)blockIdx.x < nbr) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < d.m) eval_row_at(d, r, use_trial, with_jac);
  } else {
    const int v = (blockIdx.x - nbr) * blockDim.x + threadIdx.x;
    if (v < d.n) eval_var_at(d, v, use_trial);
  }
}

// --------------------------------------------------------- parameter update

// Writes new parameters into the device parameter buffers (Sec. 3.3,
// set_parameter_value): nothing structural changes.  src holds, per
// instance in [i0, i1), nx initial-state values, sp_len setpoint values and
// one u_prev (each part optional, flagged by the have_* arguments).
__global__ void k_set_params(Dev d, int i0, int i1, const double* x0, const double* sp,
                             const double* up, int sp_len) {
  const int nx = d.mc.nx;
  const int cnt = i1 - i0;
  const size_t total = (size_t)cnt * (nx + sp_len + 1);
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int li = (int)(t / (nx + sp_len + 1));
    const int q = (int)(t % (nx + sp_len + 1));
    const int i = i0 + li;
    if (q < nx) {
      if (x0) d.p_x0[(size_t)i * nx + q] = x0[(size_t)li * nx + q];
    } else if (q < nx + sp_len) {
      if (sp) d.p_sp[(size_t)i * d.sp_stride + (q - nx)] = sp[(size_t)li * sp_len + (q - nx)];
    } else {
      if (up) d.p_uprev[i] = up[li];
    }
  }
}

// All instances' parameters from arrays packed one instance after another,
// with T_i setpoints for instance i (instances of unequal horizons): one
// block per instance, spoff[i] = first setpoint of instance i.
__global__ void k_set_params_packed(Dev d, const int* spoff, const double* x0, const double* sp, const double* up) {
  const int i = blockIdx.x, nx = d.mc.nx;
  const int s0 = spoff[i], len = spoff[i + 1] - s0;
  for (int q = threadIdx.x; q < nx + len + 1; q += blockDim.x) {
    if (q < nx) {
      if (x0) d.p_x0[(size_t)i * nx + q] = x0[(size_t)i * nx + q];
    } else if (q < nx + len) {
      if (sp) d.p_sp[(size_t)i * d.sp_stride + (q - nx)] = sp[s0 + (q - nx)];
    } else if (up) {
      d.p_uprev[i] = up[i];
    }
  }
}

// One step of the closed loop (Algorithm 1) on the device, for every
// instance: the new initial state is the solution's x_1 (the plant is the
// same model) and, for the distillation, the new u_prev its u_1.
__global__ void k_shift_params(Dev d) {
  const int nx = d.mc.nx;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < d.n_inst * (nx + 1); t += gridDim.x * blockDim.x) {
    const int i = t / (nx + 1), q = t % (nx + 1);
    const double* yi = d.y + d.inst_voff[i];
    if (q < nx) d.p_x0[(size_t)i * nx + q] = yi[nx + q];
    else if (d.mc.model == MODEL_DISTILL) d.p_uprev[i] = yi[2 * nx];
    else if (d.mc.model == MODEL_DDAE) d.p_uprev[i] = yi[2 * nx + d.mc.N];
  }
}

// Cold-start trajectory from the parameters: x_k = p_x0 for all k, controls
// at u_prev (distillation) or the midpoint of their bounds, then pushed into
// the bounds (W&B Sec. 3.6).  Warm start only pushes the previous point.
__global__ void k_init_vars(Dev d, int warm, double push) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.n) return;
  const ModelConst& mc = d.mc;
  const int i = d.var_inst[v];
  const int lv = v - d.inst_voff[i];
  const int nx = mc.nx, nu = mc.nu;
  const double lo = d.yL[v], hi = d.yU[v];
  double y = d.y[v];
  if (!warm) {
    if (lv < nx) y = d.p_x0[(size_t)i * nx + lv];
    else {
      const int q = (lv - nx) % (nx + nu);
      if (q < nx) y = d.p_x0[(size_t)i * nx + q];
      else if (mc.model == MODEL_DISTILL || mc.model == MODEL_PPLATE) y = d.p_uprev[i];
      else if (mc.model == MODEL_DDAE) {
        // the algebraic variables consistent with x0 and u_prev
        const int cq = q - nx, N = mc.N;
        const double u = d.p_uprev[i];
        if (cq < N) {
          const double x = d.p_x0[(size_t)i * nx + cq];
          y = mc.alpha * x / (1.0 + (mc.alpha - 1.0) * x);
        } else {
          y = (cq == N) ? u : (cq == N + 1) ? u * mc.D : (cq == N + 2) ? u * mc.D + mc.D : u * mc.D + mc.F;
        }
      }
      else y = (isfinite(lo) && isfinite(hi)) ? 0.5 * (lo + hi) : 0.0;
    }
  }
  double pl = isfinite(lo) ? push * fmax(1.0, fabs(lo)) : 0.0;
  double pu = isfinite(hi) ? push * fmax(1.0, fabs(hi)) : 0.0;
  if (isfinite(lo) && isfinite(hi)) { pl = fmin(pl, push * (hi - lo)); pu = fmin(pu, push * (hi - lo)); }
  if (isfinite(lo) && y < lo + pl) y = lo + pl;
  if (isfinite(hi) && y > hi - pu) y = hi - pu;
  d.y[v] = y;
  if (!warm) {
    d.zL[v] = isfinite(lo) ? 1.0 : 0.0;
    d.zU[v] = isfinite(hi) ? 1.0 : 0.0;
  } else {
    d.zL[v] = isfinite(lo) ? fmax(d.zL[v], push) : 0.0;
    d.zU[v] = isfinite(hi) ? fmax(d.zU[v], push) : 0.0;
  }
}

__global__ void k_init_rows(Dev d, int warm, double push) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= d.m) return;
  const double gam = d.mc.gamma;
  if (d.mc.kkt == 1) {
    // HyKKT form: the multipliers lambda (wp) start at 0 cold and are kept
    // warm; wm stays 0 and the lifted slacks are unused (set to 1)
    if (!warm) d.wp[r] = 0.0;
    d.wm[r] = 0.0;
    d.sp[r] = d.sm[r] = d.bp[r] = d.bm[r] = 1.0;
    return;
  }
  if (!warm) {
    d.sp[r] = fmax(gam - d.h[r], push);
    d.sm[r] = fmax(gam + d.h[r], push);
    d.wp[r] = d.wm[r] = 1.0;
    d.bp[r] = d.bm[r] = 1.0;
  } else {
    d.sp[r] = fmax(d.sp[r], push);
    d.sm[r] = fmax(d.sm[r], push);
    d.bp[r] = fmax(d.bp[r], push);
    d.bm[r] = fmax(d.bm[r], push);
  }
}

}  // namespace nmpc
