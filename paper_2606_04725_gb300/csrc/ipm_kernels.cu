// Interior-point kernels: condensed-system assembly (eq. liftedkkt-pd), step
// recovery (eqs. infiniteOCP-condensed/augmented), step-length and
// line-search reductions (eq. infiniteOCP-lineSearch), and the per-instance
// control of barrier parameter, inertia correction and termination
// (eqs. infiniteOCP-innerTol/outerTol, Algorithm 2).
//
// Reductions are deterministic: every chunk of 2048 elements (never crossing
// an instance) is reduced by one block in a fixed tree order, and the
// per-instance control thread combines its chunks in index order.
#include <cfloat>

#include "kernels.h"

namespace nmpc {

__device__ __forceinline__ bool fin(double x) { return isfinite(x); }

// Fixed-order block reduction of NV doubles per thread with operator OP
// (0 sum, 1 max, 2 min).  Result valid in thread 0.
template <int NV>
__device__ void block_reduce(double (&v)[NV], const int (&op)[NV]) {
  __shared__ double sh[NV][TPB / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    for (int o = 16; o > 0; o >>= 1) {
      double t = __shfl_down_sync(0xffffffffu, v[q], o);
      v[q] = op[q] == 0 ? v[q] + t : (op[q] == 1 ? fmax(v[q], t) : fmin(v[q], t));
    }
    if (lane == 0) sh[q][wid] = v[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double a = sh[q][0];
      for (int w = 1; w < TPB / 32; ++w) a = op[q] == 0 ? a + sh[q][w] : (op[q] == 1 ? fmax(a, sh[q][w]) : fmin(a, sh[q][w]));
      v[q] = a;
    }
  }
  __syncthreads();
}

__global__ void k_ctl_init(Dev d, double mu0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n_inst) return;
  Ctl c{};
  c.mu = mu0;
  c.tau = fmax(TAU_MIN, 1.0 - mu0);
  c.status = ST_RUNNING;
  c.first = 1;
  d.ctl[i] = c;
}

// ----------------------------------------------------------- evaluation

// Stationarity, feasibility and complementarity of the lifted barrier
// problem (W&B eq. (5)) plus objective, log-barrier and theta sums.
__global__ void k_red_eval(Dev d) {
  const Chunk ch = d.chunks[blockIdx.x];
  const Ctl& c = d.ctl[ch.inst];
  if (c.status != ST_RUNNING) return;
  const double gam = d.mc.gamma;
  const int WH = d.mc.WH;
  double v[10] = {0.0, 0.0, 0.0, DBL_MAX, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const int op[10] = {1, 1, 1, 2, 0, 0, 0, 0, 0, 0};
  if (ch.kind == 0) {
    for (int j = ch.begin + threadIdx.x; j < ch.end; j += TPB) {
      double r = d.grad[j];
      for (int q = d.Hcsc_ptr[j]; q < d.Hcsc_ptr[j + 1]; ++q) {
        const int s = d.Hcsc_slot[q], row = s / WH;
        r += d.Hv[s] * (d.wp[row] - d.wm[row]);
      }
      const double yj = d.y[j], lo = d.yL[j], hi = d.yU[j];
      if (fin(lo)) {
        r -= d.zL[j];
        const double p = (yj - lo) * d.zL[j];
        v[2] = fmax(v[2], p); v[3] = fmin(v[3], p);
        v[5] += d.zL[j];
        v[7] += log(yj - lo);
      }
      if (fin(hi)) {
        r += d.zU[j];
        const double p = (hi - yj) * d.zU[j];
        v[2] = fmax(v[2], p); v[3] = fmin(v[3], p);
        v[5] += d.zU[j];
        v[7] += log(hi - yj);
      }
      if (!fin(r)) v[9] += 1.0;
      v[0] = fmax(v[0], fabs(r));
      v[6] += d.fvar[j];
    }
  } else {
    for (int r = ch.begin + threadIdx.x; r < ch.end; r += TPB) {
      const double h = d.h[r];
      if (!fin(h)) v[9] += 1.0;
      v[0] = fmax(v[0], fmax(fabs(d.wp[r] - d.bp[r]), fabs(d.wm[r] - d.bm[r])));
      const double cp = h - gam + d.sp[r], cm = -h - gam + d.sm[r];
      v[1] = fmax(v[1], fmax(fabs(cp), fabs(cm)));
      const double pp = d.sp[r] * d.bp[r], pm = d.sm[r] * d.bm[r];
      v[2] = fmax(v[2], fmax(pp, pm)); v[3] = fmin(v[3], fmin(pp, pm));
      v[4] += fabs(d.wp[r]) + fabs(d.wm[r]);
      v[5] += d.bp[r] + d.bm[r];
      v[7] += log(d.sp[r]) + log(d.sm[r]);
      v[8] += fabs(cp) + fabs(cm);
    }
  }
  block_reduce<10>(v, op);
  if (threadIdx.x == 0) {
    RedEval e;
    e.dual = v[0]; e.prim = v[1]; e.cmax = v[2]; e.cmin = v[3]; e.sum_l = v[4]; e.sum_z = v[5];
    e.f = v[6]; e.logsum = v[7]; e.theta = v[8]; e.nonfinite = v[9];
    d.red_eval[blockIdx.x] = e;
  }
}

// Convergence tests and barrier update (Algorithm 2 outer loop; W&B A-2/A-3).
__global__ void k_ctl_pre(Dev d, int max_iter) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n_inst) return;
  Ctl c = d.ctl[i];
  if (c.status != ST_RUNNING) return;
  double dual = 0, prim = 0, cmax = 0, cmin = DBL_MAX, sl = 0, sz = 0, f = 0, lg = 0, th = 0, nf = 0;
  for (int q = d.inst_chunk_ptr[i]; q < d.inst_chunk_ptr[i + 1]; ++q) {
    const RedEval& e = d.red_eval[d.inst_chunk_list[q]];
    dual = fmax(dual, e.dual); prim = fmax(prim, e.prim); cmax = fmax(cmax, e.cmax); cmin = fmin(cmin, e.cmin);
    sl += e.sum_l; sz += e.sum_z; f += e.f; lg += e.logsum; th += e.theta; nf += e.nonfinite;
  }
  const double mrows = d.inst_m[i], nz = d.inst_nz[i];
  const double sd = fmax(S_MAX, (sl + sz) / (2.0 * mrows + nz)) / S_MAX;
  const double sc = fmax(S_MAX, sz / nz) / S_MAX;
  c.E0 = fmax(fmax(dual / sd, prim), cmax / sc);
  c.E0u = fmax(fmax(dual, prim), cmax);
  c.f = f;
  if (nf > 0 || !fin(f) || !fin(th)) { c.status = 13; d.ctl[i] = c; return; }
  if (c.E0 <= d.mc.tol) { c.status = ST_CONVERGED; d.ctl[i] = c; return; }
  if (c.iter >= max_iter) { c.status = 10; d.ctl[i] = c; return; }
  const double mu_min = d.mc.tol / 10.0;
  auto emu = [&](double mu) { return fmax(fmax(dual / sd, prim), fmax(cmax - mu, mu - cmin) / sc); };
  double Emu = emu(c.mu);
  while (Emu <= KAPPA_EPS * c.mu && c.mu > mu_min) {
    c.mu = fmax(mu_min, fmin(KAPPA_MU * c.mu, pow(c.mu, THETA_MU)));
    c.tau = fmax(TAU_MIN, 1.0 - c.mu);
    c.nf = 0;
    Emu = emu(c.mu);
  }
  c.Emu = Emu;
  c.logsum = lg;
  c.theta = th;
  c.phi = f - c.mu * lg;
  if (c.iter == 0) {
    c.theta_max = 1e4 * fmax(1.0, th);
    c.theta_min = 1e-4 * fmax(1.0, th);
  }
  c.need_factor = 1;
  c.factor_fail = 0;
  c.dw = 0.0;
  d.ctl[i] = c;
}

// ------------------------------------------------------------- assembly

// zero the factor panels of every instance that is (re)factored now
__global__ void k_zero_L(Dev d, const long long* inst_Lbeg, const long long* inst_Lend) {
  const int i = blockIdx.y;
  if (!d.ctl[i].need_factor) return;
  const long long b = inst_Lbeg[i], e = inst_Lend[i];
  for (long long t = b + blockIdx.x * (long long)blockDim.x + threadIdx.x; t < e; t += (long long)gridDim.x * blockDim.x)
    d.Lval[t] = 0.0;
}

// Per row: D_r = Q+ + Q- (the lifted pair's barrier weight) and
// v_r = (w+ - w-) + (Q+ r4+ - r2+) - (Q- r4- - r2-), so that the condensed
// right-hand side is -(grad f - mu/(y-yL) + mu/(yU-y) + H^T v).
__global__ void k_rows_pre(Dev d, double* Drow) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= d.m) return;
  const Ctl& c = d.ctl[d.row_inst[r]];
  if (c.status != ST_RUNNING) return;
  const double mu = c.mu, gam = d.mc.gamma;
  const double sp = d.sp[r], sm = d.sm[r];
  const double Qp = d.bp[r] / sp, Qm = d.bm[r] / sm;
  Drow[r] = Qp + Qm;
  const double r4p = d.h[r] - gam + sp, r4m = -d.h[r] - gam + sm;
  const double r2p = d.wp[r] - mu / sp, r2m = d.wm[r] - mu / sm;
  d.rowv[r] = (d.wp[r] - d.wm[r]) + (Qp * r4p - r2p) - (Qm * r4m - r2m);
}

// K_c = W + Sigma_y + delta_w I + H^T D H gathered per stored factor entry
// (fixed term order: deterministic, no atomics).
__global__ void k_assemble(Dev d, const int* tgt_inst, const double* Drow) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d.n_tgt) return;
  const Ctl& c = d.ctl[tgt_inst[t]];
  if (!c.need_factor) return;
  const int WH = d.mc.WH;
  double v = 0.0;
  for (int q = d.tw_ptr[t]; q < d.tw_ptr[t + 1]; ++q) v += d.Wv[d.tw_idx[q]];
  for (int q = d.th_ptr[t]; q < d.th_ptr[t + 1]; ++q) {
    const int a = d.th_a[q], b = d.th_b[q];
    v += d.Hv[a] * Drow[a / WH] * d.Hv[b];
  }
  const int j = d.tgt_diag[t];
  if (j >= 0) {
    double sig = c.dw;
    const double yj = d.y[j];
    if (fin(d.yL[j])) sig += d.zL[j] / (yj - d.yL[j]);
    if (fin(d.yU[j])) sig += d.zU[j] / (d.yU[j] - yj);
    v += sig;
  }
  d.Lval[d.tgt_L[t]] = v;
}

// Inertia correction after a factorization attempt (W&B Algorithm IC on
// delta_w only; positive pivots <=> inertia of eq. infiniteOCP-inertia).
__global__ void k_ctl_factor(Dev d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n_inst) return;
  Ctl c = d.ctl[i];
  if (!c.need_factor) return;
  if (!c.factor_fail) {
    c.need_factor = 0;
    if (c.dw > 0.0) c.dw_last = c.dw;
  } else {
    c.factor_fail = 0;
    c.inertia_retries++;
    if (c.dw == 0.0) c.dw = (c.dw_last == 0.0) ? DELTA_W0 : fmax(DELTA_WMIN, KAPPA_W_MINUS * c.dw_last);
    else c.dw = (c.dw_last == 0.0) ? KAPPA_W_PLUS_BAR * c.dw : KAPPA_W_PLUS * c.dw;
    if (c.dw > DELTA_WMAX) { c.status = 12; c.need_factor = 0; }
  }
  d.ctl[i] = c;
}

// right-hand side of eq. liftedkkt-pd, scattered into the factor ordering
__global__ void k_rhs(Dev d) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.n) return;
  const Ctl& c = d.ctl[d.var_inst[v]];
  if (c.status != ST_RUNNING) return;
  const int WH = d.mc.WH;
  const double mu = c.mu;
  double r1 = d.grad[v];
  for (int q = d.Hcsc_ptr[v]; q < d.Hcsc_ptr[v + 1]; ++q) {
    const int s = d.Hcsc_slot[q];
    r1 += d.Hv[s] * d.rowv[s / WH];
  }
  if (fin(d.yL[v])) r1 -= mu / (d.y[v] - d.yL[v]);
  if (fin(d.yU[v])) r1 += mu / (d.yU[v] - d.y[v]);
  d.b[d.perm[v]] = -r1;
}

// --------------------------------------------------------------- recovery

__global__ void k_recover_vars(Dev d) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.n) return;
  const Ctl& c = d.ctl[d.var_inst[v]];
  if (c.status != ST_RUNNING) return;
  const double mu = c.mu;
  const double dy = d.b[d.perm[v]];
  d.dy[v] = dy;
  const double yv = d.y[v];
  double dzl = 0.0, dzu = 0.0;
  if (fin(d.yL[v])) { const double g = yv - d.yL[v]; dzl = mu / g - d.zL[v] - d.zL[v] / g * dy; }
  if (fin(d.yU[v])) { const double g = d.yU[v] - yv; dzu = mu / g - d.zU[v] + d.zU[v] / g * dy; }
  d.dzL[v] = dzl;
  d.dzU[v] = dzu;
}

// ds = -r4 -+ H dy, dw = -r2 - Q ds, db = mu/s - b - Q ds (eliminated rows of
// eq. infiniteOCP-augmented for both lifted sides)
__global__ void k_recover_rows(Dev d) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= d.m) return;
  const Ctl& c = d.ctl[d.row_inst[r]];
  if (c.status != ST_RUNNING) return;
  const int WH = d.mc.WH;
  const double mu = c.mu, gam = d.mc.gamma;
  double Hd = 0.0;
  for (int s = 0; s < WH; ++s) {
    const int col = d.Hcol[(size_t)r * WH + s];
    if (col >= 0) Hd += d.Hv[(size_t)r * WH + s] * d.dy[col];
  }
  const double sp = d.sp[r], sm = d.sm[r];
  const double Qp = d.bp[r] / sp, Qm = d.bm[r] / sm;
  const double r4p = d.h[r] - gam + sp, r4m = -d.h[r] - gam + sm;
  const double dsp = -r4p - Hd, dsm = -r4m + Hd;
  d.dsp[r] = dsp;
  d.dsm[r] = dsm;
  d.dwp[r] = -(d.wp[r] - mu / sp) - Qp * dsp;
  d.dwm[r] = -(d.wm[r] - mu / sm) - Qm * dsm;
  d.dbp[r] = mu / sp - d.bp[r] - Qp * dsp;
  d.dbm[r] = mu / sm - d.bm[r] - Qm * dsm;
}

// fraction-to-the-boundary step limits and grad(phi_mu)^T d
__global__ void k_red_dir(Dev d) {
  const Chunk ch = d.chunks[blockIdx.x];
  const Ctl& c = d.ctl[ch.inst];
  if (c.status != ST_RUNNING) return;
  const double mu = c.mu, tau = c.tau;
  double v[3] = {1.0, 1.0, 0.0};
  const int op[3] = {2, 2, 0};
  if (ch.kind == 0) {
    for (int j = ch.begin + threadIdx.x; j < ch.end; j += TPB) {
      const double dy = d.dy[j], yj = d.y[j];
      double gp = d.grad[j];
      if (fin(d.yL[j])) {
        const double g = yj - d.yL[j];
        if (dy < 0.0) v[0] = fmin(v[0], -tau * g / dy);
        gp -= mu / g;
        if (d.dzL[j] < 0.0) v[1] = fmin(v[1], -tau * d.zL[j] / d.dzL[j]);
      }
      if (fin(d.yU[j])) {
        const double g = d.yU[j] - yj;
        if (dy > 0.0) v[0] = fmin(v[0], tau * g / dy);
        gp += mu / g;
        if (d.dzU[j] < 0.0) v[1] = fmin(v[1], -tau * d.zU[j] / d.dzU[j]);
      }
      v[2] += gp * dy;
    }
  } else {
    for (int r = ch.begin + threadIdx.x; r < ch.end; r += TPB) {
      const double sp = d.sp[r], sm = d.sm[r];
      if (d.dsp[r] < 0.0) v[0] = fmin(v[0], -tau * sp / d.dsp[r]);
      if (d.dsm[r] < 0.0) v[0] = fmin(v[0], -tau * sm / d.dsm[r]);
      if (d.dbp[r] < 0.0) v[1] = fmin(v[1], -tau * d.bp[r] / d.dbp[r]);
      if (d.dbm[r] < 0.0) v[1] = fmin(v[1], -tau * d.bm[r] / d.dbm[r]);
      v[2] -= mu * (d.dsp[r] / sp + d.dsm[r] / sm);
    }
  }
  block_reduce<3>(v, op);
  if (threadIdx.x == 0) d.red_dir[blockIdx.x] = RedDir{v[0], v[1], v[2], 0.0};
}

// start of the backtracking filter line search (W&B Sec. 2.3): alpha_min
__global__ void k_ctl_dir(Dev d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n_inst) return;
  Ctl c = d.ctl[i];
  if (c.status != ST_RUNNING) return;
  double ap = 1.0, ad = 1.0, g = 0.0;
  for (int q = d.inst_chunk_ptr[i]; q < d.inst_chunk_ptr[i + 1]; ++q) {
    const RedDir& e = d.red_dir[d.inst_chunk_list[q]];
    ap = fmin(ap, e.ap); ad = fmin(ad, e.ad); g += e.gphi;
  }
  c.alpha_pri = ap;
  c.alpha_dual = ad;
  c.gphi = g;
  double amin;
  if (g < 0.0) {
    amin = fmin(GAMMA_THETA, GAMMA_PHI * c.theta / (-g));
    if (c.theta <= c.theta_min) amin = fmin(amin, DELTA_SW * pow(c.theta, S_THETA) / pow(-g, S_PHI));
    amin *= GAMMA_ALPHA;
  } else {
    amin = GAMMA_ALPHA * GAMMA_THETA;
  }
  c.alpha_min = amin;
  c.ls_trials0 = c.ls_trials;
  c.alpha = ap;
  c.phase = 0;
  c.augment = 0;
  if (c.alpha >= amin) c.ls_active = 1;
  else { c.ls_active = 0; c.status = 11; }
  d.ctl[i] = c;
}

// trial point y + alpha dy, s + alpha ds for instances still searching
__global__ void k_trial_point(Dev d) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < d.n) {
    const Ctl& c = d.ctl[d.var_inst[t]];
    if (c.ls_active) d.yt[t] = d.y[t] + c.alpha * d.dy[t];
  } else if (t < d.n + d.m) {
    const int r = t - d.n;
    const Ctl& c = d.ctl[d.row_inst[r]];
    if (c.ls_active) {
      d.spt[r] = d.sp[r] + c.alpha * d.dsp[r];
      d.smt[r] = d.sm[r] + c.alpha * d.dsm[r];
    }
  }
}

__global__ void k_red_trial(Dev d) {
  const Chunk ch = d.chunks[blockIdx.x];
  const Ctl& c = d.ctl[ch.inst];
  if (!c.ls_active) return;
  const double gam = d.mc.gamma;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  const int op[4] = {0, 0, 0, 0};
  if (ch.kind == 0) {
    for (int j = ch.begin + threadIdx.x; j < ch.end; j += TPB) {
      const double y = d.yt[j];
      v[0] += d.fvart[j];
      if (fin(d.yL[j])) v[1] += log(y - d.yL[j]);
      if (fin(d.yU[j])) v[1] += log(d.yU[j] - y);
    }
  } else {
    for (int r = ch.begin + threadIdx.x; r < ch.end; r += TPB) {
      const double h = d.ht[r];
      if (!fin(h)) v[3] += 1.0;
      v[1] += log(d.spt[r]) + log(d.smt[r]);
      v[2] += fabs(h - gam + d.spt[r]) + fabs(-h - gam + d.smt[r]);
    }
  }
  block_reduce<4>(v, op);
  if (threadIdx.x == 0) d.red_trial[blockIdx.x] = RedTrial{v[0], v[1], v[2], v[3]};
}

// filter acceptance test of one trial (W&B Sec. 2.3, A-5.2 .. A-5.4)
__global__ void k_ctl_ls(Dev d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n_inst) return;
  Ctl c = d.ctl[i];
  if (!c.ls_active) return;
  double f = 0, lg = 0, th = 0, nf = 0;
  for (int q = d.inst_chunk_ptr[i]; q < d.inst_chunk_ptr[i + 1]; ++q) {
    const RedTrial& e = d.red_trial[d.inst_chunk_list[q]];
    f += e.f; lg += e.logsum; th += e.theta; nf += e.nonfinite;
  }
  c.ls_trials++;
  const double phit = f - c.mu * lg, thetat = th;
  c.ft = f; c.logsum_t = lg; c.theta_t = th;
  bool ok = nf == 0 && fin(phit) && fin(thetat) && thetat <= c.theta_max;
  const double* fth = d.filt_th + (size_t)i * FILTER_CAP;
  const double* fph = d.filt_ph + (size_t)i * FILTER_CAP;
  for (int q = 0; ok && q < c.nf; ++q) if (thetat >= fth[q] && phit >= fph[q]) ok = false;
  bool accepted = false;
  if (ok) {
    const bool sw = c.gphi < 0.0 && c.alpha * pow(-c.gphi, S_PHI) > DELTA_SW * pow(c.theta, S_THETA);
    if (c.theta <= c.theta_min && sw) {
      if (phit <= c.phi + ETA_PHI * c.alpha * c.gphi) { accepted = true; c.augment = 0; }
    } else if (thetat <= (1.0 - GAMMA_THETA) * c.theta || phit <= c.phi - GAMMA_PHI * c.theta) {
      accepted = true;
      c.augment = 1;
    }
  }
  if (accepted) {
    c.ls_active = 0;
    c.phase = 1;
  } else {
    c.alpha *= 0.5;
    if (c.alpha < c.alpha_min) { c.ls_active = 0; c.status = 11; }
  }
  d.ctl[i] = c;
}

// accept the step; bound multipliers take the dual step and the safeguard
// of W&B eq. (16)
__global__ void k_update_vars(Dev d) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.n) return;
  const Ctl& c = d.ctl[d.var_inst[v]];
  if (c.phase != 1 || c.status != ST_RUNNING) return;
  const double y = d.yt[v], mu = c.mu, ad = c.alpha_dual;
  d.y[v] = y;
  if (fin(d.yL[v])) {
    const double g = y - d.yL[v];
    const double z = d.zL[v] + ad * d.dzL[v];
    d.zL[v] = fmax(fmin(z, KAPPA_SIGMA * mu / g), mu / (KAPPA_SIGMA * g));
  }
  if (fin(d.yU[v])) {
    const double g = d.yU[v] - y;
    const double z = d.zU[v] + ad * d.dzU[v];
    d.zU[v] = fmax(fmin(z, KAPPA_SIGMA * mu / g), mu / (KAPPA_SIGMA * g));
  }
}

__global__ void k_update_rows(Dev d) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= d.m) return;
  const Ctl& c = d.ctl[d.row_inst[r]];
  if (c.phase != 1 || c.status != ST_RUNNING) return;
  const double a = c.alpha, ad = c.alpha_dual, mu = c.mu;
  const double sp = d.spt[r], sm = d.smt[r];
  d.sp[r] = sp;
  d.sm[r] = sm;
  d.wp[r] += a * d.dwp[r];
  d.wm[r] += a * d.dwm[r];
  const double bp = d.bp[r] + ad * d.dbp[r], bm = d.bm[r] + ad * d.dbm[r];
  d.bp[r] = fmax(fmin(bp, KAPPA_SIGMA * mu / sp), mu / (KAPPA_SIGMA * sp));
  d.bm[r] = fmax(fmin(bm, KAPPA_SIGMA * mu / sm), mu / (KAPPA_SIGMA * sm));
}

__global__ void k_ctl_post(Dev d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n_inst) return;
  Ctl c = d.ctl[i];
  if (c.phase != 1) return;
  if (c.iter <= d.max_iter) {
    double* t = d.trace + ((size_t)i * (d.max_iter + 2) + c.iter) * 8;
    t[0] = c.mu; t[1] = c.alpha; t[2] = c.alpha_dual; t[3] = c.dw;
    t[4] = c.theta; t[5] = c.phi; t[6] = c.Emu; t[7] = c.ls_trials - c.ls_trials0;
  }
  if (c.augment && c.nf < FILTER_CAP) {
    d.filt_th[(size_t)i * FILTER_CAP + c.nf] = (1.0 - GAMMA_THETA) * c.theta;
    d.filt_ph[(size_t)i * FILTER_CAP + c.nf] = c.phi - GAMMA_PHI * c.theta;
    c.nf++;
  }
  c.iter++;
  c.phase = 0;
  d.ctl[i] = c;
}

// flags[0] = any instance running, [1] = any needs a factorization,
// [2] = any line search active
__global__ void k_summary(Dev d, int* flags) {
  __shared__ int f[3];
  if (threadIdx.x < 3) f[threadIdx.x] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < d.n_inst; i += blockDim.x) {
    const Ctl& c = d.ctl[i];
    if (c.status == ST_RUNNING) atomicOr(&f[0], 1);
    if (c.need_factor) atomicOr(&f[1], 1);
    if (c.ls_active) atomicOr(&f[2], 1);
  }
  __syncthreads();
  if (threadIdx.x < 3) flags[threadIdx.x] = f[threadIdx.x];
}

}  // namespace nmpc
