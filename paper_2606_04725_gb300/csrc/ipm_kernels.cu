// Interior-point kernels: condensed-system assembly (eq. liftedkkt-pd), step
// recovery (eqs. infiniteOCP-condensed/augmented), step-length and
// line-search reductions (eq. infiniteOCP-lineSearch), and the per-instance
// control of barrier parameter, inertia correction and termination
// (eqs. infiniteOCP-innerTol/outerTol, Algorithm 2).
//
// Reductions are deterministic: every chunk of RED_CHUNK elements (never
// crossing an instance) is reduced by one block in a fixed tree order, and
// one warp per instance combines its chunks in a fixed lane order and tree.
// Maxima and minima of non-negative values are taken on the bit patterns
// (integer operations), which order like the values: on this GPU every FP64
// instruction, compares included, costs tens of cycles.
#include <cfloat>

#include "kernels.h"

namespace nmpc {

__device__ __forceinline__ bool fin(double x) { return isfinite(x); }

// Running product of positive numbers kept as mantissa in [1, 2) times 2^e:
// sum_i log(x_i) = log(m) + e log 2 with one logarithm per chunk.  A
// non-positive or non-finite factor makes m non-finite (caught by callers).
__device__ __forceinline__ void logacc_mul(double& m, double& e, double x) {
  m *= x;
  const long long b = __double_as_longlong(m);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0 || ex == 0x7ff || m <= 0.0) {  // zero, subnormal, inf/nan or negative: leave to the caller
    if (!(m > 0.0) || ex == 0x7ff) m = __longlong_as_double(0x7ff8000000000000LL);
    else { int q; m = frexp(m, &q); e += q; }
    return;
  }
  e += ex - 1023;
  m = __longlong_as_double((b & ~(0x7ffLL << 52)) | (1023LL << 52));
}

constexpr double LN2 = 0.69314718055994530941723212145818;

// combine chunk partials (mantissa products) exactly as elements: one log at the end
__device__ __forceinline__ double logacc_value(double m, double e) { return log(m) + e * LN2; }

// max / min of doubles that are non-negative or -0 (negative values lose
// against 0 in max, which is how the callers use it: max(0, x_1, x_2, ...))
__device__ __forceinline__ double max_nn(double a, double b) {
  return __longlong_as_double(max(__double_as_longlong(a), __double_as_longlong(b)));
}
__device__ __forceinline__ double min_nn(double a, double b) {
  return __longlong_as_double(min(__double_as_longlong(a), __double_as_longlong(b)));
}

// combine one partial into another with operator op (0 sum, 1 max, 2 min)
__device__ __forceinline__ double combine(int op, double a, double b) {
  return op == 0 ? a + b : (op == 1 ? max_nn(a, b) : min_nn(a, b));
}

// Fixed-order warp reduction of NV doubles; result in lane 0.  Operator 3
// marks a log-product pair (mantissa in slot q, exponent sum in slot q+1).
template <int NV>
__device__ __forceinline__ void warp_reduce(double (&v)[NV], const int (&op)[NV]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const double t = __shfl_down_sync(0xffffffffu, v[q], o);
      if (op[q] == 3) {
        const double te = __shfl_down_sync(0xffffffffu, v[q + 1], o);
        logacc_mul(v[q], v[q + 1], t);
        v[q + 1] += te;
        ++q;
      } else {
        v[q] = combine(op[q], v[q], t);
      }
    }
  }
}

// Fixed-order block reduction (RED_CHUNK threads); result in thread 0.
template <int NV>
__device__ void block_reduce(double (&v)[NV], const int (&op)[NV]) {
  constexpr int NW = RED_CHUNK / 32;
  __shared__ double sh[NV][NW];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  warp_reduce<NV>(v, op);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[q][wid] = v[q];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = sh[q][0];
    for (int w = 1; w < NW; ++w) {
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        if (op[q] == 3) {
          logacc_mul(v[q], v[q + 1], sh[q][w]);
          v[q + 1] += sh[q + 1][w];
          ++q;
        } else {
          v[q] = combine(op[q], v[q], sh[q][w]);
        }
      }
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

// ---------------------------------------------------- fused step endings
// Every reduction kernel ends its step itself.  A chunk block stores its
// partial, then thread 0 fences (device scope) and arrives on its instance's
// counter; the block that arrives last sees every partial of the instance,
// and its warp 0 combines them and runs the instance's control step.  In the
// graph-driven loop the last instance to finish (a second counter) then sets
// the graph's conditions.  The block that completes a counter resets it, so
// every counter is zero again when the kernel ends.
__device__ __forceinline__ bool arrive_last(int* cnt, int total) {  // thread 0 only
  __threadfence();
  const int t = atomicAdd(cnt, 1);
  if (t != total - 1) return false;
  *cnt = 0;
  __threadfence();
  return true;
}
// uniform over the block: this block is the last of instance inst to arrive
__device__ __forceinline__ bool last_of_instance(const Dev& d, int inst) {
  __shared__ int s_last;
  if (threadIdx.x == 0) s_last = arrive_last(d.red_cnt + inst, d.inst_chunk_ptr[inst + 1] - d.inst_chunk_ptr[inst]);
  __syncthreads();
  return s_last != 0;
}
// uniform over the block: this block runs instance inst's control step.  An
// instance that took part stores a partial in every chunk, so its step runs
// on the last of its chunk blocks to arrive; one that did not (stopped, or
// not searching) has no partials: its first chunk block runs the step at
// once and the others leave without touching a counter -- in the last
// iterations of a batch most blocks are such, and each fence and atomic
// costs.
__device__ __forceinline__ bool runs_control(const Dev& d, int inst, bool active) {
  if (active) return last_of_instance(d, inst);
  return (int)blockIdx.x == d.inst_chunk_ptr[inst];  // chunks are numbered instance after instance
}
// uniform over the block: this block finished the last instance
__device__ __forceinline__ bool last_instance(const Dev& d) {
  __shared__ int s_last;
  if (threadIdx.x == 0) s_last = arrive_last(d.red_cnt + d.n_inst, d.n_inst);
  __syncthreads();
  return s_last != 0;
}

// any instance running / needing a factorization / searching / in CG (block-wide)
__device__ __forceinline__ void any_flags(const Dev& d, int* run, int* fac, int* ls, int* cg) {
  __shared__ int f[4];
  if (threadIdx.x < 4) f[threadIdx.x] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < d.n_inst; i += blockDim.x) {
    const Ctl& c = d.ctl[i];
    if (c.status == ST_RUNNING) atomicOr(&f[0], 1);
    if (c.need_factor) atomicOr(&f[1], 1);
    if (c.ls_active) atomicOr(&f[2], 1);
    if (c.cg_active) atomicOr(&f[3], 1);
  }
  __syncthreads();
  *run = f[0];
  *fac = f[1];
  *ls = f[2];
  *cg = f[3];
}

// Set the graph's conditions at the end of a step (block-wide) and count the
// trip.  The interior-point loop runs as one CUDA graph with conditional
// nodes: WHILE over iterations, IF on "still running", WHILE over inertia
// corrections, WHILE over line-search trials.  Every loop also stops at a trip
// limit, whatever the control state says, so a graph launch always ends.
enum StepEnd { END_EVAL = 0, END_FACTOR = 1, END_DIR = 2, END_TRIAL = 3, END_CG0 = 4, END_CG = 5 };
__device__ void set_conditions(const Dev& d, const CondArgs& ca, int kind) {
  int run, fac, ls, cg;
  any_flags(d, &run, &fac, &ls, &cg);
  if (threadIdx.x != 0) return;
  int* ctr = ca.counters;
  if (kind == END_CG0 || kind == END_CG) {  // the CG start, or a CG step (a trip)
    if (ctr[3] >= ca.cap_cg) cg = 0;
    cudaGraphSetConditional(ca.h_cg, cg ? 1u : 0u);
    if (kind == END_CG) ++ctr[3];
    return;
  }
  if (kind == END_EVAL) {
    if (ctr[0] >= ca.cap_iter) run = 0;
    cudaGraphSetConditional(ca.h_run, run ? 1u : 0u);
    cudaGraphSetConditional(ca.h_if, run ? 1u : 0u);
    cudaGraphSetConditional(ca.h_fac, (run && fac) ? 1u : 0u);
    ++ctr[0];
  } else if (kind == END_FACTOR) {
    if (ctr[1] >= ca.cap_inner) fac = 0;
    cudaGraphSetConditional(ca.h_fac, fac ? 1u : 0u);
    ++ctr[1];
  } else {
    if (ctr[2] >= ca.cap_inner) ls = 0;
    cudaGraphSetConditional(ca.h_ls, ls ? 1u : 0u);
    if (kind == END_TRIAL) ++ctr[2];
  }
}

// ----------------------------------------------------------- evaluation

// Stationarity, feasibility and complementarity of the lifted barrier
// problem (W&B eq. (5)) plus objective, log-barrier and theta sums.
__device__ void ctl_pre_warp(const Dev& d, int i, int lane, int max_iter);
__device__ void ctl_post(const Dev& d, int i, Ctl& c, bool write);

__global__ void k_red_eval(Dev d, int max_iter, CondArgs ca) {
  const Chunk ch = d.chunks[blockIdx.x];
  const Ctl& c = d.ctl[ch.inst];
  const bool active = c.status == ST_RUNNING;  // uniform over the block
  if (active) {
    const double gam = d.mc.gamma;
    const int WH = d.mc.WH;
    // dual, prim, cmax, cmin, sum_l, sum_z, f, log-mantissa, log-exponent, theta, nonfinite
    double v[11] = {0.0, 0.0, 0.0, DBL_MAX, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0};
    const int op[11] = {1, 1, 1, 2, 0, 0, 0, 3, 0, 0, 0};
    if (ch.kind == 0) {
      for (int t = ch.begin + threadIdx.x; t < ch.end; t += RED_CHUNK) {
        const int j = d.red_var[t];  // longest H columns first: lanes of a warp loop alike
        double r = d.grad[j];
        for (int q = d.Hcsc_ptr[j]; q < d.Hcsc_ptr[j + 1]; ++q) {
          const int s = d.Hcsc_slot[q];
          r += d.Hv[s] * d.lam[s / WH];
        }
        const double yj = d.y[j], lo = d.yL[j], hi = d.yU[j];
        if (fin(lo)) {
          r -= d.zL[j];
          const double p = (yj - lo) * d.zL[j];
          v[2] = max_nn(v[2], p); v[3] = min_nn(v[3], p);
          v[5] += d.zL[j];
          logacc_mul(v[7], v[8], yj - lo);
        }
        if (fin(hi)) {
          r += d.zU[j];
          const double p = (hi - yj) * d.zU[j];
          v[2] = max_nn(v[2], p); v[3] = min_nn(v[3], p);
          v[5] += d.zU[j];
          logacc_mul(v[7], v[8], hi - yj);
        }
        if (!fin(r)) v[10] += 1.0;
        v[0] = max_nn(v[0], fabs(r));
        v[6] += d.fvar[j];
      }
    } else if (d.mc.kkt == 1) {
      // HyKKT form: the equalities h = 0 themselves, multipliers lambda = wp
      for (int r = ch.begin + threadIdx.x; r < ch.end; r += RED_CHUNK) {
        const double h = d.h[r];
        if (!fin(h)) v[10] += 1.0;
        v[1] = max_nn(v[1], fabs(h));
        v[4] += fabs(d.wp[r]);
        v[9] += fabs(h);
      }
    } else {
      for (int r = ch.begin + threadIdx.x; r < ch.end; r += RED_CHUNK) {
        const double h = d.h[r];
        if (!fin(h)) v[10] += 1.0;
        v[0] = max_nn(v[0], max_nn(fabs(d.wp[r] - d.bp[r]), fabs(d.wm[r] - d.bm[r])));
        const double cp = h - gam + d.sp[r], cm = -h - gam + d.sm[r];
        v[1] = max_nn(v[1], max_nn(fabs(cp), fabs(cm)));
        const double pp = d.sp[r] * d.bp[r], pm = d.sm[r] * d.bm[r];
        v[2] = max_nn(v[2], max_nn(pp, pm)); v[3] = min_nn(v[3], min_nn(pp, pm));
        v[4] += fabs(d.wp[r]) + fabs(d.wm[r]);
        v[5] += d.bp[r] + d.bm[r];
        logacc_mul(v[7], v[8], d.sp[r]);
        logacc_mul(v[7], v[8], d.sm[r]);
        v[9] += fabs(cp) + fabs(cm);
      }
    }
    block_reduce<11>(v, op);
    if (threadIdx.x == 0) {
      RedEval e;
      e.dual = v[0]; e.prim = v[1]; e.cmax = v[2]; e.cmin = v[3]; e.sum_l = v[4]; e.sum_z = v[5];
      e.f = v[6]; e.lgm = v[7]; e.lge = v[8]; e.theta = v[9]; e.nonfinite = v[10];
      d.red_eval[blockIdx.x] = e;
    }
  }
  if (!runs_control(d, ch.inst, active)) return;
  if (threadIdx.x < 32) ctl_pre_warp(d, ch.inst, threadIdx.x, max_iter);
  if (ca.on && last_instance(d)) set_conditions(d, ca, END_EVAL);
}

// Convergence tests and barrier update (Algorithm 2 outer loop; W&B A-2/A-3).
// (warp 0 of the last chunk block of instance i)
__device__ void ctl_pre_warp(const Dev& d, int i, int lane, int max_iter) {
  Ctl c = d.ctl[i];
  if (c.phase == 1) {  // the previous iteration accepted a step
    ctl_post(d, i, c, lane == 0);
    if (c.status != ST_RUNNING) {
      if (lane == 0) d.ctl[i] = c;
      return;
    }
  }
  if (c.status != ST_RUNNING) return;
  // chunk partials: lanes in chunk order, then a fixed shuffle tree
  double v[11] = {0.0, 0.0, 0.0, DBL_MAX, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0};
  const int op[11] = {1, 1, 1, 2, 0, 0, 0, 3, 0, 0, 0};
  for (int q = d.inst_chunk_ptr[i] + lane; q < d.inst_chunk_ptr[i + 1]; q += 32) {
    const RedEval& e = d.red_eval[d.inst_chunk_list[q]];
    v[0] = max_nn(v[0], e.dual); v[1] = max_nn(v[1], e.prim); v[2] = max_nn(v[2], e.cmax); v[3] = min_nn(v[3], e.cmin);
    v[4] += e.sum_l; v[5] += e.sum_z; v[6] += e.f; v[9] += e.theta; v[10] += e.nonfinite;
    logacc_mul(v[7], v[8], e.lgm);
    v[8] += e.lge;
  }
  warp_reduce<11>(v, op);
  if (lane) return;
  const double dual = v[0], prim = v[1], cmax = v[2], cmin = v[3], sl = v[4], sz = v[5], f = v[6], th = v[9], nf = v[10];
  const double lg = logacc_value(v[7], v[8]);
  // W&B eq. (5)'s scaling: s_d over the rows' multipliers (2m lifted, m HyKKT) and
  // the bound multipliers (inst_nz counts the 2m slack bounds of the lifted rows)
  const bool hy = d.mc.kkt == 1;
  const double mrows = d.inst_m[i], nz = hy ? d.inst_nz[i] - 2.0 * mrows : (double)d.inst_nz[i];
  const double sd = fmax(S_MAX, (sl + sz) / ((hy ? 1.0 : 2.0) * mrows + nz)) / S_MAX;
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
// H_rs D_r for the WH slots of row r: each H^T D H term of the assembly is
// then one multiply-add, (H_ra D_r) H_rb, and the product H_ra D_r is formed
// once per slot instead of once per term.
__device__ __forceinline__ void row_hd(const Dev& d, int r, double D) {
  const int WH = d.mc.WH;
  for (int s = 0; s < WH; ++s) d.HD[(size_t)r * WH + s] = d.Hv[(size_t)r * WH + s] * D;
}

__device__ void rows_pre_at(const Dev& d, double* Drow, int r) {
  const Ctl& c = d.ctl[d.row_inst[r]];
  if (c.status != ST_RUNNING) return;
  if (d.mc.kkt == 1) {
    // HyKKT: K_gamma's weight gamma on every row, and v_r = lambda_r + gamma h_r,
    // so that the right-hand side is g = a + gamma H^T c with a = -(grad phi_mu
    // + H^T lambda), c = -h (the augmented first block row)
    const double gh = d.mc.hy_gamma;
    Drow[r] = gh;
    d.rowv[r] = d.wp[r] + gh * d.h[r];
    row_hd(d, r, gh);
    return;
  }
  const double mu = c.mu, gam = d.mc.gamma;
  const double sp = d.sp[r], sm = d.sm[r], isp = d.isp[r], ism = d.ism[r];
  const double Qp = d.bp[r] * isp, Qm = d.bm[r] * ism;
  Drow[r] = Qp + Qm;
  row_hd(d, r, Qp + Qm);
  const double r4p = d.h[r] - gam + sp, r4m = -d.h[r] - gam + sm;
  const double r2p = d.wp[r] - mu * isp, r2m = d.wm[r] - mu * ism;
  d.rowv[r] = (d.wp[r] - d.wm[r]) + (Qp * r4p - r2p) - (Qm * r4m - r2m);
}

__global__ void k_rows_pre(Dev d, double* Drow) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < d.m) rows_pre_at(d, Drow, r);
}

// k_zero_L and k_rows_pre in one launch (both precede the assembly and are
// independent): blocks 0 .. zx*n_inst-1 zero instance b / zx's panels with zx
// blocks each, the rest evaluate the rows
__global__ void k_zero_rows(Dev d, const long long* inst_Lbeg, const long long* inst_Lend, double* Drow, int zx) {
  const int zb = zx * d.n_inst;
  if ((int)blockIdx.x < zb) {
    const int i = blockIdx.x / zx, bx = blockIdx.x % zx;
    if (!d.ctl[i].need_factor) return;
    const long long e = inst_Lend[i];
    for (long long t = inst_Lbeg[i] + bx * (long long)blockDim.x + threadIdx.x; t < e; t += (long long)zx * blockDim.x)
      d.Lval[t] = 0.0;
  } else {
    const int r = (blockIdx.x - zb) * blockDim.x + threadIdx.x;
    if (r < d.m) rows_pre_at(d, Drow, r);
  }
}

// K_c = W + Sigma_y + delta_w I + H^T D H gathered per stored factor entry
// (fixed term order: deterministic, no atomics).
__global__ void k_assemble(Dev d, const int* tgt_inst, const double* Drow) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d.n_tgt) return;
  const Ctl& c = d.ctl[tgt_inst[t]];
  if (!c.need_factor) return;
  double v = 0.0;
  for (int q = d.tw_ptr[t]; q < d.tw_ptr[t + 1]; ++q) v += d.Wv[d.tw_idx[q]];
  for (int q = d.th_ptr[t]; q < d.th_ptr[t + 1]; ++q) v += d.HD[d.th_a[q]] * d.Hv[d.th_b[q]];
  const int j = d.tgt_diag[t];
  if (j >= 0) {
    // Sigma_y = zL/(y - yL) + zU/(yU - y) (reciprocals are 0 where a bound is absent)
    v += c.dw + d.zL[j] * d.igL[j] + d.zU[j] * d.igU[j];
    d.Kdiag[d.perm[j]] = v;
  }
  d.Lval[d.tgt_L[t]] = v;
}

// Inertia correction after a factorization attempt (W&B Algorithm IC on
// delta_w only; positive pivots <=> inertia of eq. infiniteOCP-inertia).
__device__ void ctl_factor_one(const Dev& d, int i) {
  Ctl c = d.ctl[i];
  if (!c.need_factor) return;
  if (!c.factor_fail) {
    c.need_factor = 0;
    if (c.dw > 0.0) c.dw_last = c.dw;
  } else {
    c.factor_fail = 0;
    c.inertia_retries++;
    // the first trial value is always tried; a raised value above dw_max ends the instance
    if (c.dw == 0.0) {
      c.dw = (c.dw_last == 0.0) ? DELTA_W0 : fmax(DELTA_WMIN, KAPPA_W_MINUS * c.dw_last);
    } else {
      c.dw = (c.dw_last == 0.0) ? KAPPA_W_PLUS_BAR * c.dw : KAPPA_W_PLUS * c.dw;
      if (c.dw > d.mc.dw_max) { c.status = 12; c.need_factor = 0; }
    }
  }
  d.ctl[i] = c;
}

// One block: a thread per instance, then the graph's conditions.
__global__ void k_ctl_factor(Dev d, CondArgs ca) {
  for (int i = threadIdx.x; i < d.n_inst; i += blockDim.x) ctl_factor_one(d, i);
  if (ca.on) {
    __syncthreads();
    set_conditions(d, ca, END_FACTOR);
  }
}


// right-hand side of eq. liftedkkt-pd, scattered into the factor ordering
__global__ void k_rhs(Dev d) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d.n) return;
  const int v = d.red_var[t];  // longest H columns first: lanes of a warp loop alike
  const Ctl& c = d.ctl[d.var_inst[v]];
  if (c.status != ST_RUNNING) return;
  const int WH = d.mc.WH;
  const double mu = c.mu;
  double r1 = d.grad[v];
  for (int q = d.Hcsc_ptr[v]; q < d.Hcsc_ptr[v + 1]; ++q) {
    const int s = d.Hcsc_slot[q];
    r1 += d.Hv[s] * d.rowv[s / WH];
  }
  r1 += mu * (d.igU[v] - d.igL[v]);
  d.b[d.perm[v]] = -r1;
}

// --------------------------------------------------------------- recovery

__device__ void recover_var(const Dev& d, int v) {
  const Ctl& c = d.ctl[d.var_inst[v]];
  if (c.status != ST_RUNNING) return;
  const double mu = c.mu;
  const double dy = d.b[d.perm[v]];
  d.dy[v] = dy;
  double dzl = 0.0, dzu = 0.0;
  if (fin(d.yL[v])) { const double ig = d.igL[v]; dzl = mu * ig - d.zL[v] - d.zL[v] * ig * dy; }
  if (fin(d.yU[v])) { const double ig = d.igU[v]; dzu = mu * ig - d.zU[v] + d.zU[v] * ig * dy; }
  d.dzL[v] = dzl;
  d.dzU[v] = dzu;
}

// ds = -r4 -+ H dy, dw = -r2 - Q ds, db = mu/s - b - Q ds (eliminated rows of
// eq. infiniteOCP-augmented for both lifted sides)
__device__ void recover_row(const Dev& d, int r) {
  const Ctl& c = d.ctl[d.row_inst[r]];
  if (c.status != ST_RUNNING) return;
  const int WH = d.mc.WH;
  const double mu = c.mu, gam = d.mc.gamma;
  double Hd = 0.0;
  for (int s = 0; s < WH; ++s) {
    const int pos = d.Hpos[(size_t)r * WH + s];
    if (pos >= 0) Hd += d.Hv[(size_t)r * WH + s] * d.b[pos];  // dy, read where the solve left it
  }
  const double sp = d.sp[r], sm = d.sm[r], isp = d.isp[r], ism = d.ism[r];
  const double Qp = d.bp[r] * isp, Qm = d.bm[r] * ism;
  const double r4p = d.h[r] - gam + sp, r4m = -d.h[r] - gam + sm;
  const double dsp = -r4p - Hd, dsm = -r4m + Hd;
  d.dsp[r] = dsp;
  d.dsm[r] = dsm;
  d.dwp[r] = -(d.wp[r] - mu * isp) - Qp * dsp;
  d.dwm[r] = -(d.wm[r] - mu * ism) - Qm * dsm;
  d.dbp[r] = mu * isp - d.bp[r] - Qp * dsp;
  d.dbm[r] = mu * ism - d.bm[r] - Qm * dsm;
}


// Fraction-to-the-boundary step limits and grad(phi_mu)^T d.  The limits are
// tau / max_i(-dv_i / v_i) over components moving toward their bound, with
// the stored reciprocals, so the chunk needs no division per element.
__device__ void ctl_dir_warp(const Dev& d, int i, int lane);

__global__ void k_red_dir(Dev d, CondArgs ca) {
  const Chunk ch = d.chunks[blockIdx.x];
  const Ctl& c = d.ctl[ch.inst];
  const bool active = c.status == ST_RUNNING;  // uniform over the block
  if (active) {
    const double mu = c.mu, tau = c.tau;
    double v[3] = {0.0, 0.0, 0.0};  // max primal ratio, max dual ratio, gphi
    const int op[3] = {1, 1, 0};
    // the chunk's elements are recovered by the threads that reduce them
    if (ch.kind == 0) {
      for (int j = ch.begin + threadIdx.x; j < ch.end; j += RED_CHUNK) {
        recover_var(d, j);
        const double dy = d.dy[j];
        double gp = d.grad[j];
        if (fin(d.yL[j])) {
          const double ig = d.igL[j];
          v[0] = max_nn(v[0], -dy * ig);
          gp -= mu * ig;
          v[1] = max_nn(v[1], -d.dzL[j] * d.izL[j]);
        }
        if (fin(d.yU[j])) {
          const double ig = d.igU[j];
          v[0] = max_nn(v[0], dy * ig);
          gp += mu * ig;
          v[1] = max_nn(v[1], -d.dzU[j] * d.izU[j]);
        }
        v[2] += gp * dy;
      }
    } else if (d.mc.kkt != 1) {  // HyKKT: lambda's step is the CG iterate, no slacks
      for (int r = ch.begin + threadIdx.x; r < ch.end; r += RED_CHUNK) {
        recover_row(d, r);
        const double isp = d.isp[r], ism = d.ism[r];
        v[0] = max_nn(v[0], max_nn(-d.dsp[r] * isp, -d.dsm[r] * ism));
        v[1] = max_nn(v[1], max_nn(-d.dbp[r] * d.ibp[r], -d.dbm[r] * d.ibm[r]));
        v[2] -= mu * (d.dsp[r] * isp + d.dsm[r] * ism);
      }
    }
    block_reduce<3>(v, op);
    if (threadIdx.x == 0) {
      const double ap = v[0] > tau ? tau / v[0] : 1.0;
      const double ad = v[1] > tau ? tau / v[1] : 1.0;
      d.red_dir[blockIdx.x] = RedDir{ap, ad, v[2], 0.0};
    }
  }
  if (!runs_control(d, ch.inst, active)) return;
  if (threadIdx.x < 32) ctl_dir_warp(d, ch.inst, threadIdx.x);
  if (ca.on && last_instance(d)) set_conditions(d, ca, END_DIR);
}

// start of the backtracking filter line search (W&B Sec. 2.3): alpha_min
// (warp 0 of the last chunk block of instance i)
__device__ void ctl_dir_warp(const Dev& d, int i, int lane) {
  Ctl c = d.ctl[i];
  if (c.status != ST_RUNNING) return;
  double v[3] = {1.0, 1.0, 0.0};
  const int op[3] = {2, 2, 0};
  for (int q = d.inst_chunk_ptr[i] + lane; q < d.inst_chunk_ptr[i + 1]; q += 32) {
    const RedDir& e = d.red_dir[d.inst_chunk_list[q]];
    v[0] = min_nn(v[0], e.ap); v[1] = min_nn(v[1], e.ad); v[2] += e.gphi;
  }
  warp_reduce<3>(v, op);
  if (lane) return;
  const double ap = v[0], ad = v[1], g = v[2];
  c.alpha_pri = ap;
  c.alpha_dual = ad;
  c.gphi = g;
  double amin;
  // switching-condition powers, fixed within the iteration's line search
  c.sw_gphi = g < 0.0 ? pow(-g, S_PHI) : 0.0;
  c.sw_theta = DELTA_SW * pow(c.theta, S_THETA);
  if (g < 0.0) {
    amin = fmin(GAMMA_THETA, GAMMA_PHI * c.theta / (-g));
    if (c.theta <= c.theta_min) amin = fmin(amin, c.sw_theta / c.sw_gphi);
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
    if (c.ls_active && d.mc.kkt != 1) {
      d.spt[r] = d.sp[r] + c.alpha * d.dsp[r];
      d.smt[r] = d.sm[r] + c.alpha * d.dsm[r];
    }
  }
}

__device__ void ctl_ls_warp(const Dev& d, int i, int lane);

__global__ void k_red_trial(Dev d, CondArgs ca) {
  const Chunk ch = d.chunks[blockIdx.x];
  const Ctl& c = d.ctl[ch.inst];
  const bool active = c.ls_active != 0;  // uniform over the block
  if (active) {
    const double gam = d.mc.gamma;
    double v[5] = {0.0, 1.0, 0.0, 0.0, 0.0};  // f, log-mantissa, log-exponent, theta, nonfinite
    const int op[5] = {0, 3, 0, 0, 0};
    if (ch.kind == 0) {
      for (int j = ch.begin + threadIdx.x; j < ch.end; j += RED_CHUNK) {
        const double y = d.yt[j];
        v[0] += d.fvart[j];
        if (fin(d.yL[j])) logacc_mul(v[1], v[2], y - d.yL[j]);
        if (fin(d.yU[j])) logacc_mul(v[1], v[2], d.yU[j] - y);
      }
    } else if (d.mc.kkt == 1) {  // HyKKT: theta = ||h||_1, no slack barrier terms
      for (int r = ch.begin + threadIdx.x; r < ch.end; r += RED_CHUNK) {
        const double h = d.ht[r];
        if (!fin(h)) v[4] += 1.0;
        v[3] += fabs(h);
      }
    } else {
      for (int r = ch.begin + threadIdx.x; r < ch.end; r += RED_CHUNK) {
        const double h = d.ht[r];
        if (!fin(h)) v[4] += 1.0;
        logacc_mul(v[1], v[2], d.spt[r]);
        logacc_mul(v[1], v[2], d.smt[r]);
        v[3] += fabs(h - gam + d.spt[r]) + fabs(-h - gam + d.smt[r]);
      }
    }
    block_reduce<5>(v, op);
    if (threadIdx.x == 0) d.red_trial[blockIdx.x] = RedTrial{v[0], v[1], v[2], v[3], v[4]};
  }
  if (!runs_control(d, ch.inst, active)) return;
  if (threadIdx.x < 32) ctl_ls_warp(d, ch.inst, threadIdx.x);
  if (ca.on && last_instance(d)) set_conditions(d, ca, END_TRIAL);
}

// filter acceptance test of one trial (W&B Sec. 2.3, A-5.2 .. A-5.4)
// (warp 0 of the last chunk block of instance i)
__device__ void ctl_ls_warp(const Dev& d, int i, int lane) {
  Ctl c = d.ctl[i];
  if (!c.ls_active) return;
  double v[5] = {0.0, 1.0, 0.0, 0.0, 0.0};  // f, log-mantissa, log-exponent, theta, nonfinite
  const int op[5] = {0, 3, 0, 0, 0};
  for (int q = d.inst_chunk_ptr[i] + lane; q < d.inst_chunk_ptr[i + 1]; q += 32) {
    const RedTrial& e = d.red_trial[d.inst_chunk_list[q]];
    v[0] += e.f; v[3] += e.theta; v[4] += e.nonfinite;
    logacc_mul(v[1], v[2], e.lgm);
    v[2] += e.lge;
  }
  warp_reduce<5>(v, op);
  const double f = __shfl_sync(0xffffffffu, v[0], 0), th = __shfl_sync(0xffffffffu, v[3], 0);
  const double nf = __shfl_sync(0xffffffffu, v[4], 0);
  const double lg = logacc_value(__shfl_sync(0xffffffffu, v[1], 0), __shfl_sync(0xffffffffu, v[2], 0));
  const double phit = f - c.mu * lg, thetat = th;
  // filter test: lanes over the entries, any rejecting entry rejects
  bool blocked = false;
  {
    const double* fth = d.filt_th + (size_t)i * FILTER_CAP;
    const double* fph = d.filt_ph + (size_t)i * FILTER_CAP;
    for (int q = lane; q < c.nf; q += 32) blocked = blocked || (thetat >= fth[q] && phit >= fph[q]);
  }
  blocked = __any_sync(0xffffffffu, blocked);
  if (lane) return;
  c.ls_trials++;
  c.ft = f; c.logsum_t = lg; c.theta_t = th;
  const bool ok = nf == 0 && fin(phit) && fin(thetat) && thetat <= c.theta_max && !blocked;
  bool accepted = false;
  if (ok) {
    const bool sw = c.gphi < 0.0 && c.alpha * c.sw_gphi > c.sw_theta;
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

// Keep a bound multiplier z within [mu/(kappa g), kappa mu/g] for gap g
// (W&B eq. (16)); the division happens only when the bound is active.
__device__ __forceinline__ double safeguard(double z, double g, double mu) {
  const double p = z * g;
  if (p > KAPPA_SIGMA * mu) return KAPPA_SIGMA * mu / g;
  if (p < mu / KAPPA_SIGMA) return mu / (KAPPA_SIGMA * g);
  return z;
}

// accept the step; bound multipliers take the dual step and the safeguard
// of W&B eq. (16)
__device__ void update_var(const Dev& d, int v) {
  const Ctl& c = d.ctl[d.var_inst[v]];
  if (c.phase != 1 || c.status != ST_RUNNING) return;
  const double y = d.yt[v], mu = c.mu, ad = c.alpha_dual;
  d.y[v] = y;
  if (fin(d.yL[v])) d.zL[v] = safeguard(d.zL[v] + ad * d.dzL[v], y - d.yL[v], mu);
  if (fin(d.yU[v])) d.zU[v] = safeguard(d.zU[v] + ad * d.dzU[v], d.yU[v] - y, mu);
}

__device__ void update_row(const Dev& d, int r) {
  const Ctl& c = d.ctl[d.row_inst[r]];
  if (c.phase != 1 || c.status != ST_RUNNING) return;
  if (d.mc.kkt == 1) {  // HyKKT: lambda takes the primal step
    d.wp[r] += c.alpha * d.dwp[r];
    return;
  }
  const double a = c.alpha, ad = c.alpha_dual, mu = c.mu;
  const double sp = d.spt[r], sm = d.smt[r];
  d.sp[r] = sp;
  d.sm[r] = sm;
  d.wp[r] += a * d.dwp[r];
  d.wm[r] += a * d.dwm[r];
  d.bp[r] = safeguard(d.bp[r] + ad * d.dbp[r], sp, mu);
  d.bm[r] = safeguard(d.bm[r] + ad * d.dbm[r], sm, mu);
}

// variables (threads 0 .. n-1) and rows (n .. n+m-1) in one launch
__global__ void k_update(Dev d) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < d.n) update_var(d, t);
  else if (t < d.n + d.m) update_row(d, t - d.n);
}

// The bookkeeping of the step accepted in the previous iteration (trace
// record, filter entry on an augmenting step, iteration count), run by the
// evaluation's control step (ctl_pre_warp) before its tests.
__device__ void ctl_post(const Dev& d, int i, Ctl& c, bool write) {
  if (write && c.iter <= d.max_iter) {
    double* t = d.trace + ((size_t)i * (d.max_iter + 2) + c.iter) * 8;
    t[0] = c.mu; t[1] = c.alpha; t[2] = c.alpha_dual; t[3] = c.dw;
    t[4] = c.theta; t[5] = c.phi; t[6] = c.Emu; t[7] = c.ls_trials - c.ls_trials0;
  }
  if (c.augment && c.nf < FILTER_CAP) {
    if (write) {
      d.filt_th[(size_t)i * FILTER_CAP + c.nf] = (1.0 - GAMMA_THETA) * c.theta;
      d.filt_ph[(size_t)i * FILTER_CAP + c.nf] = c.phi - GAMMA_PHI * c.theta;
    }
    c.nf++;
  }
  c.iter++;
  c.phase = 0;
}

// ------------------------------------------------------------------ HyKKT
// The Newton system with the equalities kept,
//   [Wh  H^T] [dy  ]   [a]   a = -(grad phi_mu + H^T lambda), c = -h,
//   [H   0  ] [dlam] = [c],  Wh = W + Sigma_y + delta_w I,
// solved as the hybrid direct-iterative method that Sec. 3.2.2 cites
// (Regev et al. 2023, after Golub & Greif 2003): with the factor of
// K_gamma = Wh + gamma H^T H and g = a + gamma H^T c (k_rhs, rows_pre_at),
//   u = K_gamma^-1 g,  S dlam = H u - c  with S = H K_gamma^-1 H^T  (CG),
//   dy = K_gamma^-1 (g - H^T dlam).
// Every instance runs its own CG (the batch's S is block diagonal) from
// dlam = 0 until ||r||^2 <= cg_tol^2 ||r_0||^2, cg_max_iter steps, or
// p^T S p <= 0.  One CG step:
//   k_cg_apply  b = H^T (r + beta p)                       (variables)
//   solves      b = K_gamma^-1 b, instances in CG only
//   k_red_cg1   p = r + beta p, q = H b, alpha = r^T r / p^T q
//   k_red_cg2   dlam += alpha p, r -= alpha q, beta = r'^T r' / r^T r, stop test
// p's update happens in k_red_cg1 with the r and beta that k_cg_apply used.
// Dot products are deterministic chunk reductions like the others.

__device__ __forceinline__ double row_times_b(const Dev& d, int r) {  // (H b)_r, b in factor order
  const int WH = d.mc.WH;
  double s = 0.0;
  for (int q = 0; q < WH; ++q) {
    const int pos = d.Hpos[(size_t)r * WH + q];
    if (pos >= 0) s += d.Hv[(size_t)r * WH + q] * d.b[pos];
  }
  return s;
}

// control of instance i's CG after a dot product (warp 0 of the instance's
// last chunk block): step 0 the start (r_0^T r_0), 1 alpha (p^T q), 2 beta and
// the stop test (r^T r after the update)
__device__ void ctl_cg_warp(const Dev& d, int i, int lane, int step) {
  Ctl c = d.ctl[i];
  if (c.status != ST_RUNNING || (step > 0 && !c.cg_active)) return;
  double v[1] = {0.0};
  const int op[1] = {0};
  for (int q = d.inst_chunk_ptr[i] + lane; q < d.inst_chunk_ptr[i + 1]; q += 32) v[0] += d.red_cg[d.inst_chunk_list[q]];
  warp_reduce<1>(v, op);
  if (lane) return;
  const double s = v[0];
  if (step == 0) {
    c.cg_rr = s;
    c.cg_stop = d.mc.cg_tol * d.mc.cg_tol * s;
    c.cg_beta = 0.0;
    c.cg_it = 0;
    c.cg_active = (s > c.cg_stop && d.mc.cg_max_iter > 0) ? 1 : 0;
  } else if (step == 1) {
    if (s > 0.0) c.cg_alpha = c.cg_rr / s;
    else c.cg_active = 0;  // p^T S p <= 0 (or not finite): stop with the current dlam
  } else {
    c.cg_beta = s / c.cg_rr;
    c.cg_rr = s;
    c.cg_it++;
    c.cg_total++;
    c.cg_active = (s > c.cg_stop && c.cg_it < d.mc.cg_max_iter) ? 1 : 0;
  }
  c.solve_skip = c.cg_active ? 0 : 1;
  d.ctl[i] = c;
}

// After u = K_gamma^-1 g (in b): r_0 = H u + h, p = 0 and dlam = 0, then r_0^T r_0
__global__ void k_red_cg0(Dev d, CondArgs ca) {
  const Chunk ch = d.chunks[blockIdx.x];
  const Ctl& c = d.ctl[ch.inst];
  if (c.status == ST_RUNNING && ch.kind == 1) {  // uniform over the block
    double v[1] = {0.0};
    const int op[1] = {0};
    for (int r = ch.begin + threadIdx.x; r < ch.end; r += RED_CHUNK) {
      const double t = row_times_b(d, r) + d.h[r];
      d.cg_r[r] = t;
      d.cg_p[r] = 0.0;
      d.dwp[r] = 0.0;
      v[0] += t * t;
    }
    block_reduce<1>(v, op);
    if (threadIdx.x == 0) d.red_cg[blockIdx.x] = v[0];
  } else if (threadIdx.x == 0) {
    d.red_cg[blockIdx.x] = 0.0;
  }
  if (!last_of_instance(d, ch.inst)) return;
  if (threadIdx.x < 32) ctl_cg_warp(d, ch.inst, threadIdx.x, 0);
  if (ca.on && last_instance(d)) set_conditions(d, ca, END_CG0);
}

// b = H^T (r + beta p) in factor order, for the instances in CG
__global__ void k_cg_apply(Dev d) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.n) return;
  const Ctl& c = d.ctl[d.var_inst[v]];
  if (c.status != ST_RUNNING || !c.cg_active) return;
  const int WH = d.mc.WH;
  const double beta = c.cg_beta;
  double s = 0.0;
  for (int q = d.Hcsc_ptr[v]; q < d.Hcsc_ptr[v + 1]; ++q) {
    const int sl = d.Hcsc_slot[q], row = sl / WH;
    s += d.Hv[sl] * (d.cg_r[row] + beta * d.cg_p[row]);
  }
  d.b[d.perm[v]] = s;
}

// p = r + beta p, q = H K^-1 H^T p (H times the solves' result), then p^T q
__global__ void k_red_cg1(Dev d) {
  const Chunk ch = d.chunks[blockIdx.x];
  const Ctl& c = d.ctl[ch.inst];
  if (c.status == ST_RUNNING && c.cg_active && ch.kind == 1) {  // uniform over the block
    double v[1] = {0.0};
    const int op[1] = {0};
    const double beta = c.cg_beta;
    for (int r = ch.begin + threadIdx.x; r < ch.end; r += RED_CHUNK) {
      const double p = d.cg_r[r] + beta * d.cg_p[r];
      const double q = row_times_b(d, r);
      d.cg_p[r] = p;
      d.cg_q[r] = q;
      v[0] += p * q;
    }
    block_reduce<1>(v, op);
    if (threadIdx.x == 0) d.red_cg[blockIdx.x] = v[0];
  } else if (threadIdx.x == 0) {
    d.red_cg[blockIdx.x] = 0.0;
  }
  if (!last_of_instance(d, ch.inst)) return;
  if (threadIdx.x < 32) ctl_cg_warp(d, ch.inst, threadIdx.x, 1);
}

// dlam += alpha p, r -= alpha q, then r^T r and the stop test
__global__ void k_red_cg2(Dev d, CondArgs ca) {
  const Chunk ch = d.chunks[blockIdx.x];
  const Ctl& c = d.ctl[ch.inst];
  if (c.status == ST_RUNNING && c.cg_active && ch.kind == 1) {  // uniform over the block
    double v[1] = {0.0};
    const int op[1] = {0};
    const double a = c.cg_alpha;
    for (int r = ch.begin + threadIdx.x; r < ch.end; r += RED_CHUNK) {
      d.dwp[r] += a * d.cg_p[r];
      const double rn = d.cg_r[r] - a * d.cg_q[r];
      d.cg_r[r] = rn;
      v[0] += rn * rn;
    }
    block_reduce<1>(v, op);
    if (threadIdx.x == 0) d.red_cg[blockIdx.x] = v[0];
  } else if (threadIdx.x == 0) {
    d.red_cg[blockIdx.x] = 0.0;
  }
  if (!last_of_instance(d, ch.inst)) return;
  if (threadIdx.x < 32) ctl_cg_warp(d, ch.inst, threadIdx.x, 2);
  if (ca.on && last_instance(d)) set_conditions(d, ca, END_CG);
}

// right-hand side of the final solve, g - H^T dlam = -(grad phi_mu + H^T (v + dlam))
// with v = lambda + gamma h; every running instance solves again
__global__ void k_hy_rhs(Dev d) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < d.n_inst) d.ctl[v].solve_skip = 0;  // no other thread of this launch reads that field
  if (v >= d.n) return;
  const Ctl& c = d.ctl[d.var_inst[v]];
  if (c.status != ST_RUNNING) return;
  const int WH = d.mc.WH;
  double r1 = d.grad[v];
  for (int q = d.Hcsc_ptr[v]; q < d.Hcsc_ptr[v + 1]; ++q) {
    const int sl = d.Hcsc_slot[q], row = sl / WH;
    r1 += d.Hv[sl] * (d.rowv[row] + d.dwp[row]);
  }
  r1 += c.mu * (d.igU[v] - d.igL[v]);
  d.b[d.perm[v]] = -r1;
}

// flags[0] = any instance running, [1] = any needs a factorization,
// [2] = any line search active (cg = 0) or any CG running (cg = 1)
__global__ void k_summary(Dev d, int* flags, int cg) {
  __shared__ int f[3];
  if (threadIdx.x < 3) f[threadIdx.x] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < d.n_inst; i += blockDim.x) {
    const Ctl& c = d.ctl[i];
    if (c.status == ST_RUNNING) atomicOr(&f[0], 1);
    if (c.need_factor) atomicOr(&f[1], 1);
    if (cg ? c.cg_active : c.ls_active) atomicOr(&f[2], 1);
  }
  __syncthreads();
  if (threadIdx.x < 3) flags[threadIdx.x] = f[threadIdx.x];
}

}  // namespace nmpc
