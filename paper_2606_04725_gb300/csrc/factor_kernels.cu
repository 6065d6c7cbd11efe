// Numeric supernodal factorization (eq. cholesky-numeric, Sec. 3.2.3) and the
// permuted triangular solves (eqs. cholesky-lower/upper), level by level over
// the supernodal elimination tree computed once on the host.
//
// The factor is computed in the square-root-free form K = L D L^T (L unit
// lower triangular, D = diag(d_j)), which is the Cholesky factor L_c = L D^{1/2}
// written differently: the pivots d_j equal L_c,jj^2, so the inertia test of
// eq. infiniteOCP-inertia is unchanged, and the triangular solves need no
// divisions.  On this GPU an FP64 square root or division costs hundreds of
// cycles on the critical path of every column; a reciprocal costs three
// dependent FMAs after a hardware seed.
//
// Storage: each supernode's panel is m x c column-major; its diagonal holds
// 1/d_j, the entries below it hold L_ij.
//
// Multifrontal form: supernode J owns a frontal matrix whose first c_J
// columns are its factor panel and whose trailing (m_J - c_J)^2 block is the
// update matrix U_J passed to the parent.  A front is assembled from the
// condensed-matrix values already scattered into the panel plus the
// children's update matrices (extend-add in ascending child order, so the
// result is deterministic), then partially factored.  A non-positive or
// non-finite pivot flags the instance for inertia correction.
#include <cooperative_groups.h>

#include "kernels.h"

namespace nmpc {

extern __shared__ __align__(16) double dsm[];  // 16-byte aligned: bulk-copy destination

constexpr unsigned FULL = 0xffffffffu;

// Copy a front descriptor into shared memory (one round of loads by the
// first threads of the block); the caller synchronizes before reading it.
__device__ __forceinline__ void load_desc(FrontDesc* dst, const FrontDesc* src) {
  static_assert(sizeof(FrontDesc) % 8 == 0, "descriptor size");
  const long long* a = reinterpret_cast<const long long*>(src);
  long long* b = reinterpret_cast<long long*>(dst);
  for (int t = threadIdx.x; t < (int)(sizeof(FrontDesc) / 8); t += blockDim.x) b[t] = a[t];
}

// Child k of a front: size of its update matrix/vector and where they live.
struct ChildRef {
  int mc;
  const int* rel;
  const double* U;
  const double* uv;
};
__device__ __forceinline__ ChildRef child_ref(const SnDev& s, const FrontDesc& fd, int k) {
  if (k < DESC_CH) return {fd.ch_mc[k], s.sn_rel + fd.ch_relptr[k], s.U + fd.ch_Uptr[k], s.uv + fd.ch_uvptr[k]};
  const int C = s.sn_child[s.sn_child_ptr[fd.J] + k];
  return {s.sn_nrow[C] - s.sn_ncol[C], s.sn_rel + s.sn_relptr[C], s.U + s.sn_Uptr[C], s.uv + s.sn_uvptr[C]};
}

// Column index kk of flat position t in the column-major lower triangle of
// an nn x nn matrix (column kk holds nn - kk entries, starting at
// kk*nn - kk*(kk-1)/2).  Single-precision square root plus an exact integer
// correction, so no FP64 work is spent on index arithmetic.
__device__ __forceinline__ int tri_col(int t, int nn) {
  const float b = 2.0f * nn + 1.0f;
  int kk = (int)((b - sqrtf(b * b - 8.0f * (float)t)) * 0.5f);
  kk = max(0, min(kk, nn - 1));
  while (kk > 0 && kk * nn - kk * (kk - 1) / 2 > t) --kk;
  while (kk + 1 < nn && (kk + 1) * nn - (kk + 1) * kk / 2 <= t) ++kk;
  return kk;
}


// A pivot counts as positive only if it exceeds thr = pivtol * |K_jj| (K_jj
// the assembled diagonal): a pivot at rounding level is a zero eigenvalue,
// the wrong inertia of eq. infiniteOCP-inertia (which requires n_0 = 0).
// Compared on the bit patterns (thr >= 0, and non-negative doubles order like
// their bit patterns): p > thr, and p finite.  Integer work keeps the test off
// the FP64 pipe, whose every instruction costs tens of cycles on this GPU.
__device__ __forceinline__ bool pivot_ok(double p, double thr) {
  const long long pb = __double_as_longlong(p), tb = __double_as_longlong(thr);
  return pb > tb && pb < 0x7ff0000000000000LL;
}

__device__ __forceinline__ void flag_fail(Ctl* ctl) { *(volatile int*)&ctl->factor_fail = 1; }

// ---------------------------------------------------------------------------
// Single-CTA front factorization (fallback when the cluster kernel's shared
// memory does not fit, or when selected by option).  Right-looking, one
// column at a time: pivot, reciprocal, scaled column, rank-1 update of the
// trailing lower triangle with the unscaled column kept aside.
// ---------------------------------------------------------------------------
__device__ void factor_front_smem(Ctl* ctl, double* F, int m, int c, double* wcol, const double* kd, double pivtol) {
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ double inv_s;
  for (int j = 0; j < c; ++j) {
    double* colj = F + (size_t)j * m;
    if (tid == 0) {
      double p = colj[j];
      if (!pivot_ok(p, pivtol * fabs(kd[j]))) { flag_fail(ctl); p = 1.0; }
      inv_s = recip_nr(p);
      colj[j] = inv_s;
    }
    __syncthreads();
    const double inv = inv_s;
    for (int i = j + 1 + tid; i < m; i += nt) {
      const double w = colj[i];
      wcol[i] = w;
      colj[i] = w * inv;
    }
    __syncthreads();
    const int nn = m - j - 1;
    const int tot = nn * (nn + 1) / 2;
    for (int t = tid; t < tot; t += nt) {
      const int kk = tri_col(t, nn);
      const int ii = kk + (t - (kk * nn - kk * (kk - 1) / 2));
      const int k = j + 1 + kk, i = j + 1 + ii;
      F[i + (size_t)k * m] = fma(-colj[i], wcol[k], F[i + (size_t)k * m]);
    }
    __syncthreads();
  }
}

__global__ void k_factor_level(Dev d, SnDev s, const FrontDesc* dl, int smem_cap) {
  __shared__ FrontDesc fd;
  load_desc(&fd, dl + blockIdx.x);
  __syncthreads();
  Ctl* ctl = d.ctl + fd.inst;
  if (!ctl->need_factor) return;
  const int m = fd.m, c = fd.c, mu = m - c;
  double* Lp = s.L + fd.Lptr;
  double* Up = s.U + fd.Uptr;
  const double* kd = s.Kdiag + fd.first;
  const int tid = threadIdx.x, nt = blockDim.x;
  if ((long long)m * m + m <= smem_cap) {
    // ---- whole front in shared memory
    double* F = dsm;
    double* wcol = dsm + (size_t)m * m;
    for (int t = tid; t < m * c; t += nt) F[t] = Lp[t];
    for (int t = m * c + tid; t < m * m; t += nt) F[t] = 0.0;
    __syncthreads();
    for (int q = 0; q < fd.nchild; ++q) {
      const ChildRef ch = child_ref(s, fd, q);
      const int mc = ch.mc;
      const int* rel = ch.rel;
      const double* UC = ch.U;
      const int tot = mc * (mc + 1) / 2;
      for (int t = tid; t < tot; t += nt) {
        const int b = tri_col(t, mc);
        const int a = b + (t - (b * mc - b * (b - 1) / 2));
        F[rel[a] + (size_t)rel[b] * m] += UC[a + (size_t)b * mc];
      }
      __syncthreads();
    }
    factor_front_smem(ctl, F, m, c, wcol, kd, s.pivtol);
    for (int t = tid; t < m * c; t += nt) Lp[t] = F[t];
    for (int t = tid; t < mu * mu; t += nt) {
      const int a = t % mu, b = t / mu;
      Up[t] = F[(c + a) + (size_t)(c + b) * m];
    }
    return;
  }
  // ---- large front: panel in the factor array, update matrix in scratch,
  // unscaled pivot column in shared memory (m doubles)
  double* F = Lp;  // m x c, ld m
  double* G = Up;  // mu x mu, ld mu
  double* wcol = dsm;
  for (int t = tid; t < mu * mu; t += nt) G[t] = 0.0;
  __syncthreads();
  for (int q = 0; q < fd.nchild; ++q) {
    const ChildRef ch = child_ref(s, fd, q);
    const int mc = ch.mc;
    const int* rel = ch.rel;
    const double* UC = ch.U;
    const int tot = mc * (mc + 1) / 2;
    for (int t = tid; t < tot; t += nt) {
      const int b = tri_col(t, mc);
      const int a = b + (t - (b * mc - b * (b - 1) / 2));
      const int ra = rel[a], rb = rel[b];
      const double v = UC[a + (size_t)b * mc];
      if (rb < c) F[ra + (size_t)rb * m] += v;
      else G[(ra - c) + (size_t)(rb - c) * mu] += v;
    }
    __syncthreads();
  }
  __shared__ double invg;
  for (int j = 0; j < c; ++j) {
    double* colj = F + (size_t)j * m;
    if (tid == 0) {
      double dj = colj[j];
      if (!pivot_ok(dj, s.pivtol * fabs(kd[j]))) { flag_fail(ctl); dj = 1.0; }
      invg = recip_nr(dj);
      colj[j] = invg;
    }
    __syncthreads();
    const double inv = invg;
    for (int i = j + 1 + tid; i < m; i += nt) {
      const double w = colj[i];
      wcol[i] = w;
      colj[i] = w * inv;
    }
    __syncthreads();
    const int nn = m - j - 1;
    const int tot = nn * (nn + 1) / 2;
    for (int t = tid; t < tot; t += nt) {
      const int kk = tri_col(t, nn);
      const int ii = kk + (t - (kk * nn - kk * (kk - 1) / 2));
      const int i = j + 1 + ii, k = j + 1 + kk;
      if (k < c) F[i + (size_t)k * m] = fma(-colj[i], wcol[k], F[i + (size_t)k * m]);
      else G[(i - c) + (size_t)(k - c) * mu] = fma(-colj[i], wcol[k], G[(i - c) + (size_t)(k - c) * mu]);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Cluster-cooperative front factorization (blocked, right-looking, LDL^T).
//
// Cost model behind the layout: on this GPU an FP64 warp instruction keeps
// its SM sub-partition's FP64 unit busy for about 64 cycles whether one lane
// or all 32 are active, and a warp's FP64 instructions do not overlap.  So
// the pivot chain must use as few FP64 instructions per column as possible,
// run in a warp of its own sub-partition, and every other FP64 instruction
// should keep all lanes busy on the other sub-partitions.
//
// One thread-block cluster of Q CTAs factors one front.  Columns are dealt to
// the CTAs block-cyclically in blocks of PB = 8 columns (block b -> CTA b % Q);
// every CTA holds all m rows of its own columns in shared memory.  Pivot
// panel P (columns jb = P*PB .. jb + w - 1) is factored by its owner
// (panel_factor):
//   phase 1, in parallel on different sub-partitions:
//     warp 0: applies the previous panel to the PB x PB diagonal block (one
//       lane per lower-triangle entry: 28 entries of columns 1..7 in warp 0,
//       the 8 entries of column 0 by warp 1), then runs the pivot chain: per
//       column a shuffle of the pivot, its reciprocal (recip_nr: a seed and
//       three FMAs), and one multiply and one FMA that update every remaining
//       entry of the block at once -- five FP64 instructions per column, of
//       which four are on the chain (the product of the two column entries is
//       formed while the reciprocal is computed);
//     warps 1-3, 5-7: apply the previous panel to the rows below the block;
//   phase 2: every row below the pivot block is solved against it (w-step
//     forward substitution, one row per thread).
// The scaled panel L (diagonal 1/d_j) and the unscaled panel W = L D go to
// global memory (the factor and a scratch copy); a per-CTA counter, written
// with release semantics at cluster scope after a block barrier, tells the
// other CTAs that panel P is ready, and they read it from L2.  Every CTA
// applies each published panel to its own columns (F_ik -= sum_j L_ij W_kj).
// Lookahead: the owner of panel p+1 factors it right after reading panel p
// and only then updates its other columns, so the pivot chain never waits for
// the bulk update.  Waits are bounded (spin_limit polls); a wait that runs out
// sets the instance's factor-failure flag and the workspace timeout flag, and
// the kernel runs to completion on whatever data it has.
// ---------------------------------------------------------------------------
constexpr int PB = 8;

__device__ __forceinline__ int ld_acquire_cluster(const int* p) {
  int v;
  asm volatile("ld.acquire.cluster.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_cluster(int* p, int v) {
  asm volatile("st.release.cluster.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Hand-off of single values between warps of a CTA without fences: a slot
// holds SENTINEL (a signaling NaN, which no arithmetic produces: arithmetic
// results are quiet NaNs at worst) until its value is stored; one 64-bit
// store publishes the value together with its readiness.
constexpr long long SENTINEL = 0x7ff4deadbeef0001LL;
__device__ __forceinline__ double take(const double* slot, long long limit, int* timeout) {
  const volatile double* v = slot;
  double x = *v;
  long long it = 0;
  while (__double_as_longlong(x) == SENTINEL) {
    if (++it > limit) {
      *(volatile int*)timeout = 1;
      break;
    }
    x = *v;
  }
  return x;
}

__device__ __forceinline__ void bar_pair() { asm volatile("bar.sync 1, 64;" ::: "memory"); }  // warps 0 and 1

// Fl[i + lc*m] -= sum_{jj<w} Pl[i + jj*m] * Pw[k + jj*m] for own columns
// k in [kb, ke) (local column lc0 + k - kb) and rows i in [k, m), by the
// threads tid = 0 .. nt-1 of the caller's group (by default the block).
__device__ __forceinline__ void rank_update(double* Fl, const double* Pl, const double* Pw, int m, int w,
                                            int kb, int ke, int lc0, int tid = threadIdx.x,
                                            int nt = blockDim.x) {
  const int rows = m - kb;
  const int cols = ke - kb;
  for (int t = tid; t < rows * cols; t += nt) {
    const int kk = t / rows;
    const int i = kb + (t - kk * rows);
    const int k = kb + kk;
    if (i < k) continue;
    double* f = Fl + i + (size_t)(lc0 + kk) * m;
    double acc = *f;
#pragma unroll
    for (int jj = 0; jj < PB; ++jj)
      if (jj < w) acc = fma(-Pl[i + (size_t)jj * m], Pw[k + (size_t)jj * m], acc);
    *f = acc;
  }
}

// slot-A lane of diagonal-block entry (r, k), 1 <= k <= r <= 7
__device__ __forceinline__ int tri_lane(int r, int k) { return r * (r - 1) / 2 + k - 1; }

// Factor pivot panel of this CTA: block columns jb .. kend-1 (pivots
// jb .. jb+w-1) at local columns lc0 ..; the previous panel (Pl, Pw, width
// wprev; wprev = 0 for none) is applied to the block first.  Expects 256
// threads: warp 0 runs the pivot chain; NB = 192: warps 1-3 and 5-7 (the
// other three sub-partitions) do the bulk work and warp 4 idles, so that no
// bulk FP64 instruction of this CTA shares warp 0's sub-partition (the
// cluster kernel, one CTA per SM); NB = 224: warps 1-7 (the dataflow kernel,
// whose second CTA on the SM shares that sub-partition anyway: measured 1%
// faster there).
// Warp 0 publishes each finished pivot column (W of the diagonal block and
// 1/d_j) through the sentinel slots pub[j*PB + k] (pub[j*PB + j] = 1/d_j), so
// the rows below are solved one column behind the chain instead of after it.
constexpr int FCT = 256;
constexpr int NBULK = 192;       // threads of warps 1-3, 5-7
constexpr int NBULK_FLOW = 224;  // threads of warps 1-7

// Lg/Wg receive the panel's L and W: entry (i, jb + jj) at Lg[i + (jb + jj - gc0) m]
// and Wg[i + (jb + jj - gcw) m], i.e. 0 for a whole front's panel (in global
// memory, or in place in Fl), jb for an m x PB buffer that holds this panel only.  extra(bt) runs on the bulk
// threads (bt = 0 .. NB-1) while warp 0 runs the pivot chain, after the
// previous panel has been applied to this one: work that touches neither
// this panel's columns nor its buffers (the single-CTA front uses it for the
// previous panel's update of the other columns).
struct NoExtra {
  __device__ void operator()(int) const {}
};
template <int NB = NBULK, class Extra = NoExtra>
__device__ void panel_factor(Ctl* ctl, double* Fl, double* invd, const double* thr, double* Lg, double* Wg,
                             const double* Pl, const double* Pw, int wprev, int m, int jb, int w, int lc0,
                             double* sB, double* pub, int* s_timeout, long long limit, int gc0, int gcw,
                             Extra extra = Extra()) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  double* Fp = Fl + (size_t)lc0 * m;  // block column kk at Fp + kk*m
  const int kend = min(jb + PB, m), nb = kend - jb;
  if (warp == 0) {
    const int rA0 = 1 + (lane >= 1) + (lane >= 3) + (lane >= 6) + (lane >= 10) + (lane >= 15) + (lane >= 21);
    const bool inA = lane < 28;
    const int rA = inA ? rA0 : 7;
    const int kA = inA ? 1 + lane - (rA0 - 1) * rA0 / 2 : 7;
    const bool vA = inA && rA < nb;
    double a = vA ? Fp[(jb + rA) + (size_t)kA * m] : 0.0;
    for (int j = 0; j < wprev; ++j)
      if (vA) a = fma(-Pl[(jb + rA) + (size_t)j * m], Pw[(jb + kA) + (size_t)j * m], a);
    // rows of the block below the pivots are solved by the bulk warps: hand them over
    if (vA && rA >= w && kA < w) Fp[(jb + rA) + (size_t)kA * m] = a;
    bar_pair();  // column 0 of the block from warp 1
    const int rB = lane & 7;
    double b = (lane < nb) ? sB[lane] : 0.0;
    double inv[PB];
    bool bad = false;
#pragma unroll
    for (int jj = 0; jj < PB; ++jj) {
      inv[jj] = 0.0;
      if (jj < w) {
        // column jj of the diagonal block is final: publish it
        if (jj == 0) {
          if (lane < w) Fp[jb + lane] = b;
          if (lane > 0 && lane < w) pub[lane] = b;
        } else if (vA && kA == jj && rA < w) {
          Fp[(jb + rA) + (size_t)jj * m] = a;
          if (rA > jj) pub[jj * PB + rA] = a;
        }
        double x, y;
        if (jj == 0) {
          x = __shfl_sync(FULL, b, rA);
          y = __shfl_sync(FULL, b, kA);
        } else {
          x = __shfl_sync(FULL, a, tri_lane(max(rA, jj), jj));
          y = __shfl_sync(FULL, a, tri_lane(max(kA, jj), jj));
        }
        const double p = (jj == 0) ? __shfl_sync(FULL, b, 0) : __shfl_sync(FULL, a, tri_lane(jj, jj));
        const double xy = x * y;  // independent of the pivot: off the chain p -> 1/p -> next pivot
        const double iv = recip_nr(p);
        inv[jj] = iv;
        if (lane == 0) {
          bad = bad || !pivot_ok(p, thr[jj]);
          invd[jj] = iv;
          pub[jj * PB + jj] = iv;
        }
        if (vA && kA > jj && rA < w) a = fma(-xy, iv, a);
      }
    }
    // outputs of the pivot block: L and W to global memory, trailing block columns in place
    double ik = inv[1];
#pragma unroll
    for (int k = 2; k < PB; ++k)
      if (kA == k) ik = inv[k];
    if (vA && rA < w && kA < w) {
      Lg[(jb + rA) + (size_t)(jb + kA - gc0) * m] = (rA == kA) ? ik : a * ik;
      Wg[(jb + rA) + (size_t)(jb + kA - gcw) * m] = a;
    }
    if (vA && kA >= w) Fp[(jb + rA) + (size_t)kA * m] = a;
    if (lane < w) {
      Lg[(jb + rB) + (size_t)(jb - gc0) * m] = (rB == 0) ? inv[0] : b * inv[0];
      Wg[(jb + rB) + (size_t)(jb - gcw) * m] = b;
    }
    if (lane == 0 && bad) flag_fail(ctl);
  } else if (NB == FCT - 32 || (warp & 3) != 0) {
    static_assert(NB == FCT - 32 || NB == FCT - 64, "bulk warps: 1-7, or 1-3 and 5-7");
    const int bt = ((NB == FCT - 32 || warp < 4) ? warp - 1 : warp - 2) * 32 + lane;  // 0 .. NB-1
    if (warp == 1) {
      for (int t = lane; t < PB * PB; t += 32) pub[t] = __longlong_as_double(SENTINEL);
      // column 0 of the diagonal block: previous panel applied, handed to warp 0
      if (lane < nb) {
        double v = Fp[jb + lane];
        for (int j = 0; j < wprev; ++j) v = fma(-Pl[(jb + lane) + (size_t)j * m], Pw[jb + (size_t)j * m], v);
        sB[lane] = v;
        if (lane >= w) Fp[jb + lane] = v;
      }
      bar_pair();
    }
    if (wprev > 0) {
      // rows below the diagonal block: previous panel applied, one entry per thread
      const int rows = m - kend;
      for (int t = bt; t < rows * nb; t += NB) {
        const int kk = t / rows;
        const int i = kend + (t - kk * rows);
        double acc = Fp[i + (size_t)kk * m];
#pragma unroll
        for (int j = 0; j < PB; ++j)
          if (j < wprev) acc = fma(-Pl[i + (size_t)j * m], Pw[(jb + kk) + (size_t)j * m], acc);
        Fp[i + (size_t)kk * m] = acc;
      }
    }
    asm volatile("bar.sync 2, %0;" ::"r"(NB) : "memory");
    extra(bt);
    // rows below the pivot block, one column behind the chain:
    // l_ij = (F_ij - sum_{k<j} l_ik W_jk) / d_j
    for (int i = jb + w + bt; i < m; i += NB) {
      double f[PB];
#pragma unroll
      for (int k = 0; k < PB; ++k) f[k] = (k < w) ? Fp[i + (size_t)k * m] : 0.0;
#pragma unroll
      for (int jj = 0; jj < PB; ++jj) {
        if (jj < w) {
          const double lj = f[jj] * take(pub + jj * PB + jj, limit, s_timeout);
          Lg[i + (size_t)(jb + jj - gc0) * m] = lj;
          Wg[i + (size_t)(jb + jj - gcw) * m] = f[jj];
#pragma unroll
          for (int k = jj + 1; k < PB; ++k)
            if (k < w) f[k] = fma(-lj, take(pub + jj * PB + k, limit, s_timeout), f[k]);
        }
      }
    }
  }
  __syncthreads();
}

__global__ void k_factor_cluster(Dev d, SnDev s, const FrontDesc* dl) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int Q = (int)cluster.num_blocks();
  const int q = (int)cluster.block_rank();
  __shared__ FrontDesc fd;
  load_desc(&fd, dl + blockIdx.x / Q);
  __syncthreads();
  Ctl* ctl = d.ctl + fd.inst;
  if (!ctl->need_factor) return;  // uniform over the cluster: same instance
  const int m = fd.m, c = fd.c, mu = m - c;
  double* Lp = s.L + fd.Lptr;
  double* Wp = s.W + fd.Wptr;
  double* Up = s.U + fd.Uptr;
  const double* kd = s.Kdiag + fd.first;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nblk = (m + PB - 1) / PB;
  const int my_blocks = (nblk - q + Q - 1) / Q;  // blocks q, q+Q, ...
  const int ncl = my_blocks * PB;
  double* Pw = dsm;                          // m x PB: current panel, unscaled
  double* Pl = Pw + (size_t)m * PB;          // m x PB: current panel, scaled
  double* Fl = Pl + (size_t)m * PB;          // m x ncl, ld m: own columns
  double* thr = Fl + (size_t)m * ncl;        // ncl: pivot thresholds of own columns
  double* invd = thr + ncl;                  // ncl: 1/d of own pivot columns
  __shared__ int s_pub;                      // panels of this CTA published so far
  __shared__ int s_timeout;
  __shared__ double s_pubv[PB * PB];         // pivot columns of the current panel, published by warp 0
  __shared__ double sB[PB];
  // ---- assemble: own columns from the condensed values, then the children
  for (int t0 = tid; t0 < m * ncl; t0 += 4 * nt) {
    double v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = t0 + u * nt;
      const int i = t % m, lc = t / m;
      const int k = ((lc / PB) * Q + q) * PB + lc % PB;
      v[u] = (t < m * ncl && k < c) ? Lp[i + (size_t)k * m] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (t0 + u * nt < m * ncl) Fl[t0 + u * nt] = v[u];
  }
  for (int lc = tid; lc < ncl; lc += nt) {
    const int k = ((lc / PB) * Q + q) * PB + lc % PB;
    thr[lc] = (k < c) ? s.pivtol * fabs(kd[k]) : 0.0;
  }
  if (tid == 0) { s_pub = 0; s_timeout = 0; }
  __syncthreads();
  // children's update matrices through the precomputed extend-add map: this
  // CTA's entries only, four per thread in flight
  {
    const long long* ap = s.amap_ptr + fd.abase + (long long)q * (fd.nchild + 1);
    for (int k = 0; k < fd.nchild; ++k) {
      const double* UC = child_ref(s, fd, k).U;
      const long long b0 = ap[k], b1 = ap[k + 1];
      for (long long e0 = b0 + tid; e0 < b1; e0 += 4 * nt) {
        IdxPair pr[4];
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const long long e = e0 + (long long)u * nt;
          pr[u].dst = -1;
          if (e < b1) {
            pr[u] = s.amap[e];
            v[u] = UC[pr[u].src];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (pr[u].dst >= 0) Fl[pr[u].dst] += v[u];
      }
      __syncthreads();
    }
  }
  cluster.sync();  // every CTA assembled and initialized its counter
  const int npan = (c + PB - 1) / PB;
  const long long limit = s.spin_limit;
  if (q == 0 && npan > 0) {
    panel_factor(ctl, Fl, invd, thr, Lp, Wp, Pl, Pw, 0, m, 0, min(PB, c), 0, sB, s_pubv, &s_timeout, limit, 0, 0);
    if (tid == 0) st_release_cluster(&s_pub, 1);
  }
  for (int p = 0; p < npan; ++p) {
    const int jb = p * PB, w = min(PB, c - jb);
    const int owner = p % Q;
    // ---- wait for panel p, then read rows jb+w..m-1 of it from L2
    if (owner != q) {
      if (tid == 0) {
        const int* rp = cluster.map_shared_rank(&s_pub, owner);
        long long it = 0;
        while (!s_timeout && ld_acquire_cluster(rp) <= p / Q) {
          if (++it > limit) s_timeout = 1;
        }
      }
      __syncthreads();
    }
    {
      const int r0 = jb + w, rows = m - r0;
      for (int t0 = tid; t0 < rows * w; t0 += 2 * nt) {
        double vw[2], vl[2];
        int o[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int t = t0 + u * nt;
          o[u] = -1;
          if (t < rows * w) {
            const int jj = t / rows;
            const int i = r0 + (t - jj * rows);
            const size_t g = i + (size_t)(jb + jj) * m;
            vw[u] = __ldcg(Wp + g);
            vl[u] = __ldcg(Lp + g);
            o[u] = i + jj * m;
          }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
          if (o[u] >= 0) { Pw[o[u]] = vw[u]; Pl[o[u]] = vl[u]; }
      }
    }
    __syncthreads();
    // ---- lookahead: the owner of panel p+1 applies panel p to it and factors it
    const int nx = p + 1;
    const bool look = nx < npan && (nx % Q) == q;
    if (look) {
      const int k0 = nx * PB;
      panel_factor(ctl, Fl, invd + (nx / Q) * PB, thr + (nx / Q) * PB, Lp, Wp, Pl, Pw, w, m, k0,
                   min(PB, c - k0), (nx / Q) * PB, sB, s_pubv, &s_timeout, limit, 0, 0);
      if (tid == 0) st_release_cluster(&s_pub, nx / Q + 1);
    }
    // ---- rank-w update of the remaining own columns
    for (int lb = 0; lb < my_blocks; ++lb) {
      const int b = lb * Q + q;
      if (b < p || (look && b == nx)) continue;
      const int k0 = b * PB;
      const int ks = (b == p) ? jb + w : k0;  // the pivot block's own trailing columns
      const int ke = min(k0 + PB, m);
      if (ks >= ke) continue;
      rank_update(Fl, Pl, Pw, m, w, ks, ke, lb * PB + (ks - k0));
    }
    __syncthreads();
  }
  cluster.sync();  // no CTA may leave while others may still poll its counter
  if (tid == 0 && s_timeout) {
    flag_fail(ctl);
    atomicExch(s.timeout, 1);
  }
  // ---- write back the update-matrix columns (the factor panel is written as it is factored)
  for (int t = tid; t < m * ncl; t += nt) {
    const int i = t % m, lc = t / m;
    const int k = ((lc / PB) * Q + q) * PB + lc % PB;
    if (k < c || k >= m || i < c) continue;
    Up[(i - c) + (size_t)(k - c) * mu] = Fl[t];
  }
}

// ---------------------------------------------------------------------------
// Triangular solves with K = L D L^T, one thread block (4 warps) per
// supernode of a level.  Forward: L y = P b over the tree (children first),
// then z = D^{-1} y; backward: L^T x = z (parents first).
//
// The panel (m x c, contiguous, 16-byte aligned) is staged in shared memory
// by one bulk asynchronous copy (cp.async.bulk, completion on an mbarrier)
// while the right-hand side is gathered.
//
// Blocked by IB columns.  A column-by-column substitution puts one FP64 FMA
// and one hand-off between lanes (shuffle or shared memory) on the critical
// path of every column, about 285 cycles each on this GPU, so a 70-column
// triangle costs about 20k cycles.  Instead the panel is transformed once per
// factorization (k_diag_inv, k_panel_scale; in place): block K of columns
// s0 .. e-1 holds X_K = T_K^{-1} on its diagonal block (T_K = unit lower
// diagonal block of L) and M_K = L_{e..m-1,K} X_K below.  Then every block of
// a solve is ONE dense product (one reduction, one barrier):
//   forward   with v the right-hand side as updated by the blocks before K,
//             y_K = X_K v_K  and  v_r -= M_rK v_K  for r >= e, since
//             L_rK y_K = L_rK X_K v_K; the update rows r >= c come out as
//             u = v_{c..m-1};
//   backward  (last block first) x_K = X_K^T z_K - M_K^T x_{e..m-1}, the
//             rows below e being the blocks already solved and the
//             ancestors' x, since L_{e..,K}^T x = X_K^{-T} M_K^T x.
// ---------------------------------------------------------------------------
constexpr int ST = 128;  // threads of a solve block

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// An mbarrier must be invalidated before its shared memory is used again
// (by this block or by the next block on the SM): every thread has passed its
// wait when this runs (the caller synchronizes first).
__device__ __forceinline__ void mbar_inval(unsigned long long* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Bound of a wait for this block's own bulk copy.  The copy completes by
// itself, so the wait does not take spin_limit (which bounds the waits on
// other blocks, and which a caller may set tiny to make those run out); this
// bound only guards against a copy that never lands.  Each poll is one
// mbarrier.try_wait, so the bound is well under a second on this GPU.
constexpr long long COPY_WAIT_LIMIT = 1LL << 24;

// bounded wait for phase 0 of the barrier; false if the limit ran out
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, long long limit) {
  unsigned done = 0;
  long long it = 0;
  do {
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_u32(bar))
        : "memory");
  } while (!done && ++it < limit);
  return done != 0;
}

// One thread's share of a dot product: sum over k = k0, k0 + g, ... < len of
// a(k) x(k).  Four terms per round, their loads issued together, two
// accumulators: the FP64 pipe, not load latency, sets the pace.
template <class A, class X>
__device__ __forceinline__ double dot_part(int k0, int len, int g, A a, X x) {
  double s0 = 0.0, s1 = 0.0;
  int k = k0;
  for (; k + 3 * g < len; k += 4 * g) {
    const double a0 = a(k), a1 = a(k + g), a2 = a(k + 2 * g), a3 = a(k + 3 * g);
    const double x0 = x(k), x1 = x(k + g), x2 = x(k + 2 * g), x3 = x(k + 3 * g);
    s0 = fma(a0, x0, s0);
    s1 = fma(a1, x1, s1);
    s0 = fma(a2, x2, s0);
    s1 = fma(a3, x3, s1);
  }
  for (; k < len; k += g) s0 = fma(a(k), x(k), s0);
  return s0 + s1;
}

// Threads per output for count outputs: the largest power of two g with
// g * count <= the block's threads, at most 32 and at most len rounded up.
__device__ __forceinline__ int dot_group(int count, int len, int nt) {
  int g = 1;
  while (g < 32 && g < len && 2 * g * count <= nt) g *= 2;
  return g;
}

// sum over g consecutive lanes (g a power of two; every lane of the warp calls)
__device__ __forceinline__ double group_sum(double v, int g) {
  for (int off = g >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
  return v;
}

// count dot products over the block, out_o = sum_{k < len} a(o, k) x(k), with
// dot_group threads per output; emit(o, out_o) runs on one thread per output.
// Threads past the last output compute with o clamped (every address a(o, k)
// reads stays in range) and emit nothing.  Every thread of the block calls.
template <class A, class X, class E>
__device__ __forceinline__ void block_dots(int count, int len, A a, X x, E emit) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int g = dot_group(count, len, nt);
  for (int o0 = 0; o0 < count; o0 += nt / g) {
    const int o = o0 + tid / g, part = tid & (g - 1);
    const int oc = min(o, count - 1);
    double acc = dot_part(part, len, g, [&](int k) { return a(oc, k); }, x);
    acc = group_sum(acc, g);
    if (part == 0 && o < count) emit(o, acc);
  }
}

// Column substitution on the untransformed panel (SnDev::solve_form 0, for
// throughput-bound solves: the least FP64 work, no transform).  The c x c
// unit triangle is a pipeline over the four warps: warp w holds rows
// 32w .. 32w+31 of the vector in registers and applies the columns in order;
// the warp that owns column j takes y_j from its own lane by a shuffle and
// stores it into its sentinel slot (slots[j]), from which the other warps
// take it.  Beyond 128 columns, or with the panel in global memory, one warp
// substitutes column by column.  The slots hold SENTINEL on entry.
__device__ void subst_lower(double* v, double* slots, const double* Ls, int m, int c, bool stage, const SnDev& s,
                            int* s_to) {
  const int tid = threadIdx.x, wp = tid >> 5, lane = tid & 31;
  if (stage && c <= ST) {
    if (32 * wp < c) {
      const int r = 32 * wp + lane;
      double x = (r < c) ? v[r] : 0.0;
      const int jmax = min(c, 32 * wp + 32);
      for (int j = 0; j < jmax; ++j) {
        const double lv = (r > j && r < c) ? Ls[r + (size_t)j * m] : 0.0;
        double yj;
        if (j < 32 * wp) {
          yj = take(slots + j, s.spin_limit, s_to);
        } else {
          yj = __shfl_sync(FULL, x, j & 31);
          if (lane == (j & 31)) *(volatile double*)(slots + j) = yj;
        }
        x = fma(-lv, yj, x);
      }
      if (r < c) v[r] = x;
    }
  } else if (tid < 32) {
    for (int j = 0; j < c; ++j) {
      const double yj = v[j];
      __syncwarp();
      for (int i = j + 1 + lane; i < c; i += 32) v[i] = fma(-Ls[i + (size_t)j * m], yj, v[i]);
      __syncwarp();
    }
  }
  __syncthreads();
}

// L_cc^T x = t in place, the last column first (same scheme as subst_lower)
__device__ void subst_upper(double* v, double* slots, const double* Ls, int m, int c, bool stage, const SnDev& s,
                            int* s_to) {
  const int tid = threadIdx.x, wp = tid >> 5, lane = tid & 31;
  if (stage && c <= ST) {
    if (32 * wp < c) {
      const int i = 32 * wp + lane;
      double x = (i < c) ? v[i] : 0.0;
      const int top = min(c, 32 * wp + 32) - 1;  // highest row of this warp
      for (int j = c - 1; j >= 32 * wp; --j) {
        const double lv = (i < j) ? Ls[j + (size_t)i * m] : 0.0;  // L(j, i)
        double xj;
        if (j > top) {
          xj = take(slots + j, s.spin_limit, s_to);
        } else {
          xj = __shfl_sync(FULL, x, j & 31);
          if (lane == (j & 31)) *(volatile double*)(slots + j) = xj;
        }
        x = fma(-lv, xj, x);
      }
      if (i < c) v[i] = x;
    }
  } else if (tid < 32) {
    for (int j = c - 1; j >= 0; --j) {
      const double xj = v[j];
      __syncwarp();
      for (int i = lane; i < j; i += 32) v[i] = fma(-Ls[j + (size_t)i * m], xj, v[i]);
      __syncwarp();
    }
  }
  __syncthreads();
}

// Forward solve of one front (all threads of the block).  The panel copy and
// the front's own right-hand side are started first; wait() (every thread
// calls it; it ends with a block barrier) then waits for the children, whose
// update vectors, written by other blocks of the same launch, are read
// through L2 (__ldcg).
template <class Wait>
__device__ bool fwd_front(const Dev& d, const SnDev& s, const FrontDesc& fd, int smem_cap, unsigned long long* bar,
                          int* s_to, int* s_lost, Wait wait) {
  const int m = fd.m, c = fd.c, first = fd.first;
  const double* Lg = s.L + fd.Lptr;
  const long long lsz = ((long long)m * c + 1) & ~1LL;
  const bool stage = lsz + m + c <= smem_cap;
  // a panel too large to stage: column substitution still stages its c x c
  // triangle (ld c) when that fits, and reads the rows below from global memory
  const long long tsz = ((long long)c * c + 1) & ~1LL;
  const bool tri = !stage && s.solve_form == 0 && c <= ST && tsz + m + c <= smem_cap;
  double* fv = dsm + (stage ? lsz : (tri ? tsz : 0));  // m: right-hand side, updated block by block
  double* ys = fv + m;                                 // c: y
  const double* Ls = stage ? dsm : Lg;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tri)
    for (int t = tid; t < c * c; t += nt) {
      const int j = t / c, i = t - j * c;
      dsm[t] = Lg[i + (size_t)j * m];
    }
  if (tid == 0 && stage) {
    // earlier generic accesses to this shared memory (a previous front of
    // this block) are ordered before the asynchronous copy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_init(bar);
    bulk_load(dsm, Lg, (unsigned)(lsz * 8), bar);
  }
  for (int i = tid; i < m; i += nt) fv[i] = (i < c) ? d.b[first + i] : 0.0;
  if (s.solve_form == 0)
    for (int j = tid; j < c; j += nt) ys[j] = __longlong_as_double(SENTINEL);
  wait();
  // The first ST entries of each of the first DESC_CH children's update
  // vectors are loaded in one round (one L2 latency); the additions then go
  // child by child, in ascending order.
  double cv[DESC_CH];
  int cr[DESC_CH];
#pragma unroll
  for (int q = 0; q < DESC_CH; ++q) {
    cr[q] = -1;
    cv[q] = 0.0;
    if (q < fd.nchild && tid < fd.ch_mc[q]) {
      cr[q] = s.sn_rel[fd.ch_relptr[q] + tid];
      cv[q] = __ldcg(s.uv + fd.ch_uvptr[q] + tid);
    }
  }
#pragma unroll
  for (int q = 0; q < DESC_CH; ++q) {
    if (q < fd.nchild) {  // uniform over the block
      if (cr[q] >= 0) fv[cr[q]] += cv[q];
      const ChildRef ch = child_ref(s, fd, q);
      for (int a = nt + tid; a < ch.mc; a += nt) fv[ch.rel[a]] += __ldcg(ch.uv + a);
      __syncthreads();
    }
  }
  for (int q = DESC_CH; q < fd.nchild; ++q) {
    const ChildRef ch = child_ref(s, fd, q);
    for (int a = tid; a < ch.mc; a += nt) fv[ch.rel[a]] += __ldcg(ch.uv + a);
    __syncthreads();
  }
  if (stage && !mbar_wait(bar, COPY_WAIT_LIMIT)) *s_lost = 1;
  __syncthreads();
  // a copy that did not land may still write this shared memory: neither the
  // barrier nor the buffer is touched again, and the block leaves
  if (*s_lost) return false;  // uniform after the barrier
  if (stage && tid == 0) mbar_inval(bar);
  double* uvJ = s.uv + fd.uvptr;  // u_i = f_i - sum_j L_ij y_j (rows c..m-1)
  if (s.solve_form == 0) {
    if (tri) subst_lower(fv, ys, dsm, c, c, true, s, s_to);  // y in place of f_0..c-1
    else subst_lower(fv, ys, Ls, m, c, stage, s, s_to);
    block_dots(
        m - c, c, [&](int r, int j) { return Ls[(c + r) + (size_t)j * m]; }, [&](int j) { return fv[j]; },
        [&](int r, double a) { uvJ[r] = fv[c + r] - a; });
    for (int j = tid; j < c; j += nt) d.b[first + j] = fv[j] * Ls[j + (size_t)j * m];  // diagonal holds 1/d_j
    return true;
  }
  for (int s0 = 0; s0 < c; s0 += IB) {
    const int bk = min(IB, c - s0), e = s0 + bk;
    const double* P = Ls + s0 + (size_t)s0 * m;  // rows s0.. of the block's columns: X_K, then M_K or L
    const double* v = fv + s0;
    // P(r, j) with the unit diagonal of X_K and its zeros above the diagonal
    auto xk = [&](int r, int j) {
      const double p = P[r + (size_t)j * m];
      return j < r ? p : (j == r ? 1.0 : 0.0);
    };
    if (s.solve_form == 2) {
      // output r < bk: y_{s0+r} = sum_j X_rj v_j; r >= bk: v_{s0+r} -= sum_j M_rj v_j
      block_dots(m - s0, bk, xk, [&](int j) { return v[j]; }, [&](int r, double a) {
        if (r < bk) ys[s0 + r] = a;
        else fv[s0 + r] -= a;
      });
      __syncthreads();
    } else {
      block_dots(bk, bk, xk, [&](int j) { return v[j]; }, [&](int r, double a) { ys[s0 + r] = a; });
      __syncthreads();
      if (e < m) {  // v_r -= L_rK y_K for r >= e
        block_dots(
            m - e, bk, [&](int r, int j) { return P[(bk + r) + (size_t)j * m]; }, [&](int j) { return ys[s0 + j]; },
            [&](int r, double a) { fv[e + r] -= a; });
        __syncthreads();
      }
    }
  }
  for (int r = c + tid; r < m; r += nt) uvJ[r - c] = fv[r];
  for (int j = tid; j < c; j += nt) d.b[first + j] = ys[j] * Ls[j + (size_t)j * m];  // diagonal holds 1/d_j
  return true;
}

// Backward solve of one front.  The panel copy and z are started first;
// wait() (as in fwd_front) then waits for the parent, after which the
// ancestors' solution values (written by other blocks of the same launch)
// are read through L2.
template <class Wait>
__device__ bool bwd_front(const Dev& d, const SnDev& s, const FrontDesc& fd, int smem_cap, unsigned long long* bar,
                          int* s_to, int* s_lost, Wait wait) {
  const int m = fd.m, c = fd.c, first = fd.first;
  const double* Lg = s.L + fd.Lptr;
  const int* rows_idx = s.sn_rows + fd.rowptr;
  const long long lsz = ((long long)m * c + 1) & ~1LL;
  const bool stage = lsz + m + c <= smem_cap;
  const long long tsz = ((long long)c * c + 1) & ~1LL;  // staged triangle only (as in fwd_front)
  const bool tri = !stage && s.solve_form == 0 && c <= ST && tsz + m + c <= smem_cap;
  double* xv = dsm + (stage ? lsz : (tri ? tsz : 0));  // m: x (pivot rows solved block by block, ancestors' x below)
  double* zs = xv + m;                                 // c: z
  const double* Ls = stage ? dsm : Lg;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tri)
    for (int t = tid; t < c * c; t += nt) {
      const int j = t / c, i = t - j * c;
      dsm[t] = Lg[i + (size_t)j * m];
    }
  if (tid == 0 && stage) {
    // earlier generic accesses to this shared memory (a previous front of
    // this block) are ordered before the asynchronous copy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_init(bar);
    bulk_load(dsm, Lg, (unsigned)(lsz * 8), bar);
  }
  for (int i = tid; i < c; i += nt) zs[i] = d.b[first + i];
  wait();  // (also orders the barrier's initialization before any thread waits on it)
  for (int i = c + tid; i < m; i += nt) xv[i] = __ldcg(d.b + rows_idx[i]);
  if (stage && !mbar_wait(bar, COPY_WAIT_LIMIT)) *s_lost = 1;
  __syncthreads();
  if (*s_lost) return false;  // as in fwd_front
  if (stage && tid == 0) mbar_inval(bar);
  if (s.solve_form == 0) {
    // t_j = z_j - sum_{i >= c} L_ij x_i, then L_cc^T x = t (z's slots become the sentinel slots)
    block_dots(
        c, m - c, [&](int j, int i) { return Ls[(c + i) + (size_t)j * m]; }, [&](int i) { return xv[c + i]; },
        [&](int j, double a) { xv[j] = zs[j] - a; });
    __syncthreads();
    for (int j = tid; j < c; j += nt) zs[j] = __longlong_as_double(SENTINEL);
    __syncthreads();
    if (tri) subst_upper(xv, zs, dsm, c, c, true, s, s_to);
    else subst_upper(xv, zs, Ls, m, c, stage, s, s_to);
    for (int j = tid; j < c; j += nt) d.b[first + j] = xv[j];
    return true;
  }
  for (int s0 = (c - 1) / IB * IB; s0 >= 0; s0 -= IB) {
    const int bk = min(IB, c - s0), e = s0 + bk, len = m - s0;
    const double* P = Ls + s0 + (size_t)s0 * m;
    if (s.solve_form == 2) {
      // x_{s0+j} = sum_{j <= i < bk} X_ij z_{s0+i} - sum_{bk <= i < len} M_ij x_{s0+i}
      // (column j of P, contiguous); one group of g threads per output j
      const int g = dot_group(bk, len, nt);
      const int j = min(tid / g, bk - 1), part = tid & (g - 1);
      const double* Pj = P + (size_t)j * m;
      const double* z = zs + s0;
      const double* x = xv + s0;
      const double az = dot_part(
          part, bk, g,
          [&](int i) {
            const double p = Pj[i];
            return i > j ? p : (i == j ? 1.0 : 0.0);
          },
          [&](int i) { return z[i]; });
      const double ax = dot_part(bk + part, len, g, [&](int i) { return Pj[i]; }, [&](int i) { return x[i]; });
      const double acc = group_sum(az - ax, g);
      if (part == 0 && tid / g < bk) xv[s0 + j] = acc;
      __syncthreads();
    } else {
      if (e < m) {  // t_K = z_K - L_{e..,K}^T x_{e..}, in place of z_K
        block_dots(
            bk, m - e, [&](int j, int i) { return P[(bk + i) + (size_t)j * m]; }, [&](int i) { return xv[e + i]; },
            [&](int j, double a) { zs[s0 + j] -= a; });
        __syncthreads();
      }
      // x_K = X_K^T t_K
      block_dots(
          bk, bk,
          [&](int j, int i) {
            const double p = P[i + (size_t)j * m];
            return i > j ? p : (i == j ? 1.0 : 0.0);
          },
          [&](int i) { return zs[s0 + i]; }, [&](int j, double a) { xv[s0 + j] = a; });
      __syncthreads();
    }
  }
  for (int j = tid; j < c; j += nt) d.b[first + j] = xv[j];
  return true;
}

// In-place inverses of the unit lower triangular IB x IB diagonal blocks of
// the panels solved by fwd_front/bwd_front (one InvItem per block, one block
// of 256 threads per item), for the instances factored in this pass.  The
// block is staged in shared memory; warp w computes columns 2w and 2w+1 of
// X = T^{-1} (one per half-warp, lane i holding x_i) by substitution
// T x = e_k: x_i = 0 for i < k, x_k = 1, then for j = k, k+1, ...: x_j is
// final and x_i -= T_ij x_j for i > j (one FMA instruction per step, x_j
// shuffled from its lane).  Warp w starts at j = 2w, so the 8 warps issue
// 64 FMA instructions in all.
__global__ void __launch_bounds__(256) k_diag_inv(Dev d, SnDev s, int i0) {
  __shared__ double sT[IB * IB];
  const InvItem it = s.inv[i0 + blockIdx.x];
  if (!d.ctl[it.inst].need_factor) return;  // uniform over the block
  double* T = s.L + it.off;
  const int ld = it.ld, bk = it.bk, tid = threadIdx.x;
  {
    const int i = tid & (IB - 1), j = tid / IB;  // 256 threads = IB x IB entries
    sT[tid] = (i > j && i < bk) ? T[i + (size_t)j * ld] : 0.0;
  }
  __syncthreads();
  const int w = tid >> 5, lane = tid & 31, hf = lane >> 4, i = lane & 15;
  const int k = 2 * w + hf;
  double x = i == k ? 1.0 : 0.0;
  for (int j = 2 * w; j < IB - 1; ++j) {
    const double xj = __shfl_sync(FULL, x, (hf << 4) + j);
    if (i > j) x = fma(-sT[i + j * IB], xj, x);
  }
  if (i > k && i < bk) T[i + (size_t)k * ld] = x;
}

// M_K = L_{e..m-1,K} X_K in place, after k_diag_inv: one block of 128
// threads per ScaleUnit (32 rows of one block), X_K staged in shared memory,
// lane r of every warp holding row r of the slice.  Output column j,
// M_j = l_j + sum_{i>j} l_i X_ij, takes IB-1-j FMAs; warp w computes the
// columns w, IB-1-w, w+4, IB-5-w (30 FMAs for IB = 16, the same in every warp).
__global__ void __launch_bounds__(128) k_panel_scale(Dev d, SnDev s, int u0) {
  static_assert(IB == 16, "column split of k_panel_scale");
  __shared__ double sX[IB * IB];
  const ScaleUnit su = s.scale[u0 + blockIdx.x];
  const InvItem it = s.inv[su.item];
  if (!d.ctl[it.inst].need_factor) return;  // uniform over the block
  const int ld = it.ld, bk = it.bk, tid = threadIdx.x;
  const double* X = s.L + it.off;
  for (int t = tid; t < IB * IB; t += blockDim.x) {
    const int i = t & (IB - 1), j = t / IB;
    sX[t] = (i > j && i < bk) ? X[i + (size_t)j * ld] : 0.0;
  }
  const int rr = su.r0 + (tid & 31), w = tid >> 5;
  const bool act = rr < it.rows;
  double* B = s.L + it.off + bk + rr;  // L(e + rr, s0 + i) = B[i ld]
  double l[IB];
#pragma unroll
  for (int i = 0; i < IB; ++i) l[i] = (act && i < bk) ? B[(size_t)i * ld] : 0.0;
  __syncthreads();
  double out[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = (q == 0) ? w : (q == 1) ? IB - 1 - w : (q == 2) ? w + 4 : IB - 5 - w;
    double acc = l[0];  // l_j, selected without indexing registers by j
#pragma unroll
    for (int i = 1; i < IB; ++i) acc = (i == j) ? l[i] : acc;
#pragma unroll
    for (int i = 1; i < IB; ++i)
      if (i > j) acc = fma(l[i], sX[i + j * IB], acc);
    out[q] = acc;
  }
  // every warp has read its row's L before any column of it is overwritten
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = (q == 0) ? w : (q == 1) ? IB - 1 - w : (q == 2) ? w + 4 : IB - 5 - w;
    if (act && j < bk) B[(size_t)j * ld] = out[q];
  }
}

__global__ void __launch_bounds__(ST) k_fwd_level(Dev d, SnDev s, const FrontDesc* dl, int smem_cap) {
  __shared__ unsigned long long bar;
  __shared__ int s_to, s_lost;
  __shared__ FrontDesc fd;
  load_desc(&fd, dl + blockIdx.x);
  if (threadIdx.x == 0) s_to = s_lost = 0;
  __syncthreads();
  if (!solve_on(d.ctl[fd.inst])) return;
  fwd_front(d, s, fd, smem_cap, &bar, &s_to, &s_lost, [] { __syncthreads(); });
  if (threadIdx.x == 0 && (s_to || s_lost)) atomicExch(s.timeout, 1);
}

__global__ void __launch_bounds__(ST) k_bwd_level(Dev d, SnDev s, const FrontDesc* dl, int smem_cap) {
  __shared__ unsigned long long bar;
  __shared__ int s_to, s_lost;
  __shared__ FrontDesc fd;
  load_desc(&fd, dl + blockIdx.x);
  if (threadIdx.x == 0) s_to = s_lost = 0;
  __syncthreads();
  if (!solve_on(d.ctl[fd.inst])) return;
  bwd_front(d, s, fd, smem_cap, &bar, &s_to, &s_lost, [] { __syncthreads(); });
  if (threadIdx.x == 0 && (s_to || s_lost)) atomicExch(s.timeout, 1);
}

// Persistent forms: one launch for the fronts desc[0 .. nf) in level order.
// Each block claims the next front from a counter, waits for the fronts it
// depends on (forward: its children; backward: its parent, which waited for
// its own parent), solves it and publishes it with a release flag.  A front
// is waited on only after a running block has claimed it, so the launch
// needs no co-residency.  flags[0] is the claim counter, flags[1 + q] front
// q's completion and flags[nf + 1] counts the blocks that have left; the last
// block to leave zeroes all of them for the next launch (they start zeroed
// with the workspace).
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void wait_done(const int* flag, long long limit, int* s_to) {
  long long it = 0;
  while (ld_acquire_gpu(flag) == 0) {
    if (++it > limit) {
      *s_to = 1;
      break;
    }
  }
}

template <bool FWD>
__device__ void solve_persistent(const Dev& d, const SnDev& s, const FrontDesc* dl, int nf, int smem_cap, int* flags,
                                 const int* list, const int* count) {
  __shared__ unsigned long long bar;
  __shared__ int s_to, s_lost;
  __shared__ int s_q;
  __shared__ FrontDesc fd;
  const int tid = threadIdx.x;
  // Claims (thread 0 only).  With a list they run over its na fronts, in
  // level order (backward: parents first).  Fronts are claimed one ahead:
  // the next front's counter increment is issued when a front starts and its
  // list entry is read while the front waits for its dependencies, so
  // neither round trip stalls the block between fronts.  Holding a claimed
  // front not yet started forms no cycle of waits: the block first finishes
  // its current front, which waits only on fronts claimed before it.
  int na = nf, k_next = 0, q_next = -1;
  bool have_next = false;
  auto resolve = [&](int k) {
    if (k >= na) return -1;
    const int kk = FWD ? k : na - 1 - k;
    return list ? list[kk] : kk;
  };
  if (tid == 0) {
    s_to = s_lost = 0;
    if (list) na = *count;
    s_q = resolve(atomicAdd(flags, 1));
  }
  for (;;) {
    __syncthreads();
    if (s_q < 0) break;
    load_desc(&fd, dl + s_q);
    if (tid == 0) {
      k_next = atomicAdd(flags, 1);  // used only once the front waits
      have_next = false;
    }
    __syncthreads();
    if (solve_on(d.ctl[fd.inst])) {  // uniform over the block
      // started before the wait: the panel copy and the front's own values
      auto wait = [&] {
        if (tid == 0) {
          if (FWD) {
            for (int c = 0; c < fd.nchild; ++c) {
              const int cp = (c < DESC_CH) ? fd.ch_pos[c] : s.pos_of_sn[s.sn_child[s.sn_child_ptr[fd.J] + c]];
              if (cp >= 0 && cp < nf) wait_done(flags + 1 + cp, s.spin_limit, &s_to);
            }
          } else if (fd.par_pos >= 0 && fd.par_pos < nf) {
            wait_done(flags + 1 + fd.par_pos, s.spin_limit, &s_to);
          }
          q_next = resolve(k_next);
          have_next = true;
        }
        __syncthreads();
      };
      if (FWD) fwd_front(d, s, fd, smem_cap, &bar, &s_to, &s_lost, wait);
      else bwd_front(d, s, fd, smem_cap, &bar, &s_to, &s_lost, wait);
    }
    // Every thread's stores are ordered before thread 0's release store by
    // the block barrier (release is cumulative), and a waiting block reads
    // them after its acquire load and its own barrier.
    __syncthreads();
    if (tid == 0) {
      st_release_gpu(flags + 1 + fd.pos, 1);
      if (!have_next) q_next = resolve(k_next);
      s_q = q_next;
      // a panel copy that did not land may still write this block's shared
      // memory: the block starts no further front, and the front it has
      // claimed is released unsolved (the timeout flag reports the failure)
      // so that no block waits for it
      if (s_lost && q_next >= 0) st_release_gpu(flags + 1 + q_next, 1);
    }
    if (s_lost) break;  // uniform: set before the barrier above
  }
  if (tid == 0 && (s_to || s_lost)) atomicExch(s.timeout, 1);
  // no block touches the flags after it has arrived here
  __shared__ int s_last;
  if (tid == 0) s_last = atomicAdd(flags + nf + 1, 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (s_last) {
    if (list) {
      const int na = *count;
      for (int k = tid; k < na; k += blockDim.x) flags[1 + list[k]] = 0;
      if (tid == 0) { flags[0] = 0; flags[nf + 1] = 0; }
    } else {
      for (int i = tid; i < nf + 2; i += blockDim.x) flags[i] = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// Dataflow factorization: one persistent launch for the fronts desc[0 .. nf)
// of the leading levels, whose fronts fit one CTA's shared memory.  Each
// block claims the next front in level order, loads the front's pivot
// columns of the condensed matrix (no dependency), waits for its children's
// completion flags (bounded waits), adds their update matrices, factors the
// pivot columns with the panel scheme of the cluster kernel on one CTA
// (panels kept in shared memory, no publication), forms the update matrix
// in one dense pass, writes L and the update matrix and publishes the front
// with a release flag.  Levels no longer wait for one
// another: a front starts as soon as its own children are done, so fronts of
// different levels and instances overlap, and one launch replaces one launch
// per level.  As in the persistent solves a front is waited on only after a
// running block has claimed it (children come first in level order), so the
// launch needs no co-residency; flags[0] is the claim counter, flags[1 + q]
// front q's completion, flags[nf + 1] counts departed blocks, and the last
// block to leave zeroes them all for the next launch.
// Shared memory (doubles): the pivot columns (m x cp, cp = c rounded up to
// PB), the update block as a packed lower triangle (mu (mu + 1) / 2), L of
// the update rows (mu x c), the L buffers of two panels (m x PB each), cp
// pivot thresholds and cp reciprocal pivots -- about half of a whole front
// more, so that two blocks share an SM.
// ---------------------------------------------------------------------------
// The update matrix of a front factored by factor_front_flow:
// U = (children's part U0) - L21 D L21^T, all pivot columns at once, one
// TR x TC output tile per thread, the columns applied in ascending order: the
// same rounding as a panel-by-panel trailing update.  Fl: m x c pivot columns
// (W, ld m); Lu: L of the update rows (mu x c, ld mu), W times the reciprocal
// pivot as the panels formed it; Up: the children's part on entry and the
// update matrix on return (global memory, ld mu, lower triangle).
template <int TR, int TC>
__device__ __forceinline__ void schur_tiles(const double* Fl, const double* Lu, double* Up, int m, int c) {
  const int mu = m - c, tid = threadIdx.x, nt = blockDim.x;
  const int nr = (mu + TR - 1) / TR, ncb = (mu + TC - 1) / TC;
  // the tiles (ta, tb) that reach the lower triangle, TR ta + TR - 1 >= TC tb,
  // column block by column block: column block tb starts at row block lo(tb)
  auto lo = [&](int tb) { return max(0, (TC * tb - TR + 1 + TR - 1) / TR); };
  int total = 0;
  for (int tb = 0; tb < ncb; ++tb) total += nr - lo(tb);
  for (int t = tid; t < total; t += nt) {
    int tb = 0, r = t;
    while (r >= nr - lo(tb)) { r -= nr - lo(tb); ++tb; }
    const int ta = lo(tb) + r;
    const int a0 = TR * ta, b0 = TC * tb;
    double acc[TR][TC];
#pragma unroll
    for (int r = 0; r < TR; ++r)
#pragma unroll
      for (int q = 0; q < TC; ++q) {
        const int a = a0 + r, b = b0 + q;
        acc[r][q] = (a < mu && b <= a) ? Up[a + (size_t)b * mu] : 0.0;
      }
    const double* col = Fl + c;
    const double* lcol = Lu;
    for (int j = 0; j < c; ++j, col += m, lcol += mu) {
      double l[TR], wv[TC];
#pragma unroll
      for (int r = 0; r < TR; ++r) l[r] = (a0 + r < mu) ? lcol[a0 + r] : 0.0;
#pragma unroll
      for (int q = 0; q < TC; ++q) wv[q] = (b0 + q < mu) ? col[b0 + q] : 0.0;
#pragma unroll
      for (int r = 0; r < TR; ++r)
#pragma unroll
        for (int q = 0; q < TC; ++q) acc[r][q] = fma(-l[r], wv[q], acc[r][q]);
    }
#pragma unroll
    for (int r = 0; r < TR; ++r)
#pragma unroll
      for (int q = 0; q < TC; ++q) {
        const int a = a0 + r, b = b0 + q;
        if (a < mu && b <= a) Up[a + (size_t)b * mu] = acc[r][q];
      }
  }
}

// The largest tiles that still give every thread of the block an output
// tile (FP64 latency is hidden across warps, and larger tiles form fewer L
// values per multiply-add).
__device__ __noinline__ void schur_update(const double* Fl, double* Lu, const double* invd, double* Up, int m, int c) {
  const int mu = m - c, nt = blockDim.x;
  auto tiles = [&](int tr, int tc) {  // tiles reaching the lower triangle
    const int nr = (mu + tr - 1) / tr, ncb = (mu + tc - 1) / tc;
    int n = 0;
    for (int tb = 0; tb < ncb; ++tb) n += nr - max(0, (tc * tb) / tr);
    return n;
  };
  // L of the update rows, once: Lu(a, j) = W(c + a, j) / d_j
  for (int t = threadIdx.x; t < mu * c; t += nt) {
    const int j = t / mu, a = t - j * mu;
    Lu[t] = Fl[(c + a) + (size_t)j * m] * invd[j];
  }
  __syncthreads();
  if (tiles(4, 4) >= nt) schur_tiles<4, 4>(Fl, Lu, Up, m, c);
  else if (tiles(2, 4) >= nt) schur_tiles<2, 4>(Fl, Lu, Up, m, c);
  else schur_tiles<2, 2>(Fl, Lu, Up, m, c);
}

__device__ void factor_front_flow(Ctl* ctl, const SnDev& s, const FrontDesc& fd, const int* flags, int nf,
                                  int* s_to, double* s_pubv, double* sB, long long limit) {
  const int m = fd.m, c = fd.c, mu = m - c;
  double* Lp = s.L + fd.Lptr;
  double* Up = s.U + fd.Uptr;
  const double* kd = s.Kdiag + fd.first;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int cp = (c + PB - 1) / PB * PB, npan = cp / PB;
  // shared memory: the pivot columns, then the panel buffers of phase 1, whose
  // space L of the update rows takes in phase 2; the update block itself is
  // accumulated in its global matrix Up (L2-resident), which keeps a block
  // small enough for three per SM
  double* Fl = dsm;                                  // m x cp, ld m: the pivot columns (W once factored)
  double* Lb = Fl + (size_t)m * cp;                  // 2 x (m x PB): L of the even / odd panels (phase 1)
  double* Lu = Lb;                                   // mu x c: L of the update rows (phase 2)
  double* thr = Lb + ((size_t)mu * c > 2 * (size_t)m * PB ? (size_t)mu * c : 2 * (size_t)m * PB);  // cp
  double* invd = thr + cp;                           // cp
  auto bL = [&](int q) { return Lb + (size_t)(q & 1) * m * PB; };
  // ---- the pivot columns from the condensed values (m x c, ld m), the update block zero
  for (int t0 = tid; t0 < m * cp; t0 += 4 * nt) {
    double v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = t0 + u * nt;
      v[u] = (t < m * c) ? Lp[t] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (t0 + u * nt < m * cp) Fl[t0 + u * nt] = v[u];
  }
  for (int t = tid; t < mu * (mu + 1) / 2; t += nt) {  // the update block's lower triangle, zero
    const int b = tri_col(t, mu);
    const int a = b + (t - (b * mu - b * (b - 1) / 2));
    Up[a + (size_t)b * mu] = 0.0;
  }
  for (int k = tid; k < cp; k += nt) thr[k] = (k < c) ? s.pivtol * fabs(kd[k]) : 0.0;
  // ---- children: wait for their completion, then add their update matrices,
  // entries of a pivot column to Fl and the others to the update block
  // (ascending child order: the result does not depend on timing)
  if (tid == 0) {
    for (int k = 0; k < fd.nchild; ++k) {
      const int q = (k < DESC_CH) ? fd.ch_pos[k] : s.pos_of_sn[s.sn_child[s.sn_child_ptr[fd.J] + k]];
      if (q >= 0 && q < nf) wait_done(flags + 1 + q, limit, s_to);
    }
  }
  __syncthreads();
  for (int k = 0; k < fd.nchild; ++k) {
    const ChildRef ch = child_ref(s, fd, k);
    const int mc = ch.mc;
    const int tot = mc * (mc + 1) / 2;
    for (int t = tid; t < tot; t += nt) {
      const int b = tri_col(t, mc);
      const int a = b + (t - (b * mc - b * (b - 1) / 2));
      const int ra = ch.rel[a], rb = ch.rel[b];  // ra >= rb
      const double v = __ldcg(ch.U + a + (size_t)b * mc);  // written by another block
      if (rb < c) Fl[ra + (size_t)rb * m] += v;
      else Up[(ra - c) + (size_t)(rb - c) * mu] += v;  // this block's own matrix: plain accesses
    }
    __syncthreads();
  }
  // ---- phase 1: blocked right-looking LDL^T of the pivot columns only
  // (panel_factor; W of each panel in place in Fl, L in a panel buffer and
  // then in the factor), the panels' update of later pivot columns
  if (npan > 0)
    panel_factor<NBULK_FLOW>(ctl, Fl, invd, thr, bL(0), Fl, nullptr, nullptr, 0, m, 0, min(PB, c), 0, sB, s_pubv, s_to, limit,
                 0, 0);
  for (int p = 0; p < npan; ++p) {
    const int jb = p * PB, w = min(PB, c - jb);
    const double* Pl = bL(p);
    const double* Pw = Fl + (size_t)jb * m;  // W of panel p: Pw[k + jj m]
    const int nx = p + 1;
    // panel p's outputs, by threads (t0, nt0): its rows jb .. m-1 of L to the
    // factor, and its update of the later pivot columns except the lookahead
    // block nx (updated and factored by panel_factor)
    auto finish = [&](int t0, int nt0) {
      const int rows = m - jb;
      for (int t = t0; t < rows * w; t += nt0) {
        const int jj = t / rows, i = jb + (t - jj * rows);
        Lp[i + (size_t)(jb + jj) * m] = Pl[i + (size_t)jj * m];
      }
      for (int b = nx + 1; b < npan; ++b) {
        const int k0 = b * PB, ke = min(k0 + PB, c);
        if (k0 < ke) rank_update(Fl, Pl, Pw, m, w, k0, ke, k0, t0, nt0);
      }
    };
    if (nx < npan) {
      // lookahead: the next panel gets this panel's update and is factored,
      // while the bulk warps finish this panel (the chain does not wait for it)
      const int k0 = nx * PB;
      panel_factor<NBULK_FLOW>(ctl, Fl, invd + k0, thr + k0, bL(nx), Fl, Pl, Pw, w, m, k0, min(PB, c - k0), k0, sB,
                               s_pubv, s_to, limit, k0, 0, [&](int bt) { finish(bt, NBULK_FLOW); });
    } else {
      finish(tid, nt);
      __syncthreads();
    }
  }
  // ---- phase 2: the update matrix U = (children's part) - L21 D L21^T for
  // the parent (schur_update)
  schur_update(Fl, Lu, invd, Up, m, c);
}

__global__ void __launch_bounds__(FCT, 3) k_factor_flow(Dev d, SnDev s, const FrontDesc* dl, int nf, int* flags,
                                                          const int* list, const int* count) {
  __shared__ FrontDesc fd;
  __shared__ int s_q, s_to, s_any_to;
  __shared__ double s_pubv[PB * PB];
  __shared__ double sB[PB];
  const int tid = threadIdx.x;
  const long long limit = s.spin_limit;
  // Claims (thread 0 only), with a list over its na fronts (level order).
  // The next front's counter increment is issued when a front starts and
  // resolved when it ends, so the round trip overlaps the factorization;
  // holding a claimed front not yet started forms no cycle of waits (the
  // block first finishes its current front, which waits only on fronts
  // claimed before it).
  int na = nf, k_next = 0;
  auto resolve = [&](int k) { return k >= na ? -1 : (list ? list[k] : k); };
  if (tid == 0) {
    s_any_to = 0;
    if (list) na = *count;
    s_q = resolve(atomicAdd(flags, 1));
  }
  for (;;) {
    if (tid == 0) s_to = 0;
    __syncthreads();
    if (s_q < 0) break;
    load_desc(&fd, dl + s_q);
    if (tid == 0) k_next = atomicAdd(flags, 1);  // used only when this front ends
    __syncthreads();
    Ctl* ctl = d.ctl + fd.inst;
    if (ctl->need_factor) factor_front_flow(ctl, s, fd, flags, nf, &s_to, s_pubv, sB, limit);  // uniform
    // every thread's stores (L, U) are ordered before thread 0's release
    // store by the barrier (release is cumulative)
    __syncthreads();
    if (tid == 0) {
      if (s_to) {  // a wait ran out: this front is unusable, and the instance is flagged
        flag_fail(ctl);
        s_any_to = 1;
      }
      st_release_gpu(flags + 1 + fd.pos, 1);
      s_q = resolve(k_next);
    }
  }
  if (tid == 0 && s_any_to) atomicExch(s.timeout, 1);
  // no block touches the flags after it has arrived here
  __shared__ int s_last;
  if (tid == 0) s_last = atomicAdd(flags + nf + 1, 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (s_last) {
    if (list) {
      const int nl = *count;  // na is thread 0's
      for (int k = tid; k < nl; k += blockDim.x) flags[1 + list[k]] = 0;
      if (tid == 0) { flags[0] = 0; flags[nf + 1] = 0; }
    } else {
      for (int i = tid; i < nf + 2; i += blockDim.x) flags[i] = 0;
    }
  }
}

__global__ void __launch_bounds__(ST, 10) k_fwd_persist(Dev d, SnDev s, const FrontDesc* dl, int nf, int smem_cap,
                                                    int* flags, const int* list, const int* count) {
  solve_persistent<true>(d, s, dl, nf, smem_cap, flags, list, count);
}
__global__ void __launch_bounds__(ST, 12) k_bwd_persist(Dev d, SnDev s, const FrontDesc* dl, int nf, int smem_cap,
                                                    int* flags, const int* list, const int* count) {
  solve_persistent<false>(d, s, dl, nf, smem_cap, flags, list, count);
}

// The fronts q in [0, nf) (level order) whose instance takes part in the
// next persistent launch, in level order: list[0 .. *count).  Mode 0: the
// instance needs a factorization; 1: it is being solved.  In the last
// iterations of a batch most instances have stopped, and claiming their
// fronts one at a time costs more than the work left.  One block: a byte per
// instance in shared memory; warp w takes the contiguous fronts of segment w,
// 32 at a time (coalesced loads, a ballot each); a scan over the warps'
// counts gives each segment's offset, and a second pass writes the fronts in
// order, so the list keeps level order (children before parents).
__global__ void __launch_bounds__(FL_THREADS) k_front_list(Dev d, SnDev s, int nf, int mode, int* list, int* count) {
  extern __shared__ unsigned char s_on[];
  __shared__ int s_warp[FL_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr unsigned FULLM = 0xffffffffu;
  for (int i = tid; i < d.n_inst; i += FL_THREADS) {
    const Ctl& c = d.ctl[i];
    s_on[i] = (unsigned char)(mode == 0 ? c.need_factor != 0 : solve_on(c));
  }
  __syncthreads();
  constexpr int NW = FL_THREADS / 32;
  const int seg = (nf + NW * 32 - 1) / (NW * 32) * 32;  // fronts per warp, a multiple of 32
  const int w0 = min(nf, wid * seg), w1 = min(nf, w0 + seg);
  int cnt = 0;
#pragma unroll 4
  for (int b = w0; b < w1; b += 32) {
    const int q = b + lane;
    cnt += __popc(__ballot_sync(FULLM, q < w1 && s_on[s.front_inst[q]]));
  }
  if (lane == 0) s_warp[wid] = cnt;
  __syncthreads();
  if (wid == 0) {  // exclusive scan of the NW = 32 warps' counts
    const int v = s_warp[lane];
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULLM, x, o);
      if (lane >= o) x += y;
    }
    s_warp[lane] = x - v;
    if (lane == 31) *count = x;
  }
  __syncthreads();
  int at = s_warp[wid];
#pragma unroll 4
  for (int b = w0; b < w1; b += 32) {
    const int q = b + lane;
    const bool on = q < w1 && s_on[s.front_inst[q]];
    const unsigned bal = __ballot_sync(FULLM, on);
    if (on) list[at + __popc(bal & ((1u << lane) - 1u))] = q;
    at += __popc(bal);
  }
}

// ---------------------------------------------------------------------------
// Large fronts (blocked LDL^T over many SMs).
//
// Fronts too large for the shared memory of a cluster are factored in place:
// the front F is the factor panel (columns < c, leading dimension m) plus the
// update matrix (rows and columns >= c, leading dimension m - c).  All fronts
// of a level are processed together, panel by panel (BNB columns):
//   k_big_zero:   zero the update matrices;
//   k_big_extend: add child k's update matrix (one launch per child index, so
//                 the order of the additions is fixed);
//   k_big_diag:   factor the BNB x BNB diagonal block in one warp per front;
//   k_big_trsm:   solve the rows below it, one row per thread; both write L
//                 (1/d_j on the diagonal) to the panel, and the pivots d_j go
//                 to dpiv, from which W = L D is formed where it is needed;
//   k_big_update: F_ik -= sum_j L_ij W_kj over the trailing lower triangle,
//                 64 x 64 tiles, each thread a 4 x 4 block of FMAs with the
//                 panel's L and W rows staged in shared memory.
// ---------------------------------------------------------------------------
constexpr int BNB = 32;      // panel width
constexpr int BT = 64;       // update tile
constexpr int BROWS = 256;   // rows per panel block (one per thread)

__device__ __forceinline__ double* front_at(double* Lp, double* Up, int m, int c, int i, int k) {
  return (k < c) ? Lp + i + (size_t)k * m : Up + (i - c) + (size_t)(k - c) * (m - c);
}

__global__ void k_big_zero(Dev d, SnDev s, const FrontDesc* dl) {
  const FrontDesc& fd = dl[blockIdx.y];
  if (!d.ctl[fd.inst].need_factor) return;
  const long long mu = fd.m - fd.c, tot = mu * mu;
  double* Up = s.U + fd.Uptr;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x)
    Up[t] = 0.0;
}

__global__ void k_big_extend(Dev d, SnDev s, const FrontDesc* dl, int k) {
  const FrontDesc& fd = dl[blockIdx.y];
  if (k >= fd.nchild || !d.ctl[fd.inst].need_factor) return;
  const ChildRef ch = child_ref(s, fd, k);
  const int m = fd.m, c = fd.c, mc = ch.mc;
  double* Lp = s.L + fd.Lptr;
  double* Up = s.U + fd.Uptr;
  // column b of the child's update matrix per block row of threads; rows a >= b
  for (long long b = blockIdx.x; b < mc; b += gridDim.x) {
    const int rb = ch.rel[b];
    for (int a = (int)b + threadIdx.x; a < mc; a += blockDim.x)
      *front_at(Lp, Up, m, c, ch.rel[a], rb) += ch.U[a + b * (long long)mc];
  }
}

// Diagonal block of panel p, one warp per front (lane r = row jb + r): L and
// 1/d_j into the factor panel, W into the scratch copy.
__global__ void __launch_bounds__(32) k_big_diag(Dev d, SnDev s, const FrontDesc* dl, int p) {
  const FrontDesc& fd = dl[blockIdx.x];
  const int m = fd.m, c = fd.c;
  const int jb = p * BNB;
  if (jb >= c) return;
  Ctl* ctl = d.ctl + fd.inst;
  if (!ctl->need_factor) return;
  const int w = min(BNB, c - jb);
  double* Lp = s.L + fd.Lptr;
  double* dp = s.dpiv + fd.first;
  const double* kd = s.Kdiag + fd.first;
  const int lane = threadIdx.x;
  double f[BNB];
#pragma unroll
  for (int k = 0; k < BNB; ++k) f[k] = (lane < w && k <= lane) ? Lp[(jb + lane) + (size_t)(jb + k) * m] : 0.0;
  double inv[BNB];
  bool bad = false;
#pragma unroll
  for (int j = 0; j < BNB; ++j) {
    inv[j] = 0.0;
    if (j < w) {
      const double piv = __shfl_sync(FULL, f[j], j);
      const double iv = recip_nr(piv);
      inv[j] = iv;
      if (lane == 0) bad = bad || !pivot_ok(piv, s.pivtol * fabs(kd[jb + j]));
      const double lj = f[j] * iv;
#pragma unroll
      for (int k = j + 1; k < BNB; ++k) {
        const double wk = __shfl_sync(FULL, f[j], k);
        if (lane >= k && lane < w) f[k] = fma(-lj, wk, f[k]);
      }
    }
  }
  if (lane < w) {
#pragma unroll
    for (int k = 0; k < BNB; ++k)
      if (k <= lane) {
        const size_t g = (jb + lane) + (size_t)(jb + k) * m;
        Lp[g] = (k == lane) ? inv[k] : f[k] * inv[k];
      }
  }
  if (lane < w) dp[jb + lane] = f[lane];  // the pivot d_j (W = L D is formed from it where needed)
  if (lane == 0 && bad) flag_fail(ctl);
}

// Rows below the diagonal block of panel p, one per thread: a w-step forward
// substitution, l_ij = (F_ij - sum_{k<j} l_ik W_jk) / d_j.
__global__ void __launch_bounds__(BROWS) k_big_trsm(Dev d, SnDev s, const FrontDesc* dl, int p) {
  __shared__ double Db[BNB * BNB];  // W of the diagonal block, column-major
  __shared__ double inv[BNB];
  const FrontDesc& fd = dl[blockIdx.y];
  const int m = fd.m, c = fd.c;
  const int jb = p * BNB;
  if (jb >= c) return;
  if (!d.ctl[fd.inst].need_factor) return;
  const int w = min(BNB, c - jb);
  const int r0 = jb + w + blockIdx.x * BROWS;
  if (r0 >= m) return;
  double* Lp = s.L + fd.Lptr;
  const double* dp = s.dpiv + fd.first;
  const int tid = threadIdx.x;
  for (int t = tid; t < BNB * BNB; t += blockDim.x) {
    const int i = t % BNB, k = t / BNB;
    Db[t] = (i < w && k < i) ? Lp[(jb + i) + (size_t)(jb + k) * m] * dp[jb + k] : 0.0;  // W = L D
  }
  if (tid < w) inv[tid] = Lp[(jb + tid) + (size_t)(jb + tid) * m];
  __syncthreads();
  const int i = r0 + tid;
  if (i >= m) return;
  double f[BNB];
#pragma unroll
  for (int k = 0; k < BNB; ++k) f[k] = (k < w) ? Lp[i + (size_t)(jb + k) * m] : 0.0;
#pragma unroll
  for (int j = 0; j < BNB; ++j) {
    if (j < w) {
      const double lj = f[j] * inv[j];
      const size_t g = i + (size_t)(jb + j) * m;
      Lp[g] = lj;
#pragma unroll
      for (int k = j + 1; k < BNB; ++k)
        if (k < w) f[k] = fma(-lj, Db[k + j * BNB], f[k]);
    }
  }
}

// Trailing update after panel p: rows and columns >= jb + w.  Tile t of the
// lower triangle of tiles (bi >= bk); 256 threads, each a 4 x 4 block.
__global__ void __launch_bounds__(256) k_big_update(Dev d, SnDev s, const FrontDesc* dl, int p) {
  __shared__ double Ls[BT][BNB + 1];
  __shared__ double Ws[BT][BNB + 1];
  const FrontDesc& fd = dl[blockIdx.y];
  const int m = fd.m, c = fd.c;
  const int jb = p * BNB;
  if (jb >= c) return;
  if (!d.ctl[fd.inst].need_factor) return;
  const int w = min(BNB, c - jb);
  const int t0 = jb + w;  // first trailing row/column
  const int R = m - t0;
  const int nb = (R + BT - 1) / BT;
  const int tile = blockIdx.x;
  if (tile >= nb * (nb + 1) / 2) return;
  // tile -> (bi, bk), bi >= bk, column-major over the lower triangle of tiles
  const int bk = tri_col(tile, nb);
  const int bi = bk + (tile - (bk * nb - bk * (bk - 1) / 2));
  const int i0 = t0 + bi * BT, k0 = t0 + bk * BT;
  const double* Lp = s.L + fd.Lptr;
  const double* dp = s.dpiv + fd.first;
  double* Lw = s.L + fd.Lptr;
  double* Uw = s.U + fd.Uptr;
  const int tid = threadIdx.x;
  for (int t = tid; t < BT * BNB; t += blockDim.x) {
    const int r = t % BT, j = t / BT;
    const int ii = i0 + r, kk = k0 + r;
    Ls[r][j] = (j < w && ii < m) ? Lp[ii + (size_t)(jb + j) * m] : 0.0;
    Ws[r][j] = (j < w && kk < m) ? Lp[kk + (size_t)(jb + j) * m] * dp[jb + j] : 0.0;  // W = L D
  }
  __syncthreads();
  const int tr = (tid % 16) * 4, tc = (tid / 16) * 4;  // this thread's 4 x 4 block
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
#pragma unroll 4
  for (int j = 0; j < BNB; ++j) {
    double la[4], wb[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) la[a] = Ls[tr + a][j];
#pragma unroll
    for (int b = 0; b < 4; ++b) wb[b] = Ws[tc + b][j];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(la[a], wb[b], acc[a][b]);
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int kk = k0 + tc + b;
    if (kk >= m) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int ii = i0 + tr + a;
      if (ii >= m || ii < kk) continue;
      double* f = front_at(Lw, Uw, m, c, ii, kk);
      *f -= acc[a][b];
    }
  }
}

// Blocked solves of one large front in one block (1024 threads): the unit
// triangle BNB columns at a time in warp 0, the rows below by all threads.
// The front vector lives in shared memory when it fits (smem_doubles), else
// in the front's slot of a global scratch vector (offset: its row list).
// ---------------------------------------------------------------------------
// Solves of the large fronts, one launch sequence per level.  A single block
// per front would carry all of a front's FP64 work on one SM (m c FMAs each
// way: 53M for the 7296-row root of the g = 64 plate); instead the columns go
// in blocks of SBW, and per block
//   forward:  one CTA per front solves the block's unit lower triangle
//             (k_bigs_fwd_diag: 32-column sub-blocks by a warp's shuffle
//             chain, each followed by the rest of the block's rows), then a
//             grid of CTAs applies the block to every row below it
//             (k_bigs_fwd_rows: rows across lanes, the block's columns split
//             over the warps, coalesced reads of L);
//   backward: first the ancestors' rows for every column (k_bigs_bwd_anc:
//             a warp per column, rows across lanes), then, last block first,
//             one CTA per front solves the block's upper triangle
//             (k_bigs_bwd_diag) and a grid of CTAs applies it to every
//             column before it (k_bigs_bwd_cols: a warp per column).
// The front vector lives in global scratch (fvec), L2-resident between the
// launches.  k_bigs_*_pre and k_bigs_*_post gather the right-hand side and
// the children's update vectors, and write the outputs.
// ---------------------------------------------------------------------------
constexpr int SBW = BIG_SBW;  // column block of the large-front solves (128)
constexpr int SBT = BIG_SBT;  // threads per CTA (256)

__device__ __forceinline__ bool big_active(const Dev& d, const FrontDesc& fd) {
  return solve_on(d.ctl[fd.inst]);
}

// f = P b on the pivot rows, 0 below, plus the children's update vectors
__global__ void __launch_bounds__(SBT) k_bigs_fwd_pre(Dev d, SnDev s, const FrontDesc* dl) {
  const FrontDesc& fd = dl[blockIdx.x];
  if (!big_active(d, fd)) return;
  double* fv = s.fvec + fd.rowptr;
  const int m = fd.m, c = fd.c, tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < m; i += nt) fv[i] = (i < c) ? d.b[fd.first + i] : 0.0;
  __syncthreads();
  for (int q = 0; q < fd.nchild; ++q) {
    const ChildRef ch = child_ref(s, fd, q);
    for (int a = tid; a < ch.mc; a += nt) fv[ch.rel[a]] += ch.uv[a];
    __syncthreads();
  }
}

// unit lower triangle of columns jb .. jb+w-1, in place on f
__global__ void __launch_bounds__(SBT) k_bigs_fwd_diag(Dev d, SnDev s, const FrontDesc* dl, int jb) {
  const FrontDesc& fd = dl[blockIdx.x];
  if (!big_active(d, fd) || jb >= fd.c) return;
  const int m = fd.m, w = min(SBW, fd.c - jb), tid = threadIdx.x, nt = blockDim.x;
  double* fv = s.fvec + fd.rowptr;
  const double* Lb = s.L + fd.Lptr + jb + (size_t)jb * m;  // L(jb + r, jb + j) = Lb[r + j m]
  __shared__ double v[SBW];
  for (int t = tid; t < w; t += nt) v[t] = fv[jb + t];
  __syncthreads();
  for (int sb = 0; sb < w; sb += 32) {
    const int ws = min(32, w - sb);
    if (tid < 32) {
      double x = (tid < ws) ? v[sb + tid] : 0.0;
      for (int j = 0; j < ws; ++j) {
        const double yj = __shfl_sync(FULL, x, j);
        if (tid > j && tid < ws) x = fma(-Lb[(sb + tid) + (size_t)(sb + j) * m], yj, x);
      }
      if (tid < ws) v[sb + tid] = x;
    }
    __syncthreads();
    for (int r = sb + ws + tid; r < w; r += nt) {
      double a = v[r];
      for (int j = 0; j < ws; ++j) a = fma(-Lb[r + (size_t)(sb + j) * m], v[sb + j], a);
      v[r] = a;
    }
    __syncthreads();
  }
  for (int t = tid; t < w; t += nt) fv[jb + t] = v[t];
}

// f_r -= sum_{j < w} L(r, jb + j) y_{jb+j} for rows r >= jb + w: 64 rows per
// CTA across the lanes, the block's columns split over 4 groups of 2 warps
__global__ void __launch_bounds__(SBT) k_bigs_fwd_rows(Dev d, SnDev s, const FrontDesc* dl, int jb) {
  const FrontDesc& fd = dl[blockIdx.y];
  if (!big_active(d, fd) || jb >= fd.c) return;
  const int m = fd.m, w = min(SBW, fd.c - jb), r0 = jb + w;
  const int row0 = r0 + blockIdx.x * 64;
  if (row0 >= m) return;  // uniform over the CTA
  double* fv = s.fvec + fd.rowptr;
  const double* Lg = s.L + fd.Lptr;
  __shared__ double y[SBW];
  __shared__ double part[4][64];
  const int tid = threadIdx.x, rr = tid & 63, grp = tid >> 6;
  for (int t = tid; t < w; t += blockDim.x) y[t] = fv[jb + t];
  __syncthreads();
  const int r = row0 + rr;
  double a = 0.0;
  if (r < m)
    for (int j = grp; j < w; j += 4) a = fma(Lg[r + (size_t)(jb + j) * m], y[j], a);
  part[grp][rr] = a;
  __syncthreads();
  if (grp == 0 && r < m) fv[r] -= (part[0][rr] + part[1][rr]) + (part[2][rr] + part[3][rr]);
}

// outputs: update vector u (rows c..m-1) and z = D^{-1} y
__global__ void __launch_bounds__(SBT) k_bigs_fwd_post(Dev d, SnDev s, const FrontDesc* dl) {
  const FrontDesc& fd = dl[blockIdx.x];
  if (!big_active(d, fd)) return;
  const double* fv = s.fvec + fd.rowptr;
  const double* Lg = s.L + fd.Lptr;
  const int m = fd.m, c = fd.c, tid = threadIdx.x, nt = blockDim.x;
  double* uvJ = s.uv + fd.uvptr;
  for (int i = c + tid; i < m; i += nt) uvJ[i - c] = fv[i];
  for (int j = tid; j < c; j += nt) d.b[fd.first + j] = fv[j] * Lg[j + (size_t)j * m];  // diagonal holds 1/d_j
}

// x = z on the pivot rows, the ancestors' solution below
__global__ void __launch_bounds__(SBT) k_bigs_bwd_pre(Dev d, SnDev s, const FrontDesc* dl) {
  const FrontDesc& fd = dl[blockIdx.x];
  if (!big_active(d, fd)) return;
  double* xv = s.fvec + fd.rowptr;
  const int* rows_idx = s.sn_rows + fd.rowptr;
  for (int i = threadIdx.x; i < fd.m; i += blockDim.x) xv[i] = (i < fd.c) ? d.b[fd.first + i] : d.b[rows_idx[i]];
}

// t_j = z_j - sum_{i >= c} L_ij x_i: a warp per column j, rows across lanes
__global__ void __launch_bounds__(SBT) k_bigs_bwd_anc(Dev d, SnDev s, const FrontDesc* dl) {
  const FrontDesc& fd = dl[blockIdx.y];
  if (!big_active(d, fd)) return;
  const int j = blockIdx.x * (SBT / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (j >= fd.c || fd.m == fd.c) return;  // uniform over the warp
  double* xv = s.fvec + fd.rowptr;
  const double* Lj = s.L + fd.Lptr + (size_t)j * fd.m;
  double a = 0.0;
  for (int i = fd.c + lane; i < fd.m; i += 32) a = fma(Lj[i], xv[i], a);
  for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(FULL, a, off);
  if (lane == 0) xv[j] -= a;
}

// unit upper triangle L_KK^T of columns jb .. jb+w-1, last sub-block first
__global__ void __launch_bounds__(SBT) k_bigs_bwd_diag(Dev d, SnDev s, const FrontDesc* dl, int jb) {
  const FrontDesc& fd = dl[blockIdx.x];
  if (!big_active(d, fd) || jb >= fd.c) return;
  const int m = fd.m, w = min(SBW, fd.c - jb), tid = threadIdx.x, nt = blockDim.x;
  double* xv = s.fvec + fd.rowptr;
  const double* Lb = s.L + fd.Lptr + jb + (size_t)jb * m;  // L(jb + r, jb + j) = Lb[r + j m]
  __shared__ double v[SBW];
  for (int t = tid; t < w; t += nt) v[t] = xv[jb + t];
  __syncthreads();
  for (int sb = (w - 1) / 32 * 32; sb >= 0; sb -= 32) {
    const int ws = min(32, w - sb);
    if (tid < 32) {
      double x = (tid < ws) ? v[sb + tid] : 0.0;
      for (int j = ws - 1; j >= 0; --j) {
        const double xj = __shfl_sync(FULL, x, j);
        if (tid < j) x = fma(-Lb[(sb + j) + (size_t)(sb + tid) * m], xj, x);  // L(sb+j, sb+tid)
      }
      if (tid < ws) v[sb + tid] = x;
    }
    __syncthreads();
    for (int i = tid; i < sb; i += nt) {  // x_i -= sum_j L(sb + j, i) x_{sb+j}
      double a = v[i];
      for (int j = 0; j < ws; ++j) a = fma(-Lb[(sb + j) + (size_t)i * m], v[sb + j], a);
      v[i] = a;
    }
    __syncthreads();
  }
  for (int t = tid; t < w; t += nt) xv[jb + t] = v[t];
}

// x_i -= sum_{j < w} L(jb + j, i) x_{jb+j} for columns i < jb: a warp per
// column, the block's rows across lanes (column i is contiguous there)
__global__ void __launch_bounds__(SBT) k_bigs_bwd_cols(Dev d, SnDev s, const FrontDesc* dl, int jb) {
  const FrontDesc& fd = dl[blockIdx.y];
  if (!big_active(d, fd) || jb >= fd.c) return;
  const int i = blockIdx.x * (SBT / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= jb) return;  // uniform over the warp
  const int m = fd.m, w = min(SBW, fd.c - jb);
  double* xv = s.fvec + fd.rowptr;
  const double* Li = s.L + fd.Lptr + jb + (size_t)i * m;  // L(jb + j, i) = Li[j]
  double a = 0.0;
  for (int j = lane; j < w; j += 32) a = fma(Li[j], xv[jb + j], a);
  for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(FULL, a, off);
  if (lane == 0) xv[i] -= a;
}

__global__ void __launch_bounds__(SBT) k_bigs_bwd_post(Dev d, SnDev s, const FrontDesc* dl) {
  const FrontDesc& fd = dl[blockIdx.x];
  if (!big_active(d, fd)) return;
  const double* xv = s.fvec + fd.rowptr;
  for (int j = threadIdx.x; j < fd.c; j += blockDim.x) d.b[fd.first + j] = xv[j];
}

}  // namespace nmpc
