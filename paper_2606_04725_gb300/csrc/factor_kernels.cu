// Numeric supernodal Cholesky (eq. cholesky-numeric, Sec. 3.2.3) and the
// permuted triangular solves (eqs. cholesky-lower/upper), level by level
// over the supernodal elimination tree computed once on the host.
//
// Storage: each supernode's panel is m x c column-major; its diagonal holds
// the reciprocals 1/L_jj (the solves multiply by them), everything else is L.
//
// Multifrontal form: supernode J owns a frontal matrix whose first c_J
// columns are its factor panel and whose trailing (m_J - c_J)^2 block is the
// update matrix U_J passed to the parent.  A front is assembled from the
// condensed-matrix values already scattered into the panel plus the
// children's update matrices (extend-add in ascending child order, so the
// result is deterministic), then partially factored: pivots, scaled
// columns and the Schur complement.  One thread block handles one
// supernode; blocks of the same level run concurrently.  A non-positive or
// non-finite pivot flags the instance for inertia correction.
#include <cooperative_groups.h>

#include "kernels.h"

namespace nmpc {

extern __shared__ double dsm[];

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

// 1/sqrt(p) for a positive pivot: an FP32 seed (rsqrtf, about 23 bits) and
// two Newton steps for f(y) = 1/y^2 - p, y <- y (3 - p y^2) / 2, which
// converge quadratically to full double precision.  Seven FP64 operations
// instead of a double division and square root: on this GPU the pivot
// arithmetic sits on the critical path of every column.  Outside the FP32
// range the exact expression is used.
__device__ __forceinline__ double rsqrt_newton(double p) {
  if (!(p >= 1e-36 && p <= 1e36)) return 1.0 / sqrt(p);
  double y = (double)rsqrtf((float)p);
  const double hp = 0.5 * p;
  y = y * fma(-hp, y * y, 1.5);
  y = y * fma(-hp, y * y, 1.5);
  return y;
}

// Front held as one m x m column-major matrix in shared memory: columns
// [0, c) become the factor panel, the trailing (m-c) block the update
// matrix.  Two barriers per pivot column j: (A) column j is scaled by
// 1/sqrt(p_j) into its final L values (the diagonal keeps 1/L_jj, which the
// solves multiply by); (B) the rank-1 Schur update F_ik -= L_ij L_kj runs over
// the flat-enumerated trailing lower triangle, one FMA per entry with all
// lanes busy.  The thread that finalizes the next diagonal entry checks it
// and computes its reciprocal square root for the next phase.
// A pivot counts as positive only if it exceeds pivtol * |K_jj| (K_jj the
// assembled diagonal): a pivot at rounding level is a zero eigenvalue, the
// wrong inertia of eq. infiniteOCP-inertia (which requires n_0 = 0).
__device__ __forceinline__ bool pivot_ok(double p, double kjj, double pivtol) {
  return p > pivtol * fabs(kjj) && p > 0.0 && isfinite(p);
}

__device__ void factor_front_smem(Ctl* ctl, double* F, int m, int c, double* rsq, const double* kd, double pivtol) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) {
    double p = F[0];
    if (!pivot_ok(p, kd[0], pivtol)) { *(volatile int*)&ctl->factor_fail = 1; p = 1.0; }
    rsq[0] = rsqrt_newton(p);
  }
  __syncthreads();
  for (int j = 0; j < c; ++j) {
    double* colj = F + (size_t)j * m;
    const double sj = rsq[j];
    for (int i = j + 1 + tid; i < m; i += nt) colj[i] *= sj;
    if (tid == 0) colj[j] = sj;
    __syncthreads();
    const int nn = m - j - 1;
    const int tot = nn * (nn + 1) / 2;
    for (int t = tid; t < tot; t += nt) {
      const int kk = tri_col(t, nn);
      const int ii = kk + (t - (kk * nn - kk * (kk - 1) / 2));
      const int k = j + 1 + kk, i = j + 1 + ii;
      double v = fma(-colj[i], colj[k], F[i + (size_t)k * m]);
      if (t == 0 && j + 1 < c) {  // (j+1, j+1): the next pivot is final now
        if (!pivot_ok(v, kd[j + 1], pivtol)) { *(volatile int*)&ctl->factor_fail = 1; v = 1.0; }
        rsq[j + 1] = rsqrt_newton(v);
      }
      F[i + (size_t)k * m] = v;
    }
    __syncthreads();
  }
}

__global__ void k_factor_level(Dev d, SnDev s, const int* list, int smem_cap) {
  const int J = list[blockIdx.x];
  const int inst = s.sn_inst[J];
  Ctl* ctl = d.ctl + inst;
  if (!ctl->need_factor) return;
  const int m = s.sn_nrow[J], c = s.sn_ncol[J], mu = m - c;
  double* Lp = s.L + s.sn_Lptr[J];
  double* Up = s.U + s.sn_Uptr[J];
  const int tid = threadIdx.x, nt = blockDim.x;
  if ((long long)m * m + c <= smem_cap) {
    // ---- whole front in shared memory
    double* F = dsm;
    double* rsq = dsm + (size_t)m * m;  // c reciprocal square roots of the pivots
    for (int t = tid; t < m * c; t += nt) F[t] = Lp[t];
    for (int t = m * c + tid; t < m * m; t += nt) F[t] = 0.0;
    __syncthreads();
    for (int q = s.sn_child_ptr[J]; q < s.sn_child_ptr[J + 1]; ++q) {
      const int C = s.sn_child[q];
      const int mc = s.sn_nrow[C] - s.sn_ncol[C];
      const int* rel = s.sn_rel + s.sn_relptr[C];
      const double* UC = s.U + s.sn_Uptr[C];
      const int tot = mc * (mc + 1) / 2;
      for (int t = tid; t < tot; t += nt) {
        const int b = tri_col(t, mc);
        const int a = b + (t - (b * mc - b * (b - 1) / 2));
        F[rel[a] + (size_t)rel[b] * m] += UC[a + (size_t)b * mc];
      }
      __syncthreads();
    }
    factor_front_smem(ctl, F, m, c, rsq, s.Kdiag + s.sn_first[J], s.pivtol);
    for (int t = tid; t < m * c; t += nt) Lp[t] = F[t];
    for (int t = tid; t < mu * mu; t += nt) {
      const int a = t % mu, b = t / mu;
      Up[t] = F[(c + a) + (size_t)(c + b) * m];
    }
    return;
  }
  // ---- large front: panel in the factor array, update matrix in scratch
  double* F = Lp;  // m x c, ld m
  double* G = Up;  // mu x mu, ld mu
  for (int t = tid; t < mu * mu; t += nt) G[t] = 0.0;
  __syncthreads();
  for (int q = s.sn_child_ptr[J]; q < s.sn_child_ptr[J + 1]; ++q) {
    const int C = s.sn_child[q];
    const int mc = s.sn_nrow[C] - s.sn_ncol[C];
    const int* rel = s.sn_rel + s.sn_relptr[C];
    const double* UC = s.U + s.sn_Uptr[C];
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
  __shared__ double pivg;
  for (int j = 0; j < c; ++j) {
    if (tid == 0) {
      double dj = F[j + (size_t)j * m];
      if (!pivot_ok(dj, s.Kdiag[s.sn_first[J] + j], s.pivtol)) { *(volatile int*)&ctl->factor_fail = 1; dj = 1.0; }
      pivg = 1.0 / sqrt(dj);
      F[j + (size_t)j * m] = pivg;  // reciprocal of L_jj (see the solves)
    }
    __syncthreads();
    const double inv = pivg;
    for (int i = j + 1 + tid; i < m; i += nt) F[i + (size_t)j * m] *= inv;
    __syncthreads();
    const int nn = m - j - 1;
    const int tot = nn * (nn + 1) / 2;
    const double* colj = F + (size_t)j * m;
    for (int t = tid; t < tot; t += nt) {
      const int kk = tri_col(t, nn);
      const int ii = kk + (t - (kk * nn - kk * (kk - 1) / 2));
      const int i = j + 1 + ii, k = j + 1 + kk;
      if (k < c) F[i + (size_t)k * m] = fma(-colj[i], colj[k], F[i + (size_t)k * m]);
      else G[(i - c) + (size_t)(k - c) * mu] = fma(-colj[i], colj[k], G[(i - c) + (size_t)(k - c) * mu]);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Cluster-cooperative front factorization (blocked, right-looking).
//
// One thread-block cluster of Q CTAs factors one front.  Columns are dealt to
// the CTAs block-cyclically in blocks of PB columns (block b -> CTA b % Q), so
// every CTA holds all m rows of its own columns in shared memory.  For each
// pivot panel (block p < ceil(c / PB)):
//   1. its owner factors the panel (pivot test, 1/sqrt(p) by Newton, column
//      scaling, rank-1 updates inside the panel);
//   2. one cluster barrier publishes it;
//   3. every CTA copies the panel rows it needs from the owner's shared memory
//      (distributed shared memory) and applies the rank-PB update to its own
//      trailing columns, one FMA per panel column and entry.
// Afterwards the owners write the factor panel (columns < c) and the update
// matrix (columns >= c) back.  Q is chosen per level so that the fronts of a
// level together occupy most SMs.  The panel diagonal keeps 1/L_jj.
// ---------------------------------------------------------------------------
constexpr int PB = 8;

__global__ void k_factor_cluster(Dev d, SnDev s, const int* list) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int Q = (int)cluster.num_blocks();
  const int q = (int)cluster.block_rank();
  const int J = list[blockIdx.x / Q];
  Ctl* ctl = d.ctl + s.sn_inst[J];
  if (!ctl->need_factor) return;  // uniform over the cluster: same instance
  const int m = s.sn_nrow[J], c = s.sn_ncol[J], mu = m - c;
  double* Lp = s.L + s.sn_Lptr[J];
  double* Up = s.U + s.sn_Uptr[J];
  const double* kd = s.Kdiag + s.sn_first[J];
  const double pivtol = s.pivtol;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nblk = (m + PB - 1) / PB;
  const int my_blocks = (nblk - q + Q - 1) / Q;  // blocks q, q+Q, ...
  double* Fl = dsm;                                // m x (my_blocks * PB), ld m
  double* P = dsm + (size_t)m * my_blocks * PB;    // panel copy: m x PB, ld m
  __shared__ double rsq_s;
  // local column of global column k (owned by this CTA)
  auto lcol = [&](int k) { return ((k / PB) / Q) * PB + (k % PB); };
  // ---- assemble: own columns from the condensed values, then the children
  for (int t = tid; t < m * my_blocks * PB; t += nt) {
    const int i = t % m, lc = t / m;
    const int k = ((lc / PB) * Q + q) * PB + lc % PB;
    Fl[t] = (k < c) ? Lp[i + (size_t)k * m] : 0.0;
  }
  __syncthreads();
  for (int qq = s.sn_child_ptr[J]; qq < s.sn_child_ptr[J + 1]; ++qq) {
    const int C = s.sn_child[qq];
    const int mc = s.sn_nrow[C] - s.sn_ncol[C];
    const int* rel = s.sn_rel + s.sn_relptr[C];
    const double* UC = s.U + s.sn_Uptr[C];
    const int tot = mc * (mc + 1) / 2;
    for (int t = tid; t < tot; t += nt) {
      const int b = tri_col(t, mc);
      const int rb = rel[b];
      if ((rb / PB) % Q != q) continue;
      const int a = b + (t - (b * mc - b * (b - 1) / 2));
      Fl[rel[a] + (size_t)lcol(rb) * m] += UC[a + (size_t)b * mc];
    }
    __syncthreads();
  }
  // ---- panels
  const int npan = (c + PB - 1) / PB;
  for (int p = 0; p < npan; ++p) {
    const int jb = p * PB, w = min(PB, c - jb);
    const int owner = p % Q;
    if (q == owner) {
      double* Fp = Fl + (size_t)lcol(jb) * m;  // panel columns are contiguous locally
      for (int jj = 0; jj < w; ++jj) {
        const int j = jb + jj;
        double* colj = Fp + (size_t)jj * m;
        if (tid == 0) {
          double piv = colj[j];
          if (!pivot_ok(piv, kd[j], pivtol)) { *(volatile int*)&ctl->factor_fail = 1; piv = 1.0; }
          rsq_s = rsqrt_newton(piv);
          colj[j] = rsq_s;
        }
        __syncthreads();
        const double sj = rsq_s;
        for (int i = j + 1 + tid; i < m; i += nt) colj[i] *= sj;
        __syncthreads();
        // rank-1 update of the remaining panel columns jj+1 .. w-1
        const int rem = w - jj - 1;
        if (rem > 0) {
          const int rows = m - j - 1;
          for (int t = tid; t < rows * rem; t += nt) {
            const int i = j + 1 + t % rows, kk = jj + 1 + t / rows;
            const int k = jb + kk;
            if (i >= k) Fp[i + (size_t)kk * m] = fma(-colj[i], colj[k], Fp[i + (size_t)kk * m]);
          }
          __syncthreads();
        }
      }
    }
    cluster.sync();  // the panel is final and visible to the cluster
    // copy rows jb..m-1 of the panel from the owner
    {
      const double* src = cluster.map_shared_rank(Fl, owner) + (size_t)((jb / PB) / Q) * PB * m;
      for (int t = tid; t < (m - jb) * w; t += nt) {
        const int i = jb + t % (m - jb), jj = t / (m - jb);
        P[i + (size_t)jj * m] = src[i + (size_t)jj * m];
      }
    }
    __syncthreads();
    // rank-w update of own columns k >= jb + w, rows i >= k (the panel's own
    // block also holds update-matrix columns when c is not a multiple of PB)
    for (int lb = 0; lb < my_blocks; ++lb) {
      const int b = lb * Q + q;
      if (b < p) continue;
      const int k0 = b * PB;
      const int ks = (b == p) ? jb + w : k0;
      const int kcnt = min(k0 + PB, m) - ks;
      if (kcnt <= 0) continue;
      const int rows = m - ks;
      for (int t = tid; t < rows * kcnt; t += nt) {
        const int i = ks + t % rows, kk = t / rows;
        const int k = ks + kk;
        if (i < k) continue;
        const int lc = lb * PB + (k - k0);
        double acc = Fl[i + (size_t)lc * m];
#pragma unroll
        for (int jj = 0; jj < PB; ++jj)
          if (jj < w) acc = fma(-P[i + (size_t)jj * m], P[k + (size_t)jj * m], acc);
        Fl[i + (size_t)lc * m] = acc;
      }
    }
    __syncthreads();
  }
  cluster.sync();  // no CTA may leave while others still read its panels
  // ---- write back own columns
  for (int t = tid; t < m * my_blocks * PB; t += nt) {
    const int i = t % m, lc = t / m;
    const int k = ((lc / PB) * Q + q) * PB + lc % PB;
    if (k >= m) continue;
    if (k < c) Lp[i + (size_t)k * m] = Fl[t];
    else if (i >= c) Up[(i - c) + (size_t)(k - c) * mu] = Fl[t];
  }
}

// Forward substitution L v = P b for one level.  The front vector of J is
// [b_J ; 0] plus the children's update vectors; after the pivot block is
// solved the remaining rows become J's update vector.  The panel is staged
// in shared memory (coalesced), the c x c triangular part runs in one warp
// (warp barriers only), the update rows in all threads.
__global__ void k_fwd_level(Dev d, SnDev s, const int* list, int smem_cap) {
  const int J = list[blockIdx.x];
  if (d.ctl[s.sn_inst[J]].status != ST_RUNNING) return;
  const int m = s.sn_nrow[J], c = s.sn_ncol[J], first = s.sn_first[J];
  const double* Lg = s.L + s.sn_Lptr[J];
  const bool stage = (long long)m * c + m <= smem_cap;  // else read the panel from global memory
  double* fv = dsm + (stage ? (size_t)m * c : 0);       // m
  const double* Ls = stage ? dsm : Lg;                   // m x c
  const int tid = threadIdx.x, nt = blockDim.x;
  if (stage)
    for (int t = tid; t < m * c; t += nt) dsm[t] = Lg[t];
  for (int i = tid; i < m; i += nt) fv[i] = (i < c) ? d.b[first + i] : 0.0;
  __syncthreads();
  for (int q = s.sn_child_ptr[J]; q < s.sn_child_ptr[J + 1]; ++q) {
    const int C = s.sn_child[q];
    const int mc = s.sn_nrow[C] - s.sn_ncol[C];
    const int* rel = s.sn_rel + s.sn_relptr[C];
    const double* uvC = s.uv + s.sn_uvptr[C];
    for (int a = tid; a < mc; a += nt) fv[rel[a]] += uvC[a];
    __syncthreads();
  }
  if (tid < 32) {
    for (int j = 0; j < c; ++j) {
      const double vj = fv[j] * Ls[j + (size_t)j * m];  // diagonal stores 1/L_jj
      __syncwarp();
      for (int i = j + 1 + tid; i < c; i += 32) fv[i] = fma(-Ls[i + (size_t)j * m], vj, fv[i]);
      if (tid == 0) fv[j] = vj;
      __syncwarp();
    }
  }
  __syncthreads();
  double* uvJ = s.uv + s.sn_uvptr[J];
  for (int i = c + tid; i < m; i += nt) {
    double a = fv[i];
    for (int j = 0; j < c; ++j) a = fma(-Ls[i + (size_t)j * m], fv[j], a);
    uvJ[i - c] = a;
  }
  for (int j = tid; j < c; j += nt) d.b[first + j] = fv[j];
}

// Backward substitution L^T x = v for one level (parents before children).
__global__ void k_bwd_level(Dev d, SnDev s, const int* list, int smem_cap) {
  const int J = list[blockIdx.x];
  if (d.ctl[s.sn_inst[J]].status != ST_RUNNING) return;
  const int m = s.sn_nrow[J], c = s.sn_ncol[J], first = s.sn_first[J];
  const double* Lg = s.L + s.sn_Lptr[J];
  const int* rows = s.sn_rows + s.sn_rowptr[J];
  const bool stage = (long long)m * c + m <= smem_cap;
  double* xv = dsm + (stage ? (size_t)m * c : 0);       // m
  const double* Ls = stage ? dsm : Lg;                   // m x c
  const int tid = threadIdx.x, nt = blockDim.x;
  if (stage)
    for (int t = tid; t < m * c; t += nt) dsm[t] = Lg[t];
  for (int i = tid; i < m; i += nt) xv[i] = (i < c) ? d.b[first + i] : d.b[rows[i]];
  __syncthreads();
  // t_j = v_j - sum_{i >= c} L_ij x_i  (x_i of ancestors, already solved)
  for (int j = tid; j < c; j += nt) {
    double a = xv[j];
    for (int i = c; i < m; ++i) a = fma(-Ls[i + (size_t)j * m], xv[i], a);
    xv[j] = a;
  }
  __syncthreads();
  if (tid < 32) {
    for (int j = c - 1; j >= 0; --j) {
      const double xj = xv[j] * Ls[j + (size_t)j * m];  // diagonal stores 1/L_jj
      __syncwarp();
      for (int i = tid; i < j; i += 32) xv[i] = fma(-Ls[j + (size_t)i * m], xj, xv[i]);
      if (tid == 0) xv[j] = xj;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int j = tid; j < c; j += nt) d.b[first + j] = xv[j];
}

}  // namespace nmpc
