// Numeric supernodal Cholesky (eq. cholesky-numeric, Sec. 3.2.3) and the
// permuted triangular solves (eqs. cholesky-lower/upper), level by level
// over the supernodal elimination tree computed once on the host.
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
#include "kernels.h"

namespace nmpc {

extern __shared__ double dsm[];

__global__ void k_factor_level(Dev d, SnDev s, const int* list, int smem_cap) {
  const int J = list[blockIdx.x];
  const int inst = s.sn_inst[J];
  Ctl* ctl = d.ctl + inst;
  if (!ctl->need_factor) return;
  const int m = s.sn_nrow[J], c = s.sn_ncol[J], mu = m - c;
  double* Lp = s.L + s.sn_Lptr[J];
  double* Up = s.U + s.sn_Uptr[J];
  const bool in_smem = (long long)m * c + (long long)mu * mu <= smem_cap;
  double* F = in_smem ? dsm : Lp;                       // m x c panel, ld m
  double* G = in_smem ? dsm + (size_t)m * c : Up;       // mu x mu update, ld mu
  const int tid = threadIdx.x, nt = blockDim.x;
  if (in_smem)
    for (int t = tid; t < m * c; t += nt) F[t] = Lp[t];
  for (int t = tid; t < mu * mu; t += nt) G[t] = 0.0;
  __syncthreads();
  // extend-add of the children's update matrices
  for (int q = s.sn_child_ptr[J]; q < s.sn_child_ptr[J + 1]; ++q) {
    const int C = s.sn_child[q];
    const int mc = s.sn_nrow[C] - s.sn_ncol[C];
    const int* rel = s.sn_rel + s.sn_relptr[C];
    const double* UC = s.U + s.sn_Uptr[C];
    for (int t = tid; t < mc * mc; t += nt) {
      const int a = t % mc, b = t / mc;
      if (a < b) continue;
      const int ra = rel[a], rb = rel[b];
      const double v = UC[t];
      if (rb < c) F[ra + (size_t)rb * m] += v;
      else G[(ra - c) + (size_t)(rb - c) * mu] += v;
    }
    __syncthreads();
  }
  // right-looking partial factorization of the front
  __shared__ double piv;
  for (int j = 0; j < c; ++j) {
    if (tid == 0) {
      double dj = F[j + (size_t)j * m];
      if (!(dj > 0.0) || !isfinite(dj)) {
        *(volatile int*)&ctl->factor_fail = 1;
        dj = 1.0;
      }
      piv = sqrt(dj);
      F[j + (size_t)j * m] = piv;
    }
    __syncthreads();
    const double inv = 1.0 / piv;
    for (int i = j + 1 + tid; i < m; i += nt) F[i + (size_t)j * m] *= inv;
    __syncthreads();
    const int nn = m - j - 1;
    const double* colj = F + (size_t)j * m;
    for (int t = tid; t < nn * nn; t += nt) {
      const int ii = t % nn, kk = t / nn;
      if (ii < kk) continue;
      const int i = j + 1 + ii, k = j + 1 + kk;
      const double upd = colj[i] * colj[k];
      if (k < c) F[i + (size_t)k * m] -= upd;
      else G[(i - c) + (size_t)(k - c) * mu] -= upd;
    }
    __syncthreads();
  }
  if (in_smem) {
    for (int t = tid; t < m * c; t += nt) Lp[t] = F[t];
    for (int t = tid; t < mu * mu; t += nt) Up[t] = G[t];
  }
}

// Forward substitution L v = P b for one level.  The front vector of J is
// [b_J ; 0] plus the children's update vectors; after the pivot block is
// solved the remaining rows become J's update vector.
__global__ void k_fwd_level(Dev d, SnDev s, const int* list) {
  const int J = list[blockIdx.x];
  if (d.ctl[s.sn_inst[J]].status != ST_RUNNING) return;
  const int m = s.sn_nrow[J], c = s.sn_ncol[J], first = s.sn_first[J];
  const double* Lp = s.L + s.sn_Lptr[J];
  double* fv = dsm;          // m
  double* vv = dsm + m;      // c
  const int tid = threadIdx.x, nt = blockDim.x;
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
  for (int j = 0; j < c; ++j) {
    const double vj = fv[j] / Lp[j + (size_t)j * m];
    for (int i = j + 1 + tid; i < c; i += nt) fv[i] -= Lp[i + (size_t)j * m] * vj;
    if (tid == 0) vv[j] = vj;
    __syncthreads();
  }
  double* uvJ = s.uv + s.sn_uvptr[J];
  for (int i = c + tid; i < m; i += nt) {
    double a = fv[i];
    for (int j = 0; j < c; ++j) a -= Lp[i + (size_t)j * m] * vv[j];
    uvJ[i - c] = a;
  }
  for (int j = tid; j < c; j += nt) d.b[first + j] = vv[j];
}

// Backward substitution L^T x = v for one level (parents before children).
__global__ void k_bwd_level(Dev d, SnDev s, const int* list) {
  const int J = list[blockIdx.x];
  if (d.ctl[s.sn_inst[J]].status != ST_RUNNING) return;
  const int m = s.sn_nrow[J], c = s.sn_ncol[J], first = s.sn_first[J];
  const double* Lp = s.L + s.sn_Lptr[J];
  const int* rows = s.sn_rows + s.sn_rowptr[J];
  double* xv = dsm;          // m: x of the update rows (ancestors, solved)
  double* tv = dsm + m;      // c
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = c + tid; i < m; i += nt) xv[i] = d.b[rows[i]];
  __syncthreads();
  for (int j = tid; j < c; j += nt) {
    double a = d.b[first + j];
    for (int i = c; i < m; ++i) a -= Lp[i + (size_t)j * m] * xv[i];
    tv[j] = a;
  }
  __syncthreads();
  for (int j = c - 1; j >= 0; --j) {
    const double xj = tv[j] / Lp[j + (size_t)j * m];
    __syncthreads();
    for (int i = tid; i < j; i += nt) tv[i] -= Lp[j + (size_t)i * m] * xj;
    if (tid == 0) xv[j] = xj;
    __syncthreads();
  }
  for (int j = tid; j < c; j += nt) d.b[first + j] = xv[j];
}

}  // namespace nmpc
