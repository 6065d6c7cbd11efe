// C ABI of the NMPC library: handle management, workspace layout, parameter
// updates and the interior-point driver (Algorithm 2 of arXiv 2606.04725).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/nmpc.h"
#include "kernels.h"
#include "structure.h"

using namespace nmpc;

namespace {

// Bump allocator over the caller's workspace (first pass only measures).
struct Carver {
  char* base = nullptr;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += std::max<size_t>(count, 1) * sizeof(T);
    return p;
  }
};

}  // namespace

struct nmpc_handle {
  Analysis A;
  nmpc_options opt{};
  cudaStream_t stream = nullptr;
  std::string err;
  size_t ws_bytes = 0;
  bool bound = false, have_solution = false;
  Dev d{};
  SnDev s{};
  // device-only arrays not in Dev/SnDev
  int* d_tgt_inst = nullptr;
  double* d_Drow = nullptr;
  long long* d_inst_Lbeg = nullptr;
  long long* d_inst_Lend = nullptr;
  int* d_flags = nullptr;
  double* d_stage = nullptr;  // staging of host parameter arrays
  int* d_inst_spoff = nullptr;  // first setpoint of each instance in a packed all-instance array
  long long sp_packed = 0;      // setpoints of all instances packed (sum of their horizons, or g*g each)
  int* h_flags = nullptr;     // pinned
  std::vector<int> lvl_ptr;
  std::vector<int> lvl_smem_factor, lvl_smem_solve, lvl_smem_bwd;  // bytes per level
  std::vector<int> lvl_cluster;                      // CTAs per front (0 = single-CTA kernel)
  std::vector<long long> desc_abase;                 // per level position: first extend-add range (-1 none)
  std::vector<long long> desc_wptr;                  // per level position: W scratch offset (cluster fronts)
  long long nW_cluster = 0;
  // levels of large fronts (blocked path over many SMs): shapes per level
  std::vector<char> lvl_big, lvl_bigsolve;
  // persistent solves over the first solve_prefix levels (fronts in level order)
  int solve_prefix = 0, solve_prefix_fronts = 0, persist_blocks_fwd = 0, persist_blocks_bwd = 0;
  int persist_smem_fwd = 0, persist_smem_bwd = 0;
  int persist_stage_cap = 0;  // doubles: panels staged by the persistent solves at most this large
  int* d_solve_flags = nullptr;
  // dataflow factorization (factor_mode 3) over the first flow_levels levels (fronts in level order)
  int flow_levels = 0, flow_fronts = 0, flow_blocks = 0, flow_smem = 0;
  int* d_flow_flags = nullptr;
  // level-ordered lists of the fronts of the instances taking part in the
  // next persistent factorization ([0, ns)) and solves ([ns, 2 ns)), and
  // their lengths ([0], [1]); used for batches (front_lists)
  int* d_front_list = nullptr;
  int* d_front_cnt = nullptr;
  bool front_lists = false;
  std::vector<int> lvl_maxm, lvl_maxc, lvl_maxmu, lvl_maxch, lvl_maxmc;
  std::vector<int> amap;                             // extend-add pairs (source, destination)
  std::vector<long long> amap_ptr;                   // ranges per (front, CTA, child)
  std::vector<int> lvl_cluster_smem;                 // bytes per CTA of the cluster kernel
  std::vector<InvItem> inv_items;                    // blocks transformed after each factorization
  std::vector<ScaleUnit> scale_units;                // 32-row slices below them
  std::vector<int> lvl_inv_ptr, lvl_scale_ptr;       // their ranges per level
  int s_form = 2;                                    // SnDev::solve_form
  int n_sm = 152;
  int cluster_ctas_per_sm = 1;  // CTAs of the cluster kernel per SM aimed at when choosing Q (2 measured no faster)
  int smem_cap_doubles = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // side stream of the panel transforms (forked per level, joined after the factorization)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool side_pending = false;  // work queued on the side stream since the last join
  std::vector<Ctl> h_ctl;
  Ctl* d_ctl_save = nullptr;
  long long launches = 0;
  double sens_residual = 0.0;  // relative residual of the last adjoint solve
  // the interior-point loop as one CUDA graph with conditional nodes
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool graph_off = false;  // host-driven loop only (allocation-free one-shot solve)
  long long nodes_eval = 0, nodes_factor = 0, nodes_solve = 0, nodes_trial = 0, nodes_update = 0;
  long long nodes_cg = 0, nodes_solve2 = 0;  // HyKKT: one CG step, the final solve and step limits
  CondArgs cond{};  // passed to the step-ending kernels; on only while the graph is captured
};

namespace {

constexpr int SMEM_FACTOR_CAP_BYTES = 200 * 1024;
constexpr int FACTOR_THREADS = 1024;  // 32 warps per front hide FP64 and shared-memory latency
constexpr int CLUSTER_THREADS = 256;  // per CTA of the cluster-cooperative front kernel (FCT in factor_kernels.cu)
constexpr int CLUSTER_PB = 8;         // column block of the cluster kernel (PB in factor_kernels.cu)
constexpr int FLOW_SMEM_CAP_BYTES = 220 * 1024;  // dynamic shared memory of a k_factor_flow block
// shared memory (doubles) of k_factor_flow for a front of m rows and c pivot
// columns: the pivot columns rounded up to whole panels, two L panel buffers
// or (later) L of the update rows, thresholds and reciprocal pivots
long long flow_need(long long m, long long c) {
  const long long cp = (c + CLUSTER_PB - 1) / CLUSTER_PB * CLUSTER_PB, mu = m - c;
  return m * cp + std::max(mu * c, 2 * m * CLUSTER_PB) + 2 * cp;
}
constexpr int SENS_REFINE = 6;        // refinement sweeps of the adjoint solve

// Memory of the update matrices.  A front's update matrix is written when its
// level is factored and read once, by its parent's extend-add; after the
// parent's level it is dead, so later levels reuse its memory.  Offsets are
// assigned by a sweep over the levels with a first-fit free list (ordered by
// offset, neighbours merged): before level t the matrices whose parents lie
// below t are freed, then level t's are placed.  The levels of the dataflow
// launch (the first flow_levels levels) run concurrently, so they are placed
// together and none of their memory is reused before the launch has ended.
// The workspace then holds the largest set of update matrices live at one
// level instead of all of them.  Returns the arena size in doubles.
long long plan_update_memory(Analysis& A, int flow_levels) {
  const int nl = (int)A.level_ptr.size() - 1, ns = (int)A.sn_first.size();
  std::vector<int> lvl(ns, 0);
  for (int l = 0; l < nl; ++l)
    for (int q = A.level_ptr[l]; q < A.level_ptr[l + 1]; ++q) lvl[A.level_sn[q]] = l;
  std::vector<std::vector<int>> frees(nl + 1);  // fronts whose matrix dies before level t
  for (int J = 0; J < ns; ++J) {
    const int p = A.sn_parent[J];
    const int dead = std::max(p >= 0 ? lvl[p] : lvl[J], flow_levels - 1) + 1;  // first level that may reuse it
    frees[std::min(dead, nl)].push_back(J);
  }
  std::map<long long, long long> free_list;  // offset -> doubles
  long long end = 0;
  auto release = [&](long long off, long long len) {
    if (len <= 0) return;
    auto it = free_list.emplace(off, len).first;
    auto nx = std::next(it);
    if (nx != free_list.end() && it->first + it->second == nx->first) { it->second += nx->second; free_list.erase(nx); }
    if (it != free_list.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) { pv->second += it->second; free_list.erase(it); }
    }
  };
  auto place = [&](long long len) {
    for (auto it = free_list.begin(); it != free_list.end(); ++it)
      if (it->second >= len) {
        const long long off = it->first, rest = it->second - len;
        free_list.erase(it);
        if (rest > 0) free_list.emplace(off + len, rest);
        return off;
      }
    const long long off = end;
    end += len;
    return off;
  };
  auto size_of = [&](int J) {
    const long long mu = A.sn_nrow[J] - A.sn_ncol[J];
    return (mu * mu + 1) & ~1LL;  // even: every matrix starts on a 16-byte boundary
  };
  for (int t = 0; t < nl; ++t) {
    for (int J : frees[t]) release(A.sn_Uptr[J], size_of(J));
    if (t > 0 && t < flow_levels) continue;  // placed with level 0
    const int l1 = (t == 0) ? std::max(1, flow_levels) : t + 1;
    for (int l = t; l < std::min(l1, nl); ++l)
      for (int q = A.level_ptr[l]; q < A.level_ptr[l + 1]; ++q) {
        const int J = A.level_sn[q];
        A.sn_Uptr[J] = place(size_of(J));
      }
  }
  A.sn_Uptr[ns] = end;
  return end;
}

nmpc_status fail(nmpc_handle* h, nmpc_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}

#define CUDA_TRY(h, call)                                                                    \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return fail(h, NMPC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Lay out (or measure) every device array inside the workspace.
void carve(nmpc_handle* h, Carver& cv) {
  Analysis& A = h->A;
  Dev& d = h->d;
  SnDev& s = h->s;
  const int ni = A.n_inst, n = A.n, m = A.m, WH = A.mc.WH;
  const size_t nch = A.chunks.size(), ns = A.sn_first.size();
  d.inst_T = cv.take<int>(ni); d.inst_voff = cv.take<int>(ni); d.inst_roff = cv.take<int>(ni);
  d.inst_woff = cv.take<int>(ni); d.inst_n = cv.take<int>(ni); d.inst_m = cv.take<int>(ni);
  d.inst_nz = cv.take<int>(ni);
  d.var_inst = cv.take<int>(n); d.row_inst = cv.take<int>(m);
  d.yL = cv.take<double>(n); d.yU = cv.take<double>(n);
  d.p_x0 = cv.take<double>((size_t)ni * A.mc.nx); d.p_sp = cv.take<double>((size_t)ni * A.sp_stride);
  d.p_uprev = cv.take<double>(ni);
  d.y = cv.take<double>(n); d.zL = cv.take<double>(n); d.zU = cv.take<double>(n);
  d.sp = cv.take<double>(m); d.sm = cv.take<double>(m); d.wp = cv.take<double>(m); d.wm = cv.take<double>(m);
  d.bp = cv.take<double>(m); d.bm = cv.take<double>(m);
  d.grad = cv.take<double>(n); d.h = cv.take<double>(m); d.Hv = cv.take<double>((size_t)m * WH);
  d.Wv = cv.take<double>(A.nW); d.fvar = cv.take<double>(n);
  d.igL = cv.take<double>(n); d.igU = cv.take<double>(n); d.izL = cv.take<double>(n); d.izU = cv.take<double>(n);
  d.isp = cv.take<double>(m); d.ism = cv.take<double>(m); d.ibp = cv.take<double>(m); d.ibm = cv.take<double>(m);
  d.Hcol = cv.take<int>((size_t)m * WH); d.Hpos = cv.take<int>((size_t)m * WH);
  d.Hcsc_ptr = cv.take<int>(n + 1); d.Hcsc_slot = cv.take<int>(A.Hcsc_slot.size());
  d.Wadj_ptr = cv.take<int>(n + 1); d.Wadj_slot = cv.take<int>(A.Wadj_slot.size());
  d.Wadj_other = cv.take<int>(A.Wadj_other.size());
  d.dy = cv.take<double>(n); d.dzL = cv.take<double>(n); d.dzU = cv.take<double>(n);
  d.dsp = cv.take<double>(m); d.dsm = cv.take<double>(m); d.dwp = cv.take<double>(m); d.dwm = cv.take<double>(m);
  d.dbp = cv.take<double>(m); d.dbm = cv.take<double>(m); d.rowv = cv.take<double>(m);
  d.lam = cv.take<double>(m); d.HD = cv.take<double>((size_t)m * WH);
  d.cg_r = d.dsp; d.cg_p = d.dsm; d.cg_q = d.dbp;  // HyKKT only, where these are unused
  d.yt = cv.take<double>(n); d.spt = cv.take<double>(m); d.smt = cv.take<double>(m); d.ht = cv.take<double>(m);
  d.fvart = cv.take<double>(n);
  d.perm = cv.take<int>(n); d.iperm = cv.take<int>(n); d.b = cv.take<double>(n);
  d.ctl = cv.take<Ctl>(ni);
  d.filt_th = cv.take<double>((size_t)ni * FILTER_CAP); d.filt_ph = cv.take<double>((size_t)ni * FILTER_CAP);
  d.chunks = cv.take<Chunk>(nch); d.inst_chunk_ptr = cv.take<int>(ni + 1); d.inst_chunk_list = cv.take<int>(nch);
  d.red_var = cv.take<int>(n);
  d.red_eval = cv.take<RedEval>(nch); d.red_dir = cv.take<RedDir>(nch); d.red_trial = cv.take<RedTrial>(nch);
  d.red_cg = cv.take<double>(nch);
  d.tgt_L = cv.take<long long>(A.tgt_L.size()); d.tgt_diag = cv.take<int>(A.tgt_diag.size());
  d.tw_ptr = cv.take<int>(A.tw_ptr.size()); d.tw_idx = cv.take<int>(A.tw_idx.size());
  d.th_ptr = cv.take<int>(A.th_ptr.size()); d.th_a = cv.take<int>(A.th_a.size()); d.th_b = cv.take<int>(A.th_b.size());
  d.Lval = cv.take<double>(A.nnzL);
  d.Kdiag = cv.take<double>(n);
  d.sn_inst = cv.take<int>(ns);
  h->d_tgt_inst = cv.take<int>(A.tgt_L.size());
  h->d_Drow = cv.take<double>(m);
  h->d_inst_Lbeg = cv.take<long long>(ni); h->d_inst_Lend = cv.take<long long>(ni);
  h->d_flags = cv.take<int>(16);  // [0..2] summary, [3] wait timeout, [4..7] adjoint norms, [8..11] graph trip counts
  h->d_stage = cv.take<double>((size_t)ni * (A.mc.nx + A.sp_stride + 1));
  h->d_inst_spoff = cv.take<int>(ni + 1);
  h->d_ctl_save = cv.take<Ctl>(ni);
  d.trace = cv.take<double>((size_t)ni * (h->opt.max_iter + 2) * 8);
  d.red_cnt = cv.take<int>(ni + 1);
  s.sn_first = cv.take<int>(ns); s.sn_ncol = cv.take<int>(ns); s.sn_nrow = cv.take<int>(ns);
  s.sn_Lptr = cv.take<long long>(ns + 1); s.sn_Uptr = cv.take<long long>(ns + 1);
  s.sn_rowptr = cv.take<long long>(ns + 1); s.sn_rows = cv.take<int>(A.sn_rows.size());
  s.sn_child_ptr = cv.take<int>(ns + 1); s.sn_child = cv.take<int>(A.sn_child.size());
  s.sn_relptr = cv.take<long long>(ns + 1); s.sn_rel = cv.take<int>(A.sn_rel.size());
  s.level_ptr = cv.take<int>(A.level_ptr.size()); s.level_sn = cv.take<int>(ns);
  s.sn_uvptr = cv.take<long long>(ns + 1);
  s.desc = cv.take<FrontDesc>(ns);
  s.pos_of_sn = cv.take<int>(ns);
  s.front_inst = cv.take<int>(ns);
  h->d_front_list = cv.take<int>(2 * ns);
  h->d_front_cnt = cv.take<int>(2);
  h->front_lists = ni > 1 && ni <= FL_MAX_INST;
  h->d_solve_flags = cv.take<int>(2 * (ns + 2));  // forward and backward persistent solves
  h->d_flow_flags = cv.take<int>(h->flow_fronts + 2);
  s.amap = cv.take<IdxPair>(h->amap.size() / 2);
  s.amap_ptr = cv.take<long long>(h->amap_ptr.size());
  s.U = cv.take<double>(A.nU);
  s.W = cv.take<double>(h->nW_cluster);
  s.dpiv = cv.take<double>(n);
  s.uv = cv.take<double>(A.nuv);
  s.fvec = cv.take<double>(A.sn_rows.size());
  s.inv = cv.take<InvItem>(h->inv_items.size());
  s.n_inv = (int)h->inv_items.size();
  s.scale = cv.take<ScaleUnit>(h->scale_units.size());
  s.n_scale = (int)h->scale_units.size();
  s.solve_form = h->s_form;
  s.L = d.Lval;
  s.Kdiag = d.Kdiag;
  s.pivtol = A.mc.pivtol;
  s.spin_limit = h->opt.spin_limit > 0 ? h->opt.spin_limit : 10000000LL;
  s.timeout = h->d_flags + 3;
  s.sn_inst = d.sn_inst;
  s.ns = (int)ns;
  d.mc = A.mc; d.n_inst = ni; d.n = n; d.m = m; d.nW = A.nW; d.sp_stride = A.sp_stride;
  d.n_chunks = (int)nch; d.n_tgt = (int)A.tgt_L.size(); d.nnzL = A.nnzL;
}

template <class T>
cudaError_t up(const T* dst, const std::vector<T>& src, cudaStream_t st) {
  if (src.empty()) return cudaSuccess;
  return cudaMemcpyAsync(const_cast<T*>(dst), src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

// cg = 1: flag [2] says whether any HyKKT conjugate-gradient loop runs
nmpc_status read_flags(nmpc_handle* h, int cg = 0) {
  k_summary<<<1, 256, 0, h->stream>>>(h->d, h->d_flags, cg);
  ++h->launches;
  CUDA_TRY(h, cudaMemcpyAsync(h->h_flags, h->d_flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (h->h_flags[3]) return fail(h, NMPC_TIMEOUT, "a bounded wait between the CTAs of a front factorization ran out");
  return NMPC_OK;
}

// the factorization of one level
nmpc_status launch_factor_level(nmpc_handle* h, int l) {
  const int cnt = h->lvl_ptr[l + 1] - h->lvl_ptr[l];
  if (!cnt) return NMPC_OK;
  if (h->lvl_cluster[l] > 0) {
    const int Q = h->lvl_cluster[l];
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cnt * Q);
    cfg.blockDim = dim3(CLUSTER_THREADS);
    cfg.dynamicSmemBytes = h->lvl_cluster_smem[l];
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = Q;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CUDA_TRY(h, cudaLaunchKernelEx(&cfg, k_factor_cluster, h->d, h->s, (const FrontDesc*)(h->s.desc + h->lvl_ptr[l])));
    ++h->launches;
    return NMPC_OK;
  }
  if (h->lvl_big[l]) {
    const FrontDesc* dl = h->s.desc + h->lvl_ptr[l];
    const long long mu2 = (long long)h->lvl_maxmu[l] * h->lvl_maxmu[l];
    k_big_zero<<<dim3((unsigned)std::max(1LL, std::min(1024LL, (mu2 + 255) / 256)), cnt), 256, 0, h->stream>>>(h->d, h->s, dl);
    ++h->launches;
    for (int k = 0; k < h->lvl_maxch[l]; ++k) {
      k_big_extend<<<dim3((unsigned)std::max(1, std::min(1024, h->lvl_maxmc[l])), cnt), 256, 0, h->stream>>>(h->d, h->s, dl, k);
      ++h->launches;
    }
    const int npan = (h->lvl_maxc[l] + BIG_NB - 1) / BIG_NB;
    for (int p = 0; p < npan; ++p) {
      const int jb = p * BIG_NB;
      k_big_diag<<<cnt, 32, 0, h->stream>>>(h->d, h->s, dl, p);
      const int rows = std::max(0, h->lvl_maxm[l] - jb - 1);
      k_big_trsm<<<dim3((unsigned)std::max(1, (rows + BIG_ROWS - 1) / BIG_ROWS), cnt), BIG_ROWS, 0, h->stream>>>(h->d, h->s, dl, p);
      const int R = std::max(0, h->lvl_maxm[l] - jb - 1);
      const long long nb = (R + BIG_TILE - 1) / BIG_TILE;
      k_big_update<<<dim3((unsigned)std::max(1LL, nb * (nb + 1) / 2), cnt), 256, 0, h->stream>>>(h->d, h->s, dl, p);
      h->launches += 3;
    }
    return NMPC_OK;
  }
  k_factor_level<<<cnt, FACTOR_THREADS, h->lvl_smem_factor[l], h->stream>>>(h->d, h->s, h->s.desc + h->lvl_ptr[l],
                                                                 h->smem_cap_doubles);
  ++h->launches;
  return NMPC_OK;
}

// All levels.  The panel transform of a level (k_diag_inv, then
// k_panel_scale) only needs that level's factor, so it runs on the side
// stream as soon as the level is factored, alongside the factorization of the
// levels above (which leave most SMs idle near the root); the main stream
// waits for it at the end, before the inertia test and the solves.  (The
// one-shot static solve creates no stream: there the transforms run in order
// on the main stream.)
nmpc_status launch_factor(nmpc_handle* h) {
  const int nl = (int)h->lvl_ptr.size() - 1;
  const bool fork = h->side != nullptr;
  cudaStream_t ts = fork ? h->side : h->stream;
  bool forked = h->side_pending;
  const int L = h->flow_levels;
  if (L > 0) {
    const int* list = nullptr;
    if (h->front_lists) {  // only the fronts of the instances that need a factorization
      k_front_list<<<1, FL_THREADS, h->A.n_inst, h->stream>>>(h->d, h->s, h->flow_fronts, 0, h->d_front_list,
                                                               h->d_front_cnt);
      ++h->launches;
      list = h->d_front_list;
    }
    k_factor_flow<<<h->flow_blocks, CLUSTER_THREADS, h->flow_smem, h->stream>>>(h->d, h->s, h->s.desc, h->flow_fronts,
                                                                              h->d_flow_flags, list, h->d_front_cnt);
    ++h->launches;
  }
  for (int l = (L > 0 ? L - 1 : 0); l < nl; ++l) {
    // the dataflow levels' panel transforms go together after its launch
    const nmpc_status st = l < L ? NMPC_OK : launch_factor_level(h, l);
    if (st != NMPC_OK) return st;
    const int i0 = h->lvl_inv_ptr[l < L ? 0 : l], i1 = h->lvl_inv_ptr[l + 1];
    const int u0 = h->lvl_scale_ptr[l < L ? 0 : l], u1 = h->lvl_scale_ptr[l + 1];
    if (i1 == i0) continue;
    if (fork) {
      CUDA_TRY(h, cudaEventRecord(h->ev_fork, h->stream));
      CUDA_TRY(h, cudaStreamWaitEvent(h->side, h->ev_fork, 0));
      forked = true;
    }
    k_diag_inv<<<i1 - i0, 256, 0, ts>>>(h->d, h->s, i0);
    ++h->launches;
    if (u1 > u0) {
      k_panel_scale<<<u1 - u0, 128, 0, ts>>>(h->d, h->s, u0);
      ++h->launches;
    }
  }
  if (forked) {
    CUDA_TRY(h, cudaEventRecord(h->ev_join, h->side));
    CUDA_TRY(h, cudaStreamWaitEvent(h->stream, h->ev_join, 0));
    h->side_pending = false;
  }
  return NMPC_OK;
}

// The large-front solves of level l (see the k_bigs_* kernels): per column
// block a one-CTA-per-front triangle and a many-CTA product.
long long launch_big_fwd(nmpc_handle* h, int l) {
  const int cnt = h->lvl_ptr[l + 1] - h->lvl_ptr[l];
  const FrontDesc* dl = h->s.desc + h->lvl_ptr[l];
  cudaStream_t st = h->stream;
  long long n = 2;
  k_bigs_fwd_pre<<<cnt, BIG_SBT, 0, st>>>(h->d, h->s, dl);
  for (int jb = 0; jb < h->lvl_maxc[l]; jb += BIG_SBW) {
    k_bigs_fwd_diag<<<cnt, BIG_SBT, 0, st>>>(h->d, h->s, dl, jb);
    const int below = h->lvl_maxm[l] - jb;
    k_bigs_fwd_rows<<<dim3((unsigned)std::max(1, (below + 63) / 64), cnt), BIG_SBT, 0, st>>>(h->d, h->s, dl, jb);
    n += 2;
  }
  k_bigs_fwd_post<<<cnt, BIG_SBT, 0, st>>>(h->d, h->s, dl);
  return n;
}

long long launch_big_bwd(nmpc_handle* h, int l) {
  const int cnt = h->lvl_ptr[l + 1] - h->lvl_ptr[l];
  const FrontDesc* dl = h->s.desc + h->lvl_ptr[l];
  cudaStream_t st = h->stream;
  const int warps = BIG_SBT / 32;
  long long n = 3;
  k_bigs_bwd_pre<<<cnt, BIG_SBT, 0, st>>>(h->d, h->s, dl);
  k_bigs_bwd_anc<<<dim3((unsigned)std::max(1, (h->lvl_maxc[l] + warps - 1) / warps), cnt), BIG_SBT, 0, st>>>(h->d, h->s, dl);
  for (int jb = (h->lvl_maxc[l] - 1) / BIG_SBW * BIG_SBW; jb >= 0; jb -= BIG_SBW) {
    k_bigs_bwd_diag<<<cnt, BIG_SBT, 0, st>>>(h->d, h->s, dl, jb);
    ++n;
    if (jb > 0) {
      k_bigs_bwd_cols<<<dim3((unsigned)((jb + warps - 1) / warps), cnt), BIG_SBT, 0, st>>>(h->d, h->s, dl, jb);
      ++n;
    }
  }
  k_bigs_bwd_post<<<cnt, BIG_SBT, 0, st>>>(h->d, h->s, dl);
  return n;
}

nmpc_status launch_solve(nmpc_handle* h) {
  const int nl = (int)h->lvl_ptr.size() - 1;
  const int L = h->opt.solve_mode == 1 ? 0 : h->solve_prefix;  // levels covered by one persistent launch
  int* fwd_flags = h->d_solve_flags;                              // zero between launches
  int* bwd_flags = h->d_solve_flags + h->solve_prefix_fronts + 2;
  const int* list = nullptr;
  const int ns = (int)h->A.sn_first.size();
  if (L > 0 && h->front_lists) {  // only the fronts of the instances being solved (both directions)
    k_front_list<<<1, FL_THREADS, h->A.n_inst, h->stream>>>(h->d, h->s, h->solve_prefix_fronts, 1,
                                                             h->d_front_list + ns, h->d_front_cnt + 1);
    ++h->launches;
    list = h->d_front_list + ns;
  }
  if (L > 0) {
    k_fwd_persist<<<h->persist_blocks_fwd, 128, h->persist_smem_fwd, h->stream>>>(
        h->d, h->s, h->s.desc, h->solve_prefix_fronts, h->persist_stage_cap, fwd_flags, list, h->d_front_cnt + 1);
    ++h->launches;
  }
  for (int l = L; l < nl; ++l) {
    const int cnt = h->lvl_ptr[l + 1] - h->lvl_ptr[l];
    if (!cnt) continue;
    if (h->lvl_bigsolve[l]) {
      h->launches += launch_big_fwd(h, l);
    } else {
      k_fwd_level<<<cnt, 128, h->lvl_smem_solve[l], h->stream>>>(h->d, h->s, h->s.desc + h->lvl_ptr[l],
                                                                 h->smem_cap_doubles);
      ++h->launches;
    }
  }
  for (int l = nl - 1; l >= L; --l) {
    const int cnt = h->lvl_ptr[l + 1] - h->lvl_ptr[l];
    if (!cnt) continue;
    if (h->lvl_bigsolve[l]) {
      h->launches += launch_big_bwd(h, l);
    } else {
      k_bwd_level<<<cnt, 128, h->lvl_smem_bwd[l], h->stream>>>(h->d, h->s, h->s.desc + h->lvl_ptr[l],
                                                               h->smem_cap_doubles);
      ++h->launches;
    }
  }
  if (L > 0) {
    k_bwd_persist<<<h->persist_blocks_bwd, 128, h->persist_smem_bwd, h->stream>>>(
        h->d, h->s, h->s.desc, h->solve_prefix_fronts, h->persist_stage_cap, bwd_flags, list, h->d_front_cnt + 1);
    ++h->launches;
  }
  return NMPC_OK;
}

// Kernel sequences of one interior-point iteration (Algorithm 2), shared by
// the host-driven loop and the graph.  Each returns the number of launches.
long long seq_eval(nmpc_handle* h) {
  Dev& d = h->d;
  cudaStream_t st = h->stream;
  const int nbr = (int)blocks_for(d.m, EW);
  k_eval<<<nbr + blocks_for(d.n, EW), EW, 0, st>>>(d, 0, 1, nbr);
  k_red_eval<<<d.n_chunks, RED_CHUNK, 0, st>>>(d, h->opt.max_iter, h->cond);
  return 2;
}

long long seq_factor(nmpc_handle* h) {
  Dev& d = h->d;
  cudaStream_t st = h->stream;
  const int ni = h->A.n_inst;
  // zeroing blocks per instance: enough to spread one instance's panels over
  // the GPU, but at most about 8k blocks in all (the blocks of instances that
  // need no factorization leave at once, yet each still has to be scheduled)
  const int zx = (int)std::max(1u, std::min({1024u, blocks_for(h->A.nnzL / std::max(1, ni) + 1, EW),
                                             (unsigned)std::max(1, 8192 / std::max(1, ni))}));
  const long long l0 = h->launches;
  k_zero_rows<<<(unsigned)((long long)zx * ni + blocks_for(d.m, EW)), EW, 0, st>>>(d, h->d_inst_Lbeg, h->d_inst_Lend,
                                                                                    h->d_Drow, zx);
  long long rhs = 0;
  if (h->side) {
    // the solves' right-hand side needs the rows' terms, not the factor:
    // computed on the side stream during the factorization (joined with the
    // panel transforms before the inertia test)
    cudaEventRecord(h->ev_fork, st);
    cudaStreamWaitEvent(h->side, h->ev_fork, 0);
    k_rhs<<<blocks_for(d.n, EW), EW, 0, h->side>>>(d);
    h->side_pending = true;
    rhs = 1;
  }
  k_assemble<<<blocks_for(d.n_tgt, EW), EW, 0, st>>>(d, h->d_tgt_inst, h->d_Drow);
  launch_factor(h);
  k_ctl_factor<<<1, TPB, 0, st>>>(d, h->cond);
  const long long levels = h->launches - l0;
  h->launches = l0;
  return 3 + rhs + levels;
}

// Lifted-KKT: right-hand side, solves, recovery and step limits.  HyKKT:
// right-hand side g, u = K^-1 g, and the CG start (seq_cg and seq_solve2 follow).
long long seq_solve(nmpc_handle* h) {
  Dev& d = h->d;
  cudaStream_t st = h->stream;
  const long long l0 = h->launches;
  long long rhs = 0;
  if (!h->side) {  // otherwise computed during the factorization (seq_factor)
    k_rhs<<<blocks_for(d.n, EW), EW, 0, st>>>(d);
    rhs = 1;
  }
  launch_solve(h);
  if (d.mc.kkt == 1) k_red_cg0<<<d.n_chunks, RED_CHUNK, 0, st>>>(d, h->cond);
  else k_red_dir<<<d.n_chunks, RED_CHUNK, 0, st>>>(d, h->cond);  // recovery, step limits, control
  const long long levels = h->launches - l0;
  h->launches = l0;
  return 1 + rhs + levels;
}

// HyKKT: one conjugate-gradient step on S = H K^-1 H^T
long long seq_cg(nmpc_handle* h) {
  Dev& d = h->d;
  cudaStream_t st = h->stream;
  const long long l0 = h->launches;
  k_cg_apply<<<blocks_for(d.n, EW), EW, 0, st>>>(d);
  launch_solve(h);
  k_red_cg1<<<d.n_chunks, RED_CHUNK, 0, st>>>(d);
  k_red_cg2<<<d.n_chunks, RED_CHUNK, 0, st>>>(d, h->cond);
  const long long levels = h->launches - l0;
  h->launches = l0;
  return 3 + levels;
}

// HyKKT: dy = K^-1 (g - H^T dlam), then recovery and step limits
long long seq_solve2(nmpc_handle* h) {
  Dev& d = h->d;
  cudaStream_t st = h->stream;
  const long long l0 = h->launches;
  k_hy_rhs<<<blocks_for(d.n, EW), EW, 0, st>>>(d);
  launch_solve(h);
  k_red_dir<<<d.n_chunks, RED_CHUNK, 0, st>>>(d, h->cond);
  const long long levels = h->launches - l0;
  h->launches = l0;
  return 2 + levels;
}

long long seq_trial(nmpc_handle* h) {
  Dev& d = h->d;
  cudaStream_t st = h->stream;
  k_trial_point<<<blocks_for((long long)d.n + d.m), TPB, 0, st>>>(d);
  const int nbr = (int)blocks_for(d.m, EW);
  k_eval<<<nbr + blocks_for(d.n, EW), EW, 0, st>>>(d, 1, 0, nbr);
  k_red_trial<<<d.n_chunks, RED_CHUNK, 0, st>>>(d, h->cond);
  return 3;
}

long long seq_update(nmpc_handle* h) {
  Dev& d = h->d;
  // the step's bookkeeping (trace, filter, count) runs in the next
  // evaluation's control step
  k_update<<<blocks_for((long long)d.n + d.m, EW), EW, 0, h->stream>>>(d);
  return 1;
}

// Add a conditional node at the current point of a stream capture; the
// capture continues after it.  Returns the node's body graph.
cudaError_t capture_conditional(cudaStream_t cs, cudaGraphConditionalHandle hc, cudaGraphConditionalNodeType type,
                                cudaGraph_t* body) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = hc;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, cg, deps, nullptr, nd, &p);
  if (e != cudaSuccess) return e;
  *body = p.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// The interior-point loop (after the initialization kernels) as one graph:
//   WHILE any instance runs:
//     evaluate, errors, barrier update (k_red_eval: reduction, then control)
//     IF any instance runs:
//       WHILE any instance needs a factorization: assemble, factor, inertia test
//       right-hand side, solves, step recovery, step limits (k_red_dir)
//         (HyKKT: right-hand side, solves, CG start; WHILE any CG runs: one CG
//          step; then the final right-hand side, solves, recovery, step limits)
//       WHILE any line search is active: trial point, evaluate, filter test
//       accept the step
// The conditions are set on the device, so a solve needs no host round trip.
nmpc_status build_graph(nmpc_handle* h) {
  cudaStream_t cs = nullptr;
  CUDA_TRY(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaStream_t saved = h->stream;
  h->stream = cs;
  cudaGraph_t g = nullptr;
  const char* step = "create";
  cudaError_t e = cudaGraphCreate(&g, 0);
  int* ctr = h->d_flags + 8;
  // trip limits: outer steps, and factorization attempts / line-search trials
  // (64 per step: far above what the inertia correction and the backtracking
  // can take before they stop by themselves)
  const int cap_iter = h->opt.max_iter + 2, cap_inner = 64 * cap_iter;
  const int cap_cg = (std::max(0, h->opt.cg_max_iter) + 1) * cap_iter;
  const bool hy = h->d.mc.kkt == 1;
  cudaGraphConditionalHandle h_run = 0, h_if = 0, h_fac = 0, h_ls = 0, h_cg = 0;  // one per conditional node
  cudaGraph_t body_iter = nullptr, body_run = nullptr, body_fac = nullptr, body_ls = nullptr, body_cg = nullptr;
  // the step-ending kernels set the conditions (restored to off below)
  if (e == cudaSuccess) { step = "handles"; e = cudaGraphConditionalHandleCreate(&h_run, g, 1, cudaGraphCondAssignDefault); }
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h_if, g, 0, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h_fac, g, 0, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h_ls, g, 0, 0);
  if (e == cudaSuccess && hy) e = cudaGraphConditionalHandleCreate(&h_cg, g, 0, 0);
  if (e == cudaSuccess) {
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h_run;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    step = "outer while node";
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p);
    if (e == cudaSuccess) body_iter = p.conditional.phGraph_out[0];
  }
  h->cond = CondArgs{h_run, h_if, h_fac, h_ls, h_cg, ctr, cap_iter, cap_inner, cap_cg, 1};
  // iteration body: evaluation (k_red_eval sets the conditions), then IF running
  if (e == cudaSuccess) step = "capture iteration body";
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, body_iter, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    h->nodes_eval = seq_eval(h);
    step = "IF node";
    e = capture_conditional(cs, h_if, cudaGraphCondTypeIf, &body_run);
    cudaGraph_t out = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &out);
    if (e == cudaSuccess) e = e2;
  }
  // running: factorization loop, solves, line-search loop, update
  if (e == cudaSuccess) step = "capture running body";
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, body_run, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    step = "factor WHILE node";
    e = capture_conditional(cs, h_fac, cudaGraphCondTypeWhile, &body_fac);
    if (e == cudaSuccess) {
      h->nodes_solve = seq_solve(h);
      if (hy) {
        step = "CG WHILE node";
        e = capture_conditional(cs, h_cg, cudaGraphCondTypeWhile, &body_cg);
        if (e == cudaSuccess) h->nodes_solve2 = seq_solve2(h);
      }
    }
    if (e == cudaSuccess) {
      step = "line-search WHILE node";
      e = capture_conditional(cs, h_ls, cudaGraphCondTypeWhile, &body_ls);
    }
    if (e == cudaSuccess) h->nodes_update = seq_update(h);
    cudaGraph_t out = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &out);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) step = "capture factor body";
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, body_fac, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    h->nodes_factor = seq_factor(h);
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(cs, &out);
  }
  if (e == cudaSuccess && hy) {
    step = "capture CG body";
    e = cudaStreamBeginCaptureToGraph(cs, body_cg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      h->nodes_cg = seq_cg(h);
      cudaGraph_t out = nullptr;
      e = cudaStreamEndCapture(cs, &out);
    }
  }
  if (e == cudaSuccess) step = "capture line-search body";
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, body_ls, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    h->nodes_trial = seq_trial(h);
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(cs, &out);
  }
  h->cond = CondArgs{};
  cudaGraphExec_t ex = nullptr;
  if (e == cudaSuccess) step = "instantiate";
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
  h->stream = saved;
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return fail(h, NMPC_ERR_CUDA, std::string("building the interior-point graph (") + step + "): " + cudaGetErrorString(e));
  }
  h->graph = g;
  h->gexec = ex;
  return NMPC_OK;
}

}  // namespace

extern "C" {

void nmpc_problem_defaults(int model, nmpc_problem* p) {
  std::memset(p, 0, sizeof(*p));
  p->model = model;
  p->n_instances = 1;
  p->dt = 1.0;
  p->alpha = 1.6; p->D = 0.2; p->F = 0.4; p->xF = 0.5; p->Ac = 1.0; p->At = 1.0; p->Ar = 1.0; p->wdu = 0.01;
  p->kappa = 0.01; p->cq = 0.01; p->rho_u = 1e-3;
  if (model == NMPC_MODEL_DISTILLATION || model == NMPC_MODEL_DISTILLATION_DAE) {
    p->N = 12; p->Nf = 5; p->xlo = 0; p->xhi = 1; p->ulo = 1; p->uhi = 5;
  }
  else if (model == NMPC_MODEL_PLATE) { p->g = 64; p->S = 8; p->xlo = -INFINITY; p->xhi = 1.2; p->ulo = 0; p->uhi = 1; }
  else if (model == NMPC_MODEL_PAPER_PLATE) {  // table pde-params, Sec. 4.2
    p->g = 21; p->S = 1; p->dt = 0.08; p->kappa = 230.0; p->rho_u = 1e-8; p->Tb = 50.0; p->qloss = 10.0;
    p->xlo = -INFINITY; p->xhi = INFINITY; p->ulo = 50.0; p->uhi = INFINITY;
  }
  else { p->xlo = 0; p->xhi = INFINITY; p->ulo = 1; p->uhi = 3; }
}

void nmpc_options_defaults(nmpc_options* o) {
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-8; o->gamma = 1e-8; o->mu0_cold = 0.1; o->mu0_warm = 1e-8;
  o->push_cold = 1e-2; o->push_warm = 1e-9; o->max_iter = 200; o->ordering = NMPC_ORDER_AUTO;
  o->nd_leaf = 1; o->use_graph = 1; o->spin_limit = 10000000LL; o->pivtol = 1e-12;
  o->dw_max = 1e40;
  o->kkt = NMPC_KKT_LIFTED; o->hykkt_gamma = 1e4; o->cg_tol = 1e-12; o->cg_max_iter = 200;
}

nmpc_status nmpc_build(const nmpc_problem* prob, const nmpc_options* opts, void* cuda_stream, nmpc_handle** out) {
  if (!prob || !out || prob->n_instances < 1 || !prob->horizons) return NMPC_ERR_INVALID;
  *out = nullptr;
  nmpc_handle* h = new (std::nothrow) nmpc_handle();
  if (!h) return NMPC_ERR_INVALID;
  if (opts) h->opt = *opts;
  else nmpc_options_defaults(&h->opt);
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  ProblemSpec sp;
  sp.model = prob->model;
  sp.T.assign(prob->horizons, prob->horizons + prob->n_instances);
  sp.N = prob->N; sp.Nf = prob->Nf; sp.g = prob->g; sp.S = prob->S; sp.dt = prob->dt;
  sp.alpha = prob->alpha; sp.D = prob->D; sp.F = prob->F; sp.xF = prob->xF;
  sp.Ac = prob->Ac; sp.At = prob->At; sp.Ar = prob->Ar; sp.wdu = prob->wdu;
  sp.kappa = prob->kappa; sp.cq = prob->cq; sp.rho_u = prob->rho_u;
  sp.xlo = prob->xlo; sp.xhi = prob->xhi; sp.ulo = prob->ulo; sp.uhi = prob->uhi;
  sp.wu = prob->wu; sp.ubar = prob->ubar;
  sp.Tb = prob->Tb; sp.qloss = prob->qloss;
  sp.gamma = h->opt.gamma; sp.tol = h->opt.tol;
  sp.ordering = h->opt.ordering; sp.nd_leaf = h->opt.nd_leaf; sp.pivtol = h->opt.pivtol;
  sp.dw_max = h->opt.dw_max;
  sp.amalgamation = h->opt.amalgamation;
  if (!(prob->dt > 0) || h->opt.max_iter < 1 || !(h->opt.tol > 0) || !(h->opt.gamma > 0) || !(h->opt.dw_max > 0) ||
      (h->opt.kkt != NMPC_KKT_LIFTED && h->opt.kkt != NMPC_KKT_HYKKT) ||
      (h->opt.kkt == NMPC_KKT_HYKKT && (!(h->opt.hykkt_gamma > 0) || !(h->opt.cg_tol >= 0) || h->opt.cg_max_iter < 0))) {
    delete h;
    return NMPC_ERR_INVALID;
  }
  std::string e = analyze(sp, h->A);
  if (!e.empty()) {
    std::fprintf(stderr, "nmpc_build: %s\n", e.c_str());
    delete h;
    return NMPC_ERR_INVALID;
  }
  // the Newton-system form (the structure is the same for both)
  h->A.mc.kkt = h->opt.kkt;
  h->A.mc.hy_gamma = h->opt.hykkt_gamma;
  h->A.mc.cg_tol = h->opt.cg_tol;
  h->A.mc.cg_max_iter = h->opt.cg_max_iter;
  // per-level launch shapes
  const Analysis& A = h->A;
  h->lvl_ptr = A.level_ptr;
  const int nl = (int)A.level_ptr.size() - 1;
  h->smem_cap_doubles = SMEM_FACTOR_CAP_BYTES / 8;
  h->lvl_smem_factor.assign(nl, 8);
  h->lvl_smem_solve.assign(nl, 8);
  // per level: cluster size Q so that the level's fronts occupy most SMs, if
  // every front fits in shared memory with that Q
  {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) h->n_sm = prop.multiProcessorCount;
  }
  h->lvl_cluster.assign(nl, 0);
  h->lvl_cluster_smem.assign(nl, 0);
  // factor_mode 3: the longest prefix of levels whose fronts each fit one
  // k_factor_flow block runs as one dataflow launch; the levels above it as
  // in mode 0
  h->flow_levels = h->flow_fronts = h->flow_smem = 0;
  if (h->opt.factor_mode == 3) {
    int L = 0;
    long long worst = 0;
    for (; L < nl; ++L) {
      long long lw = 0;
      for (int qd = A.level_ptr[L]; qd < A.level_ptr[L + 1]; ++qd)
        lw = std::max(lw, flow_need(A.sn_nrow[A.level_sn[qd]], A.sn_ncol[A.level_sn[qd]]) * 8);
      if (lw > FLOW_SMEM_CAP_BYTES) break;
      worst = std::max(worst, lw);
    }
    h->flow_levels = L;
    h->flow_fronts = A.level_ptr[L];
    h->flow_smem = (int)std::max<long long>(worst, 8);
  }
  const bool clusters = h->opt.factor_mode == 0 || h->opt.factor_mode == 3;
  for (int l = 0; l < nl; ++l) {
    const int cnt = A.level_ptr[l + 1] - A.level_ptr[l];
    int max_blocks = 1;
    for (int qd = A.level_ptr[l]; qd < A.level_ptr[l + 1]; ++qd)
      max_blocks = std::max(max_blocks, (A.sn_nrow[A.level_sn[qd]] + CLUSTER_PB - 1) / CLUSTER_PB);
    int Q = 1;
    // clusters spread over the SMs (a second CTA per SM did not speed up the distillation levels)
    while (Q < 8 && 2 * Q * cnt <= h->cluster_ctas_per_sm * h->n_sm && 2 * Q <= max_blocks) Q *= 2;
    long long worst = 0;
    bool fits = true;
    for (int qd = A.level_ptr[l]; qd < A.level_ptr[l + 1] && fits; ++qd) {
      const int sn = A.level_sn[qd];
      const long long mm = A.sn_nrow[sn];
      const long long nblk = (mm + CLUSTER_PB - 1) / CLUSTER_PB;
      const long long ncl = (nblk + Q - 1) / Q * CLUSTER_PB;
      const long long need = mm * (ncl + 2 * CLUSTER_PB) + 2 * ncl;  // doubles (layout in k_factor_cluster)
      if (need * 8 > SMEM_FACTOR_CAP_BYTES) fits = false;
      worst = std::max(worst, need * 8);
    }
    if (fits && clusters && l >= h->flow_levels) { h->lvl_cluster[l] = Q; h->lvl_cluster_smem[l] = (int)worst; }
  }
  h->lvl_big.assign(nl, 0); h->lvl_bigsolve.assign(nl, 0);
  h->lvl_maxm.assign(nl, 0); h->lvl_maxc.assign(nl, 0); h->lvl_maxmu.assign(nl, 0);
  h->lvl_maxch.assign(nl, 0); h->lvl_maxmc.assign(nl, 0);
  for (int l = 0; l < nl; ++l) {
    for (int qd = A.level_ptr[l]; qd < A.level_ptr[l + 1]; ++qd) {
      const int J = A.level_sn[qd];
      const int mm = A.sn_nrow[J], cc = A.sn_ncol[J];
      h->lvl_maxm[l] = std::max(h->lvl_maxm[l], mm);
      h->lvl_maxc[l] = std::max(h->lvl_maxc[l], cc);
      h->lvl_maxmu[l] = std::max(h->lvl_maxmu[l], mm - cc);
      h->lvl_maxch[l] = std::max(h->lvl_maxch[l], A.sn_child_ptr[J + 1] - A.sn_child_ptr[J]);
      for (int k = A.sn_child_ptr[J]; k < A.sn_child_ptr[J + 1]; ++k) {
        const int C = A.sn_child[k];
        h->lvl_maxmc[l] = std::max(h->lvl_maxmc[l], A.sn_nrow[C] - A.sn_ncol[C]);
      }
      const long long lsz = ((long long)mm * cc + 1) & ~1LL;
      if (cc > 128 || lsz + mm + cc > h->smem_cap_doubles) h->lvl_bigsolve[l] = 1;
    }
    h->lvl_big[l] = ((h->lvl_cluster[l] == 0 && clusters && l >= h->flow_levels) || h->opt.factor_mode == 2) ? 1 : 0;
  }
  // update matrices: reuse the memory of those already consumed
  h->A.nU = plan_update_memory(h->A, h->flow_levels);
  // blocks of the fronts solved one block per front (fwd_front/bwd_front)
  h->inv_items.clear();
  h->scale_units.clear();
  h->lvl_inv_ptr.assign(nl + 1, 0);
  h->lvl_scale_ptr.assign(nl + 1, 0);
  // Solve form (SnDev::solve_form).  When the solves are latency-bound (at most
  // 4 fronts per SM in every level) the panels are transformed (form 2): the
  // transform takes about eight solves' worth of FP64 work per factorization,
  // hidden under the upper levels' factorization, and cuts the per-front
  // critical path 2-3x.  When they are throughput-bound (wide batches) the
  // plain substitution does the least work (form 0).
  int widest = 0;
  for (int l = 0; l < nl; ++l) widest = std::max(widest, A.level_ptr[l + 1] - A.level_ptr[l]);
  const int form = h->opt.panel_scale == 1 ? 2 : h->opt.panel_scale == 2 ? 1 : h->opt.panel_scale == 3 ? 0
                   : (widest <= 4 * h->n_sm ? 2 : 0);
  h->s_form = form;
  const bool scaled = form == 2;
  for (int l = 0; l < nl; ++l) {
    h->lvl_inv_ptr[l] = (int)h->inv_items.size();
    h->lvl_scale_ptr[l] = (int)h->scale_units.size();
    if (h->lvl_bigsolve[l] || form == 0) continue;
    for (int qd = A.level_ptr[l]; qd < A.level_ptr[l + 1]; ++qd) {
      const int J = A.level_sn[qd];
      const int mm = A.sn_nrow[J], cc = A.sn_ncol[J];
      for (int s0 = 0; s0 < cc; s0 += IB) {
        const int bk = std::min(IB, cc - s0);
        if (bk < 2) continue;
        const int rows = mm - s0 - bk;
        if (scaled)
          for (int r0 = 0; r0 < rows; r0 += 32) h->scale_units.push_back({(int)h->inv_items.size(), r0});
        h->inv_items.push_back({A.sn_Lptr[J] + s0 + (long long)s0 * mm, mm, bk, A.sn_inst[J], rows});
      }
    }
  }
  h->lvl_inv_ptr[nl] = (int)h->inv_items.size();
  h->lvl_scale_ptr[nl] = (int)h->scale_units.size();
  h->lvl_smem_bwd.assign(nl, 8);
  for (int l = 0; l < nl; ++l)
    for (int q = A.level_ptr[l]; q < A.level_ptr[l + 1]; ++q) {
      const int sn = A.level_sn[q];
      const long long mm = A.sn_nrow[sn], cc = A.sn_ncol[sn];
      const long long need = mm * mm + mm;  // whole front plus one unscaled column
      h->lvl_smem_factor[l] = std::max<int>(h->lvl_smem_factor[l], (int)((need <= h->smem_cap_doubles ? need : mm) * 8));
      const long long lsz = (mm * cc + 1) & ~1LL;  // staged panel (k_fwd_level / k_bwd_level)
      if (h->lvl_bigsolve[l]) continue;           // the large-front solves size their own
      const long long sneed = (lsz + mm + cc <= h->smem_cap_doubles) ? lsz + mm + cc : mm + cc;
      h->lvl_smem_solve[l] = std::max<int>(h->lvl_smem_solve[l], (int)(sneed * 8));
      h->lvl_smem_bwd[l] = std::max<int>(h->lvl_smem_bwd[l], (int)(sneed * 8));
    }
  // extend-add maps of the cluster levels: for every front, cluster CTA q and
  // child k, the (source in the child's update matrix, destination in the
  // CTA's own columns) pairs of the entries that land in q's columns
  h->desc_abase.assign(A.level_sn.size(), -1);
  h->desc_wptr.assign(A.level_sn.size(), 0);
  h->nW_cluster = 0;
  for (int l = 0; l < nl; ++l) {
    if (h->lvl_cluster[l] <= 0) continue;
    for (int qd = A.level_ptr[l]; qd < A.level_ptr[l + 1]; ++qd) {
      const int J = A.level_sn[qd];
      h->desc_wptr[qd] = h->nW_cluster;
      h->nW_cluster += (A.sn_Lptr[J + 1] - A.sn_Lptr[J]);  // same padded size as the panel
    }
  }
  h->amap.clear();
  h->amap_ptr.clear();
  {
    // per front (on several host threads), then concatenated in level order
    struct FrontMap {
      std::vector<int> pairs;        // (source, destination) pairs
      std::vector<long long> ptr;    // pair offsets of each (CTA, child) range, relative
    };
    std::vector<int> fronts;  // level positions of the cluster-factored fronts
    for (int l = 0; l < nl; ++l)
      if (h->lvl_cluster[l] > 0)
        for (int qd = A.level_ptr[l]; qd < A.level_ptr[l + 1]; ++qd) fronts.push_back(qd);
    std::vector<int> lvl_of(A.level_sn.size(), 0);
    for (int l = 0; l < nl; ++l)
      for (int qd = A.level_ptr[l]; qd < A.level_ptr[l + 1]; ++qd) lvl_of[qd] = l;
    std::vector<FrontMap> fm(fronts.size());
    parallel_for((int)fronts.size(), [&](int f) {
      const int qd = fronts[f], Q = h->lvl_cluster[lvl_of[qd]];
      const int J = A.level_sn[qd];
      const int m = A.sn_nrow[J];
      FrontMap& M = fm[f];
      for (int q = 0; q < Q; ++q) {
        for (int k = A.sn_child_ptr[J]; k < A.sn_child_ptr[J + 1]; ++k) {
          M.ptr.push_back((long long)M.pairs.size() / 2);
          const int C = A.sn_child[k];
          const int mc = A.sn_nrow[C] - A.sn_ncol[C];
          const int* rel = A.sn_rel.data() + A.sn_relptr[C];
          for (int b = 0; b < mc; ++b) {
            const int rb = rel[b];
            if ((rb / CLUSTER_PB) % Q != q) continue;
            const int lc = ((rb / CLUSTER_PB) / Q) * CLUSTER_PB + rb % CLUSTER_PB;
            for (int a = b; a < mc; ++a) {
              M.pairs.push_back(a + b * mc);
              M.pairs.push_back(rel[a] + lc * m);
            }
          }
        }
        M.ptr.push_back((long long)M.pairs.size() / 2);
      }
    });
    for (size_t f = 0; f < fronts.size(); ++f) {
      const long long base = (long long)h->amap.size() / 2;
      h->desc_abase[fronts[f]] = (long long)h->amap_ptr.size();
      for (long long o : fm[f].ptr) h->amap_ptr.push_back(base + o);
      h->amap.insert(h->amap.end(), fm[f].pairs.begin(), fm[f].pairs.end());
    }
  }
  Carver cv;
  carve(h, cv);
  h->ws_bytes = (cv.off + 255) & ~size_t(255);
  *out = h;
  return NMPC_OK;
}

nmpc_status nmpc_workspace_bytes(const nmpc_handle* h, size_t* bytes) {
  if (!h || !bytes) return NMPC_ERR_INVALID;
  *bytes = h->ws_bytes;
  return NMPC_OK;
}

}  // extern "C"

namespace {

// Lay the workspace out, clear it and upload the structure (shared by the
// binding entry points).
nmpc_status upload_structure(nmpc_handle* h, void* ws) {
  Carver cv;
  cv.base = static_cast<char*>(ws);
  carve(h, cv);
  const Analysis& A = h->A;
  Dev& d = h->d;
  SnDev& s = h->s;
  cudaStream_t st = h->stream;
  std::vector<Chunk> ch = A.chunks;
  CUDA_TRY(h, cudaMemsetAsync(ws, 0, h->ws_bytes, st));
  CUDA_TRY(h, up(d.inst_T, A.inst_T, st)); CUDA_TRY(h, up(d.inst_voff, A.inst_voff, st));
  {
    std::vector<int> spoff(A.n_inst + 1, 0);
    for (int i = 0; i < A.n_inst; ++i) spoff[i + 1] = spoff[i] + (A.mc.model == MODEL_PLATE ? A.mc.nx : A.inst_T[i]);  // per stage otherwise
    h->sp_packed = spoff[A.n_inst];
    CUDA_TRY(h, cudaMemcpyAsync(h->d_inst_spoff, spoff.data(), spoff.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    CUDA_TRY(h, cudaStreamSynchronize(st));  // spoff is a local
  }
  CUDA_TRY(h, up(d.inst_roff, A.inst_roff, st)); CUDA_TRY(h, up(d.inst_woff, A.inst_woff, st));
  CUDA_TRY(h, up(d.inst_n, A.inst_n, st)); CUDA_TRY(h, up(d.inst_m, A.inst_m, st));
  CUDA_TRY(h, up(d.inst_nz, A.inst_nz, st));
  CUDA_TRY(h, up(d.var_inst, A.var_inst, st)); CUDA_TRY(h, up(d.row_inst, A.row_inst, st));
  CUDA_TRY(h, up(d.yL, A.yL, st)); CUDA_TRY(h, up(d.yU, A.yU, st));
  CUDA_TRY(h, up(d.Hcol, A.Hcol, st)); CUDA_TRY(h, up(d.Hcsc_ptr, A.Hcsc_ptr, st));
  CUDA_TRY(h, up(d.Hcsc_slot, A.Hcsc_slot, st));
  CUDA_TRY(h, up(d.Wadj_ptr, A.Wadj_ptr, st)); CUDA_TRY(h, up(d.Wadj_slot, A.Wadj_slot, st));
  CUDA_TRY(h, up(d.Wadj_other, A.Wadj_other, st));
  CUDA_TRY(h, up(d.perm, A.perm, st)); CUDA_TRY(h, up(d.iperm, A.iperm, st));
  {
    std::vector<int> hpos(A.Hcol.size());
    for (size_t q = 0; q < hpos.size(); ++q) hpos[q] = A.Hcol[q] >= 0 ? A.perm[A.Hcol[q]] : -1;
    CUDA_TRY(h, up(d.Hpos, hpos, st));
    CUDA_TRY(h, cudaStreamSynchronize(st));  // hpos goes out of scope
  }
  CUDA_TRY(h, up(d.chunks, ch, st)); CUDA_TRY(h, up(d.inst_chunk_ptr, A.inst_chunk_ptr, st));
  CUDA_TRY(h, up(d.red_var, A.red_var, st));
  CUDA_TRY(h, up(d.inst_chunk_list, A.inst_chunk_list, st));
  CUDA_TRY(h, up(d.tgt_L, A.tgt_L, st)); CUDA_TRY(h, up(d.tgt_diag, A.tgt_diag, st));
  CUDA_TRY(h, up(d.tw_ptr, A.tw_ptr, st)); CUDA_TRY(h, up(d.tw_idx, A.tw_idx, st));
  CUDA_TRY(h, up(d.th_ptr, A.th_ptr, st)); CUDA_TRY(h, up(d.th_a, A.th_a, st)); CUDA_TRY(h, up(d.th_b, A.th_b, st));
  CUDA_TRY(h, up(d.sn_inst, A.sn_inst, st));
  // instance of each assembly target and L range of each instance
  std::vector<int> tinst(A.tgt_L.size());
  std::vector<long long> lb(A.n_inst, 0), le(A.n_inst, 0);
  {
    std::vector<int> first_sn(A.n_inst, -1), last_sn(A.n_inst, -1);
    for (int q = 0; q < (int)A.sn_first.size(); ++q) {
      const int i = A.sn_inst[q];
      if (first_sn[i] < 0) first_sn[i] = q;
      last_sn[i] = q;
    }
    for (int i = 0; i < A.n_inst; ++i) { lb[i] = A.sn_Lptr[first_sn[i]]; le[i] = A.sn_Lptr[last_sn[i] + 1]; }
    size_t i = 0;
    for (size_t t = 0; t < A.tgt_L.size(); ++t) {
      while (A.tgt_L[t] >= le[i]) ++i;
      tinst[t] = (int)i;
    }
  }
  CUDA_TRY(h, up(h->d_tgt_inst, tinst, st));
  CUDA_TRY(h, up(h->d_inst_Lbeg, lb, st)); CUDA_TRY(h, up(h->d_inst_Lend, le, st));
  CUDA_TRY(h, up(s.sn_first, A.sn_first, st)); CUDA_TRY(h, up(s.sn_ncol, A.sn_ncol, st));
  CUDA_TRY(h, up(s.sn_nrow, A.sn_nrow, st)); CUDA_TRY(h, up(s.sn_Lptr, A.sn_Lptr, st));
  CUDA_TRY(h, up(s.sn_Uptr, A.sn_Uptr, st)); CUDA_TRY(h, up(s.sn_rowptr, A.sn_rowptr, st));
  CUDA_TRY(h, up(s.sn_rows, A.sn_rows, st)); CUDA_TRY(h, up(s.sn_child_ptr, A.sn_child_ptr, st));
  CUDA_TRY(h, up(s.sn_child, A.sn_child, st)); CUDA_TRY(h, up(s.sn_relptr, A.sn_relptr, st));
  CUDA_TRY(h, up(s.sn_rel, A.sn_rel, st)); CUDA_TRY(h, up(s.level_ptr, A.level_ptr, st));
  CUDA_TRY(h, up(s.level_sn, A.level_sn, st)); CUDA_TRY(h, up(s.sn_uvptr, A.sn_uvptr, st));
  {
    std::vector<FrontDesc> desc(A.level_sn.size());
    std::vector<int> pos_of(A.level_sn.size());
    for (size_t q = 0; q < A.level_sn.size(); ++q) pos_of[A.level_sn[q]] = (int)q;
    CUDA_TRY(h, up(s.pos_of_sn, pos_of, st));
    std::vector<int> finst(A.level_sn.size());
    for (size_t q = 0; q < A.level_sn.size(); ++q) finst[q] = A.sn_inst[A.level_sn[q]];
    CUDA_TRY(h, up(s.front_inst, finst, st));
    CUDA_TRY(h, cudaStreamSynchronize(st));  // finst goes out of scope
    for (size_t q = 0; q < A.level_sn.size(); ++q) {
      const int J = A.level_sn[q];
      FrontDesc& f = desc[q];
      std::memset(&f, 0, sizeof(f));
      f.J = J; f.m = A.sn_nrow[J]; f.c = A.sn_ncol[J]; f.first = A.sn_first[J]; f.inst = A.sn_inst[J];
      f.Lptr = A.sn_Lptr[J]; f.Uptr = A.sn_Uptr[J]; f.uvptr = A.sn_uvptr[J]; f.rowptr = A.sn_rowptr[J];
      f.nchild = A.sn_child_ptr[J + 1] - A.sn_child_ptr[J];
      f.abase = h->desc_abase[q];
      f.Wptr = h->desc_wptr[q];
      f.pos = (int)q;
      f.par_pos = A.sn_parent[J] >= 0 ? pos_of[A.sn_parent[J]] : -1;
      for (int k = 0; k < std::min(f.nchild, DESC_CH); ++k) {
        const int C = A.sn_child[A.sn_child_ptr[J] + k];
        f.ch_mc[k] = A.sn_nrow[C] - A.sn_ncol[C];
        f.ch_relptr[k] = A.sn_relptr[C]; f.ch_Uptr[k] = A.sn_Uptr[C]; f.ch_uvptr[k] = A.sn_uvptr[C];
        f.ch_pos[k] = pos_of[C];
      }
    }
    CUDA_TRY(h, up(s.desc, desc, st));
    if (!h->amap.empty())
      CUDA_TRY(h, cudaMemcpyAsync(const_cast<IdxPair*>(s.amap), h->amap.data(), h->amap.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    CUDA_TRY(h, up(s.amap_ptr, h->amap_ptr, st));
    CUDA_TRY(h, up(s.inv, h->inv_items, st));
    CUDA_TRY(h, up(s.scale, h->scale_units, st));
    CUDA_TRY(h, cudaStreamSynchronize(st));  // the host vector goes out of scope
  }
  CUDA_TRY(h, cudaFuncSetAttribute(k_factor_level, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_FACTOR_CAP_BYTES));
  CUDA_TRY(h, cudaFuncSetAttribute(k_factor_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_FACTOR_CAP_BYTES));
  if (h->flow_fronts > 0) {
    CUDA_TRY(h, cudaFuncSetAttribute(k_factor_flow, cudaFuncAttributeMaxDynamicSharedMemorySize, FLOW_SMEM_CAP_BYTES));
    int per_sm = 0;
    CUDA_TRY(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_factor_flow, CLUSTER_THREADS, h->flow_smem));
    h->flow_blocks = std::max(1, std::min(h->flow_fronts, std::max(1, per_sm) * h->n_sm));
  }
  // persistent solves: the longest prefix of levels without large fronts
  {
    int L = 0, nf = 0, smf = 8, smb = 8;
    while (L < (int)h->lvl_bigsolve.size() && !h->lvl_bigsolve[L]) {
      nf += A.level_ptr[L + 1] - A.level_ptr[L];
      smf = std::max(smf, h->lvl_smem_solve[L]);
      smb = std::max(smb, h->lvl_smem_bwd[L]);
      ++L;
    }
    h->solve_prefix = L;
    h->solve_prefix_fronts = nf;
    // A batch's persistent solves stage only the panels of up to
    // PERSIST_STAGE_CAP bytes (the rest read their panel from global memory):
    // the launch's shared memory is its largest staged panel's, and one level
    // of large fronts would otherwise hold every level to its occupancy.
    h->persist_stage_cap = h->smem_cap_doubles;
    if (h->front_lists) {
      h->persist_stage_cap = PERSIST_STAGE_CAP / 8;
      smf = smb = 8;
      for (int q = 0; q < nf; ++q) {
        const int sn = A.level_sn[q];
        const long long mm = A.sn_nrow[sn], cc = A.sn_ncol[sn], lsz = (mm * cc + 1) & ~1LL;
        const long long tsz = (cc * cc + 1) & ~1LL;  // the triangle alone (column substitution)
        const long long need = (lsz + mm + cc <= h->persist_stage_cap) ? lsz + mm + cc
                               : (h->s_form == 0 && cc <= 128 && tsz + mm + cc <= h->persist_stage_cap) ? tsz + mm + cc
                                                                                                          : mm + cc;
        smf = smb = std::max<int>(smf, (int)(need * 8));
      }
    }
    h->persist_smem_fwd = smf;
    h->persist_smem_bwd = smb;
    if (smf > 48 * 1024) CUDA_TRY(h, cudaFuncSetAttribute(k_fwd_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, smf));
    if (smb > 48 * 1024) CUDA_TRY(h, cudaFuncSetAttribute(k_bwd_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, smb));
    int bf = 0, bb = 0;
    CUDA_TRY(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bf, k_fwd_persist, 128, smf));
    CUDA_TRY(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bb, k_bwd_persist, 128, smb));
    h->persist_blocks_fwd = std::max(1, std::min(nf, std::max(1, bf) * h->n_sm));
    h->persist_blocks_bwd = std::max(1, std::min(nf, std::max(1, bb) * h->n_sm));
  }
  const int maxf = *std::max_element(h->lvl_smem_solve.begin(), h->lvl_smem_solve.end());
  const int maxb = *std::max_element(h->lvl_smem_bwd.begin(), h->lvl_smem_bwd.end());
  if (maxf > 48 * 1024) CUDA_TRY(h, cudaFuncSetAttribute(k_fwd_level, cudaFuncAttributeMaxDynamicSharedMemorySize, maxf));
  if (maxb > 48 * 1024) CUDA_TRY(h, cudaFuncSetAttribute(k_bwd_level, cudaFuncAttributeMaxDynamicSharedMemorySize, maxb));
  CUDA_TRY(h, cudaStreamSynchronize(st));
  h->d.max_iter = h->opt.max_iter;
  h->h_ctl.resize(A.n_inst);
  return NMPC_OK;
}

}  // namespace

extern "C" {

nmpc_status nmpc_bind(nmpc_handle* h, void* ws, size_t bytes) {
  if (!h) return NMPC_ERR_INVALID;
  if (h->bound) return fail(h, NMPC_ERR_INVALID, "workspace already bound");
  if (!ws || bytes < h->ws_bytes) return fail(h, NMPC_ERR_WORKSPACE, "workspace missing or smaller than nmpc_workspace_bytes");
  if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(h, NMPC_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  const nmpc_status st = upload_structure(h, ws);
  if (st != NMPC_OK) return st;
  CUDA_TRY(h, cudaMallocHost(&h->h_flags, 4 * sizeof(int)));
  CUDA_TRY(h, cudaEventCreate(&h->ev0));
  CUDA_TRY(h, cudaEventCreate(&h->ev1));
  CUDA_TRY(h, cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
  CUDA_TRY(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  CUDA_TRY(h, cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  h->bound = true;
  return NMPC_OK;
}

nmpc_status nmpc_set_params(nmpc_handle* h, int instance, const double* x0, const double* setpoint,
                            const double* u_prev, int on_device) {
  if (!h || !h->bound) return fail(h, NMPC_ERR_INVALID, "handle not bound");
  const Analysis& A = h->A;
  if (instance < -1 || instance >= A.n_inst) return fail(h, NMPC_ERR_INVALID, "instance out of range");
  const int i0 = instance < 0 ? 0 : instance, i1 = instance < 0 ? A.n_inst : instance + 1;
  const int cnt = i1 - i0, nx = A.mc.nx;
  // setpoint values per instance as the caller packs them
  int sp_len = A.sp_stride;
  bool packed = false;  // all instances, unequal horizons: T_i setpoints each, one after another
  if (A.mc.model != MODEL_PLATE) {
    for (int i = i0; i < i1; ++i)
      if (A.inst_T[i] != A.inst_T[i0]) packed = true;
    sp_len = A.inst_T[i0];
  }
  if (packed) {
    const double *sx = x0, *ss = setpoint, *su = u_prev;
    if (!on_device) {
      double* p = h->d_stage;  // nx + sp_stride + 1 doubles per instance: room for the packed setpoints
      if (x0) { CUDA_TRY(h, cudaMemcpyAsync(p, x0, (size_t)cnt * nx * 8, cudaMemcpyHostToDevice, h->stream)); sx = p; }
      p += (size_t)cnt * nx;
      if (setpoint) { CUDA_TRY(h, cudaMemcpyAsync(p, setpoint, (size_t)h->sp_packed * 8, cudaMemcpyHostToDevice, h->stream)); ss = p; }
      p += h->sp_packed;
      if (u_prev) { CUDA_TRY(h, cudaMemcpyAsync(p, u_prev, (size_t)cnt * 8, cudaMemcpyHostToDevice, h->stream)); su = p; }
    }
    k_set_params_packed<<<cnt, TPB, 0, h->stream>>>(h->d, h->d_inst_spoff, sx, ss, su);
    ++h->launches;
    CUDA_TRY(h, cudaGetLastError());
    if (!on_device) CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return NMPC_OK;
  }
  const double *sx = x0, *ss = setpoint, *su = u_prev;
  if (!on_device) {
    // host arrays go through the workspace's staging area (sized for all instances)
    double* p = h->d_stage;
    if (x0) { CUDA_TRY(h, cudaMemcpyAsync(p, x0, (size_t)cnt * nx * 8, cudaMemcpyHostToDevice, h->stream)); sx = p; }
    p += (size_t)cnt * nx;
    if (setpoint) { CUDA_TRY(h, cudaMemcpyAsync(p, setpoint, (size_t)cnt * sp_len * 8, cudaMemcpyHostToDevice, h->stream)); ss = p; }
    p += (size_t)cnt * sp_len;
    if (u_prev) { CUDA_TRY(h, cudaMemcpyAsync(p, u_prev, (size_t)cnt * 8, cudaMemcpyHostToDevice, h->stream)); su = p; }
  }
  const long long total = (long long)cnt * (nx + sp_len + 1);
  k_set_params<<<std::min<long long>(blocks_for(total), 1024), TPB, 0, h->stream>>>(h->d, i0, i1, sx, ss, su, sp_len);
  ++h->launches;
  CUDA_TRY(h, cudaGetLastError());
  if (!on_device) CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return NMPC_OK;
}

nmpc_status nmpc_solve(nmpc_handle* h, int warm, nmpc_info* info) {
  if (!h || !h->bound) return fail(h, NMPC_ERR_INVALID, "handle not bound");
  if (warm && !h->have_solution) warm = 0;
  Dev& d = h->d;
  const Analysis& A = h->A;
  cudaStream_t st = h->stream;
  const int ni = A.n_inst, n = A.n, m = A.m;
  const double mu0 = warm ? h->opt.mu0_warm : h->opt.mu0_cold;
  const double push = warm ? h->opt.push_warm : h->opt.push_cold;
  if (h->ev0) CUDA_TRY(h, cudaEventRecord(h->ev0, st));
  CUDA_TRY(h, cudaMemsetAsync(h->d_flags + 3, 0, sizeof(int), st));
  k_ctl_init<<<blocks_for(ni), TPB, 0, st>>>(d, mu0);
  ++h->launches;
  k_init_vars<<<blocks_for(n, EW), EW, 0, st>>>(d, warm, push);
  ++h->launches;
  k_eval_rows<<<blocks_for(m, EW), EW, 0, st>>>(d, 0, 0);
  ++h->launches;
  k_init_rows<<<blocks_for(m, EW), EW, 0, st>>>(d, warm, push);
  ++h->launches;
  CUDA_TRY(h, cudaGetLastError());
  if (h->opt.use_graph && !h->graph_off) {
    if (!h->gexec) {
      const nmpc_status gs = build_graph(h);
      if (gs != NMPC_OK) return gs;
    }
    CUDA_TRY(h, cudaMemsetAsync(h->d_flags + 8, 0, 4 * sizeof(int), st));
    CUDA_TRY(h, cudaGraphLaunch(h->gexec, st));
    int ctr[5] = {0, 0, 0, 0, 0};
    CUDA_TRY(h, cudaMemcpyAsync(ctr, h->d_flags + 8, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(h, cudaMemcpyAsync(ctr + 4, h->d_flags + 3, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(h, cudaStreamSynchronize(st));
    // kernels the graph ran: outer steps x evaluation, running steps x (solve +
    // update), factorization attempts, line-search trials, CG steps
    const long long running = std::max(0, ctr[0] - 1);
    h->launches += (long long)ctr[0] * h->nodes_eval +
                   running * (h->nodes_solve + h->nodes_solve2 + h->nodes_update) +
                   (long long)ctr[1] * h->nodes_factor + (long long)ctr[2] * h->nodes_trial +
                   (long long)ctr[3] * h->nodes_cg;
    if (ctr[4]) return fail(h, NMPC_TIMEOUT, "a bounded wait between the CTAs of a front factorization ran out");
  } else {
    for (int it = 0; it <= h->opt.max_iter + 1; ++it) {
      h->launches += seq_eval(h);
      nmpc_status rs = read_flags(h);
      if (rs != NMPC_OK) return rs;
      if (!h->h_flags[0]) break;
      for (;;) {
        h->launches += seq_factor(h);
        CUDA_TRY(h, cudaGetLastError());
        rs = read_flags(h);
        if (rs != NMPC_OK) return rs;
        if (!h->h_flags[1]) break;
      }
      h->launches += seq_solve(h);
      CUDA_TRY(h, cudaGetLastError());
      if (d.mc.kkt == 1) {
        // HyKKT: CG steps until every instance's CG has stopped (each stops
        // after at most cg_max_iter steps), then the final solve
        for (;;) {
          rs = read_flags(h, 1);
          if (rs != NMPC_OK) return rs;
          if (!h->h_flags[2]) break;
          h->launches += seq_cg(h);
          CUDA_TRY(h, cudaGetLastError());
        }
        h->launches += seq_solve2(h);
        CUDA_TRY(h, cudaGetLastError());
      }
      rs = read_flags(h);
      if (rs != NMPC_OK) return rs;
      while (h->h_flags[2]) {
        h->launches += seq_trial(h);
        CUDA_TRY(h, cudaGetLastError());
        rs = read_flags(h);
        if (rs != NMPC_OK) return rs;
      }
      h->launches += seq_update(h);
    }
  }
  if (h->ev1) CUDA_TRY(h, cudaEventRecord(h->ev1, st));
  CUDA_TRY(h, cudaMemcpyAsync(h->h_ctl.data(), d.ctl, ni * sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(h, cudaStreamSynchronize(st));
  float ms = 0.f;
  if (h->ev0 && h->ev1) cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  h->have_solution = true;
  nmpc_status ret = NMPC_OK;
  for (int i = 0; i < ni; ++i) {
    const Ctl& c = h->h_ctl[i];
    const int stt = (c.status == ST_CONVERGED) ? NMPC_OK : (c.status == ST_RUNNING ? NMPC_MAX_ITER : c.status);
    if (stt != NMPC_OK && ret == NMPC_OK) ret = (nmpc_status)stt;
    if (info) {
      nmpc_info& o = info[i];
      o.status = stt; o.iters = c.iter; o.inertia_retries = c.inertia_retries; o.ls_trials = c.ls_trials;
      o.mu_final = c.mu; o.kkt_scaled = c.E0; o.kkt_unscaled = c.E0u; o.objective = c.f; o.ms_total = ms;
      o.cg_iters = c.cg_total;
    }
  }
  return ret;
}

nmpc_status nmpc_get_solution(nmpc_handle* h, int instance, double* y, double* duals, int on_device) {
  if (!h || !h->bound) return fail(h, NMPC_ERR_INVALID, "handle not bound");
  const Analysis& A = h->A;
  if (instance < -1 || instance >= A.n_inst) return fail(h, NMPC_ERR_INVALID, "instance out of range");
  if (!h->have_solution) return fail(h, NMPC_NOT_SOLVED, "no solution yet");
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  // instance -1: every instance, packed one after another (the workspace's own layout)
  const int vo = instance < 0 ? 0 : A.inst_voff[instance], ro = instance < 0 ? 0 : A.inst_roff[instance];
  const int n = instance < 0 ? A.n : A.inst_n[instance], m = instance < 0 ? A.m : A.inst_m[instance];
  const Dev& d = h->d;
  if (y) CUDA_TRY(h, cudaMemcpyAsync(y, d.y + vo, n * 8, k, h->stream));
  if (duals) {
    double* p = duals;
    const double* src[8] = {d.zL + vo, d.zU + vo, d.sp + ro, d.sm + ro, d.wp + ro, d.wm + ro, d.bp + ro, d.bm + ro};
    const int len[8] = {n, n, m, m, m, m, m, m};
    for (int q = 0; q < 8; ++q) { CUDA_TRY(h, cudaMemcpyAsync(p, src[q], (size_t)len[q] * 8, k, h->stream)); p += len[q]; }
  }
  if (!on_device) CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return NMPC_OK;
}

nmpc_status nmpc_set_start(nmpc_handle* h, int instance, const double* y, const double* duals, int on_device) {
  if (!h || !h->bound) return fail(h, NMPC_ERR_INVALID, "handle not bound");
  const Analysis& A = h->A;
  if (instance < -1 || instance >= A.n_inst) return fail(h, NMPC_ERR_INVALID, "instance out of range");
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  // instance -1: every instance, packed as nmpc_get_solution(-1) returns them
  const int vo = instance < 0 ? 0 : A.inst_voff[instance], ro = instance < 0 ? 0 : A.inst_roff[instance];
  const int n = instance < 0 ? A.n : A.inst_n[instance], m = instance < 0 ? A.m : A.inst_m[instance];
  const Dev& d = h->d;
  if (y) CUDA_TRY(h, cudaMemcpyAsync(d.y + vo, y, n * 8, k, h->stream));
  if (duals) {
    const double* p = duals;
    double* dst[8] = {d.zL + vo, d.zU + vo, d.sp + ro, d.sm + ro, d.wp + ro, d.wm + ro, d.bp + ro, d.bm + ro};
    const int len[8] = {n, n, m, m, m, m, m, m};
    for (int q = 0; q < 8; ++q) { CUDA_TRY(h, cudaMemcpyAsync(dst[q], p, (size_t)len[q] * 8, k, h->stream)); p += len[q]; }
  }
  if (!on_device) CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  h->have_solution = true;
  return NMPC_OK;
}

int nmpc_get_trace(nmpc_handle* h, int instance, double* out, int cap) {
  if (!h || !h->bound || instance < 0 || instance >= h->A.n_inst || !h->have_solution) return -1;
  const int iters = std::min(h->h_ctl[instance].iter, h->opt.max_iter + 1);
  const int cnt = std::min(cap, iters);
  if (out && cnt > 0) {
    if (cudaMemcpyAsync(out, h->d.trace + (size_t)instance * (h->opt.max_iter + 2) * 8, (size_t)cnt * 8 * sizeof(double),
                        cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return -1;
  }
  return iters;
}

nmpc_status nmpc_sensitivity(nmpc_handle* h, int instance, const double* dloss_dy, double* dloss_dx0,
                             double* dloss_dsp, int on_device) {
  if (!h || !h->bound) return fail(h, NMPC_ERR_INVALID, "handle not bound");
  const Analysis& A = h->A;
  if (instance < 0 || instance >= A.n_inst || !dloss_dy) return fail(h, NMPC_ERR_INVALID, "bad instance or gradient");
  if (!h->have_solution) return fail(h, NMPC_NOT_SOLVED, "no converged point");
  if (A.mc.kkt != NMPC_KKT_LIFTED) return fail(h, NMPC_ERR_INVALID, "the adjoint needs the Lifted-KKT form");
  Dev& d = h->d;
  cudaStream_t st = h->stream;
  const int ni = A.n_inst, n = A.n, m = A.m;
  const int vo = A.inst_voff[instance], ni_n = A.inst_n[instance];
  const int nx = A.mc.nx;
  const int sp_len = (A.mc.model == MODEL_PLATE) ? nx : A.inst_T[instance];
  const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  double* g = d.fvart;   // natural-order right-hand side (free between solves)
  double* x = d.dy;      // adjoint solution v
  double* r = d.yt;      // refinement residual
  double* t = d.rowv;    // per-row products
  double* ta = d.dwp;    // their absolute values (backward error)
  double* sc = d.dzL;    // (|K||x|)_v + |g_v|
  CUDA_TRY(h, cudaMemcpyAsync(h->d_ctl_save, d.ctl, ni * sizeof(Ctl), cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(h, cudaMemsetAsync(h->d_flags + 3, 0, sizeof(int), st));
  k_ctl_select<<<blocks_for(ni), TPB, 0, st>>>(d.ctl, ni, instance, 0);
  ++h->launches;
  // residual data at the converged point
  k_eval_rows<<<blocks_for(m, EW), EW, 0, st>>>(d, 0, 1);
  k_eval_vars<<<blocks_for(n, EW), EW, 0, st>>>(d, 0);
  k_rows_pre<<<blocks_for(m, EW), EW, 0, st>>>(d, h->d_Drow);
  h->launches += 3;
  CUDA_TRY(h, cudaMemsetAsync(g, 0, (size_t)n * sizeof(double), st));
  CUDA_TRY(h, cudaMemcpyAsync(g + vo, dloss_dy, (size_t)ni_n * sizeof(double), kin, st));
  // v = K_f^{-1} g, then refinement sweeps v += K_f^{-1} (g - K(z*) v) with the
  // stored factor K_f; if the componentwise backward error stays above 1e-12
  // (the slack weights changed too much in the last step), K(z*) is
  // refactored in place (same symbolic analysis, delta_w = 0) and the
  // refinement repeated.
  unsigned long long* d_norms = reinterpret_cast<unsigned long long*>(h->d_flags + 4);  // 16 bytes
  auto refine = [&](int sweeps) -> nmpc_status {
    k_to_factor_order<<<blocks_for(n, EW), EW, 0, st>>>(d, g, instance);
    launch_solve(h);
    k_from_factor_order<<<blocks_for(n, EW), EW, 0, st>>>(d, x, 0, instance);
    h->launches += 2;
    for (int sweep = 0; sweep < sweeps; ++sweep) {
      k_kmat_rows<<<blocks_for(m, EW), EW, 0, st>>>(d, h->d_Drow, x, t, ta, instance);
      k_kmat_vars_residual<<<blocks_for(n, EW), EW, 0, st>>>(d, x, t, ta, g, r, sc, instance);
      k_to_factor_order<<<blocks_for(n, EW), EW, 0, st>>>(d, r, instance);
      launch_solve(h);
      k_from_factor_order<<<blocks_for(n, EW), EW, 0, st>>>(d, x, 1, instance);
      h->launches += 4;
    }
    k_kmat_rows<<<blocks_for(m, EW), EW, 0, st>>>(d, h->d_Drow, x, t, ta, instance);
    k_kmat_vars_residual<<<blocks_for(n, EW), EW, 0, st>>>(d, x, t, ta, g, r, sc, instance);
    CUDA_TRY(h, cudaMemsetAsync(d_norms, 0, 2 * sizeof(unsigned long long), st));
    k_resid_norms<<<blocks_for(n, EW), EW, 0, st>>>(d, r, sc, instance, d_norms);
    h->launches += 3;
    return NMPC_OK;
  };
  auto rel_residual = [&](double* out) -> nmpc_status {
    unsigned long long nb[2];
    CUDA_TRY(h, cudaMemcpyAsync(nb, d_norms, sizeof(nb), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(h, cudaStreamSynchronize(st));
    std::memcpy(out, &nb[0], 8);  // componentwise backward error
    return NMPC_OK;
  };
  nmpc_status rs = refine(SENS_REFINE);
  if (rs != NMPC_OK) return rs;
  double rel = 0.0;
  if ((rs = rel_residual(&rel)) != NMPC_OK) return rs;
  if (!(rel <= 1e-12)) {
    k_ctl_select<<<blocks_for(ni), TPB, 0, st>>>(d.ctl, ni, instance, 1);
    const dim3 zgrid(std::max(1u, std::min(1024u, blocks_for(A.nnzL / std::max(1, ni) + 1))), ni);
    k_zero_L<<<zgrid, TPB, 0, st>>>(d, h->d_inst_Lbeg, h->d_inst_Lend);
    k_assemble<<<blocks_for(d.n_tgt, EW), EW, 0, st>>>(d, h->d_tgt_inst, h->d_Drow);
    h->launches += 3;
    launch_factor(h);
    if ((rs = refine(SENS_REFINE)) != NMPC_OK) return rs;
    if ((rs = rel_residual(&rel)) != NMPC_OK) return rs;
  }
  h->sens_residual = rel;
  // parameter gradients, through the staging area when the caller's arrays are on the host
  double* ox = dloss_dx0;
  double* os = dloss_dsp;
  if (!on_device) {
    ox = dloss_dx0 ? h->d_stage : nullptr;
    os = dloss_dsp ? h->d_stage + nx : nullptr;
  }
  k_sens_out<<<std::max(1u, blocks_for(std::max(nx, sp_len))), TPB, 0, st>>>(d, x, h->d_Drow, instance, ox, os);
  ++h->launches;
  CUDA_TRY(h, cudaGetLastError());
  if (!on_device) {
    if (dloss_dx0) CUDA_TRY(h, cudaMemcpyAsync(dloss_dx0, ox, (size_t)nx * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (dloss_dsp) CUDA_TRY(h, cudaMemcpyAsync(dloss_dsp, os, (size_t)sp_len * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  CUDA_TRY(h, cudaMemcpyAsync(d.ctl, h->d_ctl_save, ni * sizeof(Ctl), cudaMemcpyDeviceToDevice, st));
  if (!on_device) CUDA_TRY(h, cudaStreamSynchronize(st));
  if (!(rel <= 1e-8))
    return fail(h, NMPC_INERTIA_FAIL, "adjoint system not solved to a backward error of 1e-8 (K at the solution not positive definite?)");
  return NMPC_OK;
}

__global__ void k_ctl_force(Ctl* ctl, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  ctl[i].status = ST_RUNNING;
  ctl[i].need_factor = 1;
  ctl[i].factor_fail = 0;
}

nmpc_status nmpc_time_phases(nmpc_handle* h, int reps, nmpc_phase_times* out) {
  if (!h || !h->bound || !out || reps < 1) return fail(h, NMPC_ERR_INVALID, "bad arguments");
  if (!h->have_solution) return fail(h, NMPC_NOT_SOLVED, "no iterate to time at");
  const Analysis& A = h->A;
  Dev& d = h->d;
  cudaStream_t st = h->stream;
  const int ni = A.n_inst, n = A.n, m = A.m;
  CUDA_TRY(h, cudaMemcpyAsync(h->d_ctl_save, d.ctl, ni * sizeof(Ctl), cudaMemcpyDeviceToDevice, st));
  k_ctl_force<<<blocks_for(ni), TPB, 0, st>>>(d.ctl, ni);
  const dim3 zgrid(std::max(1u, std::min(1024u, blocks_for(A.nnzL / std::max(1, ni) + 1))), ni);
  cudaEvent_t e[5];
  for (auto& x : e) CUDA_TRY(h, cudaEventCreate(&x));
  double acc[4] = {0, 0, 0, 0};
  for (int r = 0; r < reps + 1; ++r) {
    CUDA_TRY(h, cudaEventRecord(e[0], st));
    k_eval_rows<<<blocks_for(m, EW), EW, 0, st>>>(d, 0, 1);
    k_eval_vars<<<blocks_for(n, EW), EW, 0, st>>>(d, 0);
    CUDA_TRY(h, cudaEventRecord(e[1], st));
    k_zero_L<<<zgrid, TPB, 0, st>>>(d, h->d_inst_Lbeg, h->d_inst_Lend);
    k_rows_pre<<<blocks_for(m, EW), EW, 0, st>>>(d, h->d_Drow);
    k_assemble<<<blocks_for(d.n_tgt, EW), EW, 0, st>>>(d, h->d_tgt_inst, h->d_Drow);
    CUDA_TRY(h, cudaEventRecord(e[2], st));
    launch_factor(h);
    CUDA_TRY(h, cudaEventRecord(e[3], st));
    k_rhs<<<blocks_for(n, EW), EW, 0, st>>>(d);
    launch_solve(h);
    CUDA_TRY(h, cudaEventRecord(e[4], st));
    CUDA_TRY(h, cudaEventSynchronize(e[4]));
    if (r == 0) continue;  // warm-up
    for (int q = 0; q < 4; ++q) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e[q], e[q + 1]);
      acc[q] += ms;
    }
  }
  for (auto& x : e) cudaEventDestroy(x);
  CUDA_TRY(h, cudaMemcpyAsync(d.ctl, h->d_ctl_save, ni * sizeof(Ctl), cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(h, cudaStreamSynchronize(st));
  out->ms_eval = acc[0] / reps; out->ms_assemble = acc[1] / reps;
  out->ms_factor = acc[2] / reps; out->ms_solve = acc[3] / reps;
  out->reps = reps;
  return NMPC_OK;
}

nmpc_status nmpc_get_stats(const nmpc_handle* h, nmpc_stats* st) {
  if (!h || !st) return NMPC_ERR_INVALID;
  const Analysis& A = h->A;
  st->n_total = A.n; st->m_total = A.m;
  st->n_supernodes = (int)A.sn_first.size();
  st->n_levels = (int)A.level_ptr.size() - 1;
  st->nnz_L = A.nnzL_true;
  st->factor_flops = A.factor_flops;
  st->solve_flops = A.solve_flops;
  st->workspace_bytes = (long long)h->ws_bytes;
  st->analysis_ms = A.analysis_ms;
  st->max_front = A.max_front;
  st->ordering_used = A.ordering_used;
  st->kernel_launches = h->launches;
  st->amalgamation_used = A.amalgamation_used;
  return NMPC_OK;
}

nmpc_status nmpc_instance_dims(const nmpc_handle* h, int instance, int* n, int* m, int* T) {
  if (!h || instance < 0 || instance >= h->A.n_inst) return NMPC_ERR_INVALID;
  if (n) *n = h->A.inst_n[instance];
  if (m) *m = h->A.inst_m[instance];
  if (T) *T = h->A.inst_T[instance];
  return NMPC_OK;
}

long long nmpc_structure_export(const nmpc_handle* h, int what, void* out, long long cap) {
  if (!h) return -1;
  const Analysis& A = h->A;
  auto copy = [&](const std::vector<int>& v) -> long long {
    if (out) std::memcpy(out, v.data(), sizeof(int) * (size_t)std::min<long long>(cap, (long long)v.size()));
    return (long long)v.size();
  };
  switch (what) {
    case 0: return copy(A.perm);
    case 1: return copy(A.sn_first);
    case 2: return copy(A.sn_ncol);
    case 3: return copy(A.sn_nrow);
    case 4: return copy(A.sn_rows);
    case 5: return copy(A.sn_parent);
    case 6: return copy(A.level_ptr);
    case 7: return copy(A.level_sn);
    case 9: {  // reduction chunks: (instance, kind, begin, end) each
      const long long cnt = (long long)A.chunks.size();
      int* o = static_cast<int*>(out);
      for (long long c = 0; out && c < std::min(cap, cnt); ++c) {
        const Chunk& ch = A.chunks[c];
        o[4 * c] = ch.inst; o[4 * c + 1] = ch.kind; o[4 * c + 2] = ch.begin; o[4 * c + 3] = ch.end;
      }
      return cnt;
    }
    case 10: return copy(A.red_var);
    case 11: {  // entries of each variable's column of H
      std::vector<int> len(A.n);
      for (int v = 0; v < A.n; ++v) len[v] = A.Hcsc_ptr[v + 1] - A.Hcsc_ptr[v];
      return copy(len);
    }
    case 8: {
      const long long cnt = (long long)A.tgt_L.size();
      int* o = static_cast<int*>(out);
      for (long long t = 0; out && t < std::min(cap, cnt); ++t) {
        const long long L = A.tgt_L[t];
        const int s = (int)(std::upper_bound(A.sn_Lptr.begin(), A.sn_Lptr.end(), L) - A.sn_Lptr.begin()) - 1;
        const long long off = L - A.sn_Lptr[s];
        o[2 * t] = A.sn_rows[A.sn_rowptr[s] + off % A.sn_nrow[s]];
        o[2 * t + 1] = A.sn_first[s] + (int)(off / A.sn_nrow[s]);
      }
      return cnt;
    }
    default: return -1;
  }
}

void nmpc_destroy(nmpc_handle* h) {
  if (!h) return;
  if (h->bound) {
    cudaStreamSynchronize(h->stream);
    if (h->h_flags) cudaFreeHost(h->h_flags);
    if (h->side) cudaStreamSynchronize(h->side);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
  }
  delete h;
}

const char* nmpc_status_string(int s) {
  switch (s) {
    case NMPC_OK: return "ok";
    case NMPC_ERR_INVALID: return "invalid argument";
    case NMPC_ERR_CUDA: return "CUDA error";
    case NMPC_ERR_WORKSPACE: return "workspace missing or too small";
    case NMPC_MAX_ITER: return "iteration limit reached";
    case NMPC_LINESEARCH_FAIL: return "line search failed";
    case NMPC_INERTIA_FAIL: return "inertia correction failed";
    case NMPC_NONFINITE: return "non-finite residual";
    case NMPC_TIMEOUT: return "bounded device wait timed out";
    case NMPC_NOT_SOLVED: return "not solved";
    default: return "unknown status";
  }
}

const char* nmpc_last_error(const nmpc_handle* h) { return h ? h->err.c_str() : "null handle"; }

}  // extern "C"

// ------------------------------------------------------------------------
// One-shot solve without any allocation.
//
// The whole device workspace of this entry point is the file-scope array
// below (NMPC_STATIC_WORKSPACE_BYTES).  Host code may not pass the array's
// name to a kernel or a copy: in host code it names a host-side shadow, not
// device memory.  Its device address is obtained with cudaGetSymbolAddress
// once per device, with that device current, on the first call made on that
// device, and cached.
// ------------------------------------------------------------------------

static __device__ __align__(256) unsigned char g_static_workspace[NMPC_STATIC_WORKSPACE_BYTES];

namespace {
std::mutex g_static_mu;
constexpr int MAX_DEVICES = 256;
void* g_static_addr[MAX_DEVICES] = {nullptr};
}  // namespace

extern "C" nmpc_status nmpc_solve_static(const nmpc_problem* prob, const nmpc_options* opts, void* cuda_stream,
                                         const double* x0, const double* setpoint, const double* u_prev,
                                         double* y_out, nmpc_info* info, int on_device) {
  if (!prob || !y_out || prob->n_instances < 1 || !prob->horizons) return NMPC_ERR_INVALID;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return NMPC_ERR_CUDA;
  void* ws = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_static_workspace) != cudaSuccess || !p) {
        std::fprintf(stderr, "nmpc_solve_static: cudaGetSymbolAddress failed on device %d\n", dev);
        return NMPC_ERR_CUDA;
      }
      g_static_addr[dev] = p;
    }
    ws = g_static_addr[dev];
  }
  nmpc_handle* h = nullptr;
  nmpc_status st = nmpc_build(prob, opts, cuda_stream, &h);
  if (st != NMPC_OK) return st;
  if (h->ws_bytes > (size_t)NMPC_STATIC_WORKSPACE_BYTES) {
    std::fprintf(stderr,
                 "nmpc_solve_static: the problem needs %zu bytes of device workspace, more than the %d bytes "
                 "of the library's static workspace; use nmpc_build/nmpc_bind with caller memory instead\n",
                 h->ws_bytes, NMPC_STATIC_WORKSPACE_BYTES);
    delete h;
    return NMPC_ERR_WORKSPACE;
  }
  // the previous call's contents are cleared by the upload (workspace memset)
  st = upload_structure(h, ws);
  int host_flags[4] = {0, 0, 0, 0};
  if (st == NMPC_OK) {
    h->h_flags = host_flags;  // pageable host memory: no pinned allocation
    h->graph_off = true;      // the host-driven loop: instantiating a graph allocates
    h->bound = true;
    const auto t0 = std::chrono::steady_clock::now();
    st = nmpc_set_params(h, -1, x0, setpoint, u_prev, on_device);
    nmpc_status sst = NMPC_OK;
    if (st == NMPC_OK) sst = nmpc_solve(h, 0, info);
    if (st == NMPC_OK && (sst == NMPC_ERR_INVALID || sst == NMPC_ERR_CUDA || sst == NMPC_ERR_WORKSPACE)) st = sst;
    if (st == NMPC_OK) {
      double* out = y_out;
      for (int i = 0; i < h->A.n_inst && st == NMPC_OK; ++i) {
        st = nmpc_get_solution(h, i, out, nullptr, on_device);
        out += h->A.inst_n[i];
      }
      if (st == NMPC_OK && on_device && cudaStreamSynchronize(h->stream) != cudaSuccess) st = NMPC_ERR_CUDA;
      if (st == NMPC_OK) st = sst;
    }
    if (info) {
      const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      for (int i = 0; i < h->A.n_inst; ++i) info[i].ms_total = ms;
    }
  }
  if (st != NMPC_OK && !h->err.empty()) std::fprintf(stderr, "nmpc_solve_static: %s\n", h->err.c_str());
  cudaStreamSynchronize(h->stream);
  h->h_flags = nullptr;
  delete h;
  return st;
}

// ------------------------------------------------------------------------
// Autotuner: candidate option sets for the analysis and the schedule, each
// timed by one cold solve in the caller's workspace; the choice is cached per
// problem and remaining options.
// ------------------------------------------------------------------------
namespace {

std::vector<nmpc_options> tune_candidates(const nmpc_problem* p, const nmpc_options& base) {
  int Tmax = 0;
  for (int i = 0; i < p->n_instances; ++i) Tmax = std::max(Tmax, p->horizons[i]);
  std::vector<nmpc_options> c;
  for (int form : {1, 3}) {
    if (Tmax >= 8) {
      for (int leaf : {1, 2})
        for (int am : {1, 2}) {
          nmpc_options o = base;
          o.ordering = NMPC_ORDER_ND;
          o.nd_leaf = leaf;
          o.panel_scale = form;
          o.amalgamation = am;
          o.factor_mode = 0;
          c.push_back(o);
        }
      // the dataflow factorization: nested dissection, and the two-sided
      // stage order (the flops of stage order, half its depth)
      for (int ord : {NMPC_ORDER_ND, NMPC_ORDER_TWO_SIDED})
        for (int am : {1, 2}) {
          if (ord == NMPC_ORDER_TWO_SIDED && am == 2) continue;  // chains: both modes give the same partition
          nmpc_options o = base;
          o.ordering = ord;
          o.nd_leaf = 1;
          o.panel_scale = form;
          o.amalgamation = am;
          o.factor_mode = 3;
          c.push_back(o);
        }
    }
    if (Tmax < 32) {  // a chain of at most 31 stages: its depth is no worse than a tree's
      nmpc_options o = base;
      o.ordering = NMPC_ORDER_NATURAL;
      o.nd_leaf = 1;
      o.panel_scale = form;
      o.amalgamation = 1;  // a chain: both modes give the same partition
      o.factor_mode = 0;
      c.push_back(o);
    }
  }
  return c;
}

// The problem and every option except the tuned ones, byte for byte.
std::string tune_key(const nmpc_problem* p, const nmpc_options* o) {
  nmpc_problem q = *p;
  q.horizons = nullptr;
  nmpc_options r = *o;
  r.ordering = 0;
  r.nd_leaf = 0;
  r.panel_scale = 0;
  r.amalgamation = 0;
  std::string k(reinterpret_cast<const char*>(&q), sizeof(q));
  k.append(reinterpret_cast<const char*>(p->horizons), sizeof(int) * (size_t)p->n_instances);
  k.append(reinterpret_cast<const char*>(&r), sizeof(r));
  return k;
}

std::mutex g_tune_mu;
std::vector<std::pair<std::string, nmpc_options>> g_tune_cache;
// candidates built (not bound) by nmpc_autotune_workspace_bytes for the last
// problem it sized, reused by nmpc_autotune
std::string g_tune_built_key;
std::vector<nmpc_handle*> g_tune_built;

void tune_drop_built() {  // caller holds g_tune_mu
  for (nmpc_handle* h : g_tune_built) nmpc_destroy(h);
  g_tune_built.clear();
  g_tune_built_key.clear();
}

// Set the packed parameters instance by instance (horizons may differ).
nmpc_status tune_set_params(nmpc_handle* h, const nmpc_problem* p, const double* x0, const double* sp,
                            const double* up, int on_device) {
  const Analysis& A = h->A;
  const int nx = A.mc.nx;
  size_t so = 0;
  for (int i = 0; i < A.n_inst; ++i) {
    const size_t sl = (A.mc.model == MODEL_PLATE) ? (size_t)A.sp_stride : (size_t)p->horizons[i];
    const nmpc_status st = nmpc_set_params(h, i, x0 ? x0 + (size_t)i * nx : nullptr, sp ? sp + so : nullptr,
                                           up ? up + i : nullptr, on_device);
    if (st != NMPC_OK) return st;
    so += sl;
  }
  return NMPC_OK;
}

}  // namespace

extern "C" {

nmpc_status nmpc_autotune_workspace_bytes(const nmpc_problem* prob, const nmpc_options* opts, size_t* bytes) {
  if (!prob || !bytes) return NMPC_ERR_INVALID;
  nmpc_options base;
  if (opts) base = *opts;
  else nmpc_options_defaults(&base);
  size_t need = 0;
  std::vector<nmpc_handle*> built;
  for (const nmpc_options& o : tune_candidates(prob, base)) {
    nmpc_handle* h = nullptr;
    const nmpc_status st = nmpc_build(prob, &o, nullptr, &h);
    if (st != NMPC_OK) {
      for (nmpc_handle* b : built) nmpc_destroy(b);
      return st;
    }
    need = std::max(need, h->ws_bytes);
    built.push_back(h);
  }
  std::lock_guard<std::mutex> lock(g_tune_mu);
  tune_drop_built();
  g_tune_built_key = tune_key(prob, &base);
  g_tune_built = built;
  *bytes = need;
  return NMPC_OK;
}

nmpc_status nmpc_autotune(const nmpc_problem* prob, nmpc_options* opts, void* cuda_stream, void* workspace,
                          size_t bytes, const double* x0, const double* setpoint, const double* u_prev,
                          int on_device, nmpc_tune_report* report) {
  if (!prob || !opts || !workspace || prob->n_instances < 1 || !prob->horizons) return NMPC_ERR_INVALID;
  if (reinterpret_cast<uintptr_t>(workspace) & 255) return NMPC_ERR_WORKSPACE;
  if (report) std::memset(report, 0, sizeof(*report));
  const std::string key = tune_key(prob, opts);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto& e : g_tune_cache)
      if (e.first == key) {
        opts->ordering = e.second.ordering;
        opts->nd_leaf = e.second.nd_leaf;
        opts->panel_scale = e.second.panel_scale;
        opts->amalgamation = e.second.amalgamation;
        opts->factor_mode = e.second.factor_mode;
        if (report) report->cached = 1;
        return NMPC_OK;
      }
  }
  const std::vector<nmpc_options> cand = tune_candidates(prob, *opts);
  std::vector<nmpc_handle*> built;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    if (g_tune_built_key == key && g_tune_built.size() == cand.size()) {
      built = g_tune_built;
      g_tune_built.clear();
      g_tune_built_key.clear();
    } else {
      tune_drop_built();
    }
  }
  int best = -1, fitted = 0;
  double best_ms = 0.0;
  nmpc_status first_fail = NMPC_OK;
  std::vector<nmpc_info> info(prob->n_instances);
  for (size_t c = 0; c < cand.size() && (int)c < NMPC_TUNE_MAX; ++c) {
    nmpc_tune_candidate rc{cand[c].ordering, cand[c].nd_leaf, cand[c].panel_scale, NMPC_ERR_WORKSPACE, 0, 0.0,
                           cand[c].amalgamation, cand[c].factor_mode, 0.0};
    nmpc_handle* h = built.empty() ? nullptr : built[c];
    nmpc_status st = NMPC_OK;
    if (h) h->stream = static_cast<cudaStream_t>(cuda_stream);  // built without a stream
    else st = nmpc_build(prob, &cand[c], cuda_stream, &h);
    if (st != NMPC_OK) {
      for (size_t k = c + 1; k < built.size(); ++k) nmpc_destroy(built[k]);
      return st;
    }
    if (h->ws_bytes <= bytes) {
      ++fitted;
      st = nmpc_bind(h, workspace, bytes);
      if (st == NMPC_OK) st = tune_set_params(h, prob, x0, setpoint, u_prev, on_device);
      if (st == NMPC_OK) st = nmpc_solve(h, 0, info.data());
      // the time of one iteration's evaluation, assembly, factorization and
      // solves at the converged point (the rest of an iteration is the same
      // for every candidate; a cold solve's total would also weigh its
      // inertia corrections, which warm re-solves rarely need)
      nmpc_phase_times pt{};
      if (st == NMPC_OK) st = nmpc_time_phases(h, 3, &pt);
      // and two steps of the closed loop (Algorithm 1): every instance
      // restarts from its own x_1 (and u_1), warm -- the re-solve an NMPC
      // loop repeats, with its share of iterations in which only a few
      // instances of a batch are still running
      double ms_rs = 0.0;
      for (int k = 0; k < 2 && st == NMPC_OK; ++k) {
        k_shift_params<<<std::min(1024u, blocks_for((long long)h->A.n_inst * (h->A.mc.nx + 1))), TPB, 0, h->stream>>>(h->d);
        ++h->launches;
        st = nmpc_solve(h, 1, info.data());
        ms_rs += info[0].ms_total;
      }
      if (st == NMPC_ERR_CUDA || st == NMPC_ERR_INVALID || st == NMPC_TIMEOUT) {
        if (!h->err.empty()) std::fprintf(stderr, "nmpc_autotune: %s\n", h->err.c_str());
        nmpc_destroy(h);
        for (size_t k = c + 1; k < built.size(); ++k) nmpc_destroy(built[k]);
        return st;
      }
      int iters = 0;
      for (const nmpc_info& f : info) iters = std::max(iters, f.iters);
      rc.status = st;
      rc.iters = iters;
      rc.ms_per_iter = pt.ms_eval + pt.ms_assemble + pt.ms_factor + pt.ms_solve;
      rc.ms_resolve = ms_rs / 2.0;
      if (st == NMPC_OK && (best < 0 || rc.ms_resolve < best_ms)) {
        best = (int)c;
        best_ms = rc.ms_resolve;
      }
      if (st != NMPC_OK && first_fail == NMPC_OK) first_fail = st;
    }
    nmpc_destroy(h);
    if (report) report->cand[report->n_candidates++] = rc;
  }
  if (report) report->best = best;
  if (!fitted) return NMPC_ERR_WORKSPACE;
  if (best < 0) return first_fail == NMPC_OK ? NMPC_MAX_ITER : first_fail;
  opts->ordering = cand[best].ordering;
  opts->nd_leaf = cand[best].nd_leaf;
  opts->panel_scale = cand[best].panel_scale;
  opts->amalgamation = cand[best].amalgamation;
  opts->factor_mode = cand[best].factor_mode;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache.emplace_back(key, *opts);
  return NMPC_OK;
}

}  // extern "C"
