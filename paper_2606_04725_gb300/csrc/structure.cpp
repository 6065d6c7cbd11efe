// Host structure analysis: patterns, ordering, elimination tree, supernodes,
// level sets, factor layout and scatter maps (Sec. 3.2.3, Algorithm 2).
//
// Everything here depends only on the sparsity structure, which is fixed
// across interior-point iterations and NMPC re-solves, so it runs once per
// nmpc_build (the paper's "SymCholesky" plus the transcription layout).
#include "structure.h"

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <functional>
#include <numeric>
#include <mutex>
#include <stdexcept>
#include <thread>

namespace nmpc {
namespace {

struct Layout {
  int nx, nu, T, nr;  // nr: rows per backward-Euler step (nx, or 2N + 3 for the DAE column)
  int offx(int k) const { return k == 0 ? 0 : nx + (k - 1) * (nx + nu); }
  int offu(int k) const { return offx(k) + nx; }
  int n() const { return nx + T * (nx + nu); }
  int m() const { return nx + T * nr; }
  int row(int k, int q) const { return nx + nr * k + q; }  // row q of step k -> k+1
};

// Plate: actuator segments adjacent to cell (ci, cj).  Each of the four sides
// (bottom, right, top, left, in that numbering) is split into S/4 equal runs.
int plate_segments(int g, int S, int ci, int cj, int out[2]) {
  const int per_side = S / 4, run = g / per_side;
  int cnt = 0;
  const bool on_side[4] = {cj == 0, ci == g - 1, cj == g - 1, ci == 0};
  const int pos[4] = {ci, cj, ci, cj};
  for (int side = 0; side < 4; ++side)
    if (on_side[side]) out[cnt++] = side * per_side + pos[side] / run;
  if (cnt == 2 && out[1] < out[0]) std::swap(out[0], out[1]);
  return cnt;
}

// ---------------------------------------------------------------- ordering

// Geometric nested dissection on vertex coordinates (up to 3 dimensions).
// A median cut along the dimension with the smallest vertex separator splits
// the set; the separator is every vertex on the low side adjacent to the
// high side.  Order: low part, high part, separator (recursively), so each
// separator is eliminated after the subgraphs it separates.
struct NDOrder {
  const std::vector<std::vector<int>>& adj;
  const std::vector<std::array<int, 3>>& coord;
  int leaf_max;
  bool two_sided = false;  // leaves eliminated from both ends toward their middle stage
  std::vector<int> label;  // region id of each vertex in the current call
  std::vector<int> order;
  int next_label = 1;

  NDOrder(const std::vector<std::vector<int>>& a, const std::vector<std::array<int, 3>>& c, int leaf)
      : adj(a), coord(c), leaf_max(leaf), label(a.size(), 0) {}

  void natural(std::vector<int>& set) {
    std::sort(set.begin(), set.end());
    order.insert(order.end(), set.begin(), set.end());
  }

  // A leaf spanning stages t_lo .. t_hi (time is coordinate 0): stages below
  // the middle one ascending, those above it descending, the middle stage
  // last.  A stage-coupled chain then fills only toward the middle: each
  // eliminated stage is joined to one neighbour that is still present (the
  // next one on its side), as in stage order, while the two halves are
  // independent subtrees -- the flops of stage order with half the depth.
  void leaf(std::vector<int>& set) {
    if (!two_sided || set.empty()) { natural(set); return; }
    int lo = coord[set[0]][0], hi = lo;
    for (int v : set) { lo = std::min(lo, coord[v][0]); hi = std::max(hi, coord[v][0]); }
    const int mid = lo + (hi - lo) / 2;
    auto rank = [&](int v) {
      const int t = coord[v][0];
      return t < mid ? t - lo : (t > mid ? (mid - lo) + (hi - t) : hi - lo + 1);
    };
    std::sort(set.begin(), set.end(), [&](int a, int b) {
      const int ra = rank(a), rb = rank(b);
      return ra != rb ? ra < rb : a < b;
    });
    order.insert(order.end(), set.begin(), set.end());
  }

  void run(std::vector<int>& set) {
    if ((int)set.size() <= leaf_max) { leaf(set); return; }
    int best_dim = -1, best_cut = 0;
    size_t best_sep = SIZE_MAX;
    for (int d = 0; d < 3; ++d) {
      std::vector<int> vals;
      vals.reserve(set.size());
      for (int v : set) vals.push_back(coord[v][d]);
      std::sort(vals.begin(), vals.end());
      vals.erase(std::unique(vals.begin(), vals.end()), vals.end());
      if (vals.size() < 2) continue;
      // median by vertex count among distinct values
      std::vector<int> all;
      all.reserve(set.size());
      for (int v : set) all.push_back(coord[v][d]);
      std::nth_element(all.begin(), all.begin() + all.size() / 2, all.end());
      int cut = all[all.size() / 2];
      if (cut >= vals.back()) cut = vals[vals.size() - 2];
      // separator size for this cut
      const int hi_lab = next_label++;
      for (int v : set) label[v] = (coord[v][d] > cut) ? hi_lab : -hi_lab;
      size_t sep = 0;
      for (int v : set) {
        if (label[v] != -hi_lab) continue;
        for (int w : adj[v]) if (label[w] == hi_lab) { ++sep; break; }
      }
      if (sep < best_sep) { best_sep = sep; best_dim = d; best_cut = cut; }
    }
    if (best_dim < 0) { natural(set); return; }
    const int hi_lab = next_label++;
    for (int v : set) label[v] = (coord[v][best_dim] > best_cut) ? hi_lab : -hi_lab;
    std::vector<int> lo, hi, sep;
    for (int v : set) {
      if (label[v] == hi_lab) { hi.push_back(v); continue; }
      bool s = false;
      for (int w : adj[v]) if (label[w] == hi_lab) { s = true; break; }
      (s ? sep : lo).push_back(v);
    }
    if (lo.empty() && hi.empty()) { natural(sep); return; }
    set.clear();
    set.shrink_to_fit();
    run(lo);
    run(hi);
    natural(sep);
  }
};

// ----------------------------------------------------- per-instance symbolic

struct InstSym {
  std::vector<int> pos;        // pos[local var] = local factor position
  std::vector<int> parent;     // elimination tree on positions
  std::vector<int> colcount;
  std::vector<int> sn_first, sn_ncol;
  std::vector<std::vector<int>> sn_rows;
  std::vector<int> sn_parent;
  int amalg = 0;               // amalgamation mode of this partition
};

// Elimination tree by Liu's algorithm with path compression.
// lower_rows[i] = columns k < i with a nonzero in row i.
std::vector<int> etree(int n, const std::vector<std::vector<int>>& lower_rows) {
  std::vector<int> parent(n, -1), anc(n, -1);
  for (int i = 0; i < n; ++i) {
    for (int k : lower_rows[i]) {
      int r = k;
      while (anc[r] != -1 && anc[r] != i) { int nx = anc[r]; anc[r] = i; r = nx; }
      if (anc[r] == -1) { anc[r] = i; parent[r] = i; }
    }
  }
  return parent;
}

// Sibling-limited amalgamation (mode 2) merges a supernode into a parent that
// has other children only while the merged panel stays this narrow.
constexpr int AMALG_SIBLING_COLS = 16;
// Automatic amalgamation chooses the sibling-limited mode when no front of the
// relaxed partition has more rows than this.
constexpr int AUTO_SMALL_FRONT_ROWS = 128;

void symbolic_instance(int n, const std::vector<std::pair<int, int>>& lower_edges,
                       const std::vector<int>& order, int amalg, InstSym& out) {
  // order[q] = local variable eliminated q-th
  std::vector<int> pos(n);
  for (int q = 0; q < n; ++q) pos[order[q]] = q;
  auto build_rows = [&](const std::vector<int>& p) {
    std::vector<std::vector<int>> rows(n);
    for (auto& e : lower_edges) {
      int a = p[e.first], b = p[e.second];
      if (a == b) continue;
      if (a < b) std::swap(a, b);
      rows[a].push_back(b);
    }
    for (auto& r : rows) { std::sort(r.begin(), r.end()); r.erase(std::unique(r.begin(), r.end()), r.end()); }
    return rows;
  };
  auto rows = build_rows(pos);
  std::vector<int> parent = etree(n, rows);
  // postorder the elimination tree (children in increasing order)
  std::vector<std::vector<int>> kids(n);
  std::vector<int> roots;
  for (int j = 0; j < n; ++j) (parent[j] < 0 ? roots : kids[parent[j]]).push_back(j);
  std::vector<int> post;
  post.reserve(n);
  std::vector<std::pair<int, size_t>> stack;
  for (int r : roots) {
    stack.push_back({r, 0});
    while (!stack.empty()) {
      auto& top = stack.back();
      if (top.second < kids[top.first].size()) {
        int c = kids[top.first][top.second++];
        stack.push_back({c, 0});
      } else {
        post.push_back(top.first);
        stack.pop_back();
      }
    }
  }
  std::vector<int> newpos(n);
  for (int q = 0; q < n; ++q) newpos[post[q]] = q;
  bool identity = true;
  for (int q = 0; q < n; ++q) identity &= (newpos[q] == q);
  if (!identity) {
    for (int v = 0; v < n; ++v) pos[v] = newpos[pos[v]];
    rows = build_rows(pos);
    parent = etree(n, rows);
  }
  // column counts by row-subtree traversal: row i of L covers the etree
  // paths from each k in row i of the matrix up to i
  std::vector<int> count(n, 1), mark(n, -1);
  for (int i = 0; i < n; ++i) {
    mark[i] = i;
    for (int k : rows[i]) {
      for (int j = k; mark[j] != i; j = parent[j]) { mark[j] = i; ++count[j]; }
    }
  }
  std::vector<int> nkids(n, 0);
  for (int j = 0; j < n; ++j) if (parent[j] >= 0) nkids[parent[j]]++;
  // fundamental supernodes
  std::vector<int> ff, fc;
  for (int j = 0; j < n; ++j) {
    bool join = j > 0 && parent[j - 1] == j && count[j - 1] == count[j] + 1 && nkids[j] == 1;
    if (join) fc.back()++;
    else { ff.push_back(j); fc.push_back(1); }
  }
  const int nf = (int)ff.size();
  std::vector<int> fsn_of(n);
  for (int s = 0; s < nf; ++s)
    for (int j = ff[s]; j < ff[s] + fc[s]; ++j) fsn_of[j] = s;
  std::vector<int> fpar(nf, -1);
  for (int s = 0; s < nf; ++s) {
    const int last = ff[s] + fc[s] - 1;
    if (parent[last] >= 0) fpar[s] = fsn_of[parent[last]];
  }
  // Relaxed amalgamation: a supernode whose columns end right before its
  // parent's first column is merged into the parent when the merged panel
  // keeps its share of explicit zeros small (larger panels tolerate less).
  // Merging trades a few zero flops for fewer, wider dense panels.
  std::vector<long long> nnz_true(nf, 0);
  std::vector<int> rowsz(nf);   // rows of the (possibly merged) supernode, columns included
  std::vector<int> gfirst(ff), gcols(fc);
  for (int s = 0; s < nf; ++s) {
    for (int j = ff[s]; j < ff[s] + fc[s]; ++j) nnz_true[s] += count[j];
    rowsz[s] = count[ff[s]];
  }
  std::vector<char> merged(nf, 0);
  std::vector<int> nch(nf, 0);   // children of each (possibly merged) supernode
  for (int s = 0; s < nf; ++s) if (fpar[s] >= 0) nch[fpar[s]]++;
  auto stored = [](long long c, long long r) { return c * r - c * (c - 1) / 2; };
  for (int s = 0; s < nf; ++s) {
    const int p = fpar[s];
    if (p < 0 || gfirst[s] + gcols[s] != gfirst[p]) continue;
    const long long c = gcols[s] + gcols[p];
    const long long r = rowsz[p] + gcols[s];
    const long long st = stored(c, r), nz = nnz_true[s] + nnz_true[p];
    const double zf = double(st - nz) / double(st);
    const double lim = c <= 4 ? 0.8 : (c <= 16 ? 0.5 : (c <= 48 ? 0.35 : (c <= 128 ? 0.15 : 0.05)));
    if (zf > lim) continue;
    if (amalg == 2 && nch[p] > 1 && c > AMALG_SIBLING_COLS) continue;
    merged[s] = 1;
    nch[p] += nch[s] - 1;
    gfirst[p] = gfirst[s];
    gcols[p] = (int)c;
    rowsz[p] = (int)r;
    nnz_true[p] = nz;
  }
  out.sn_first.clear(); out.sn_ncol.clear();
  std::vector<int> top_of;  // final supernode -> fundamental supernode on top of its group
  for (int s = 0; s < nf; ++s)
    if (!merged[s]) { out.sn_first.push_back(gfirst[s]); out.sn_ncol.push_back(gcols[s]); top_of.push_back(s); }
  const int ns = (int)out.sn_first.size();
  std::vector<int> sn_of(n);
  for (int s = 0; s < ns; ++s)
    for (int j = out.sn_first[s]; j < out.sn_first[s] + out.sn_ncol[s]; ++j) sn_of[j] = s;
  // lower columns: for each column j, its rows > j
  std::vector<std::vector<int>> cols(n);
  for (int i = 0; i < n; ++i) for (int k : rows[i]) cols[k].push_back(i);
  out.sn_parent.assign(ns, -1);
  out.sn_rows.assign(ns, {});
  std::vector<std::vector<int>> sn_kids(ns);
  for (int s = 0; s < ns; ++s) {
    int last = out.sn_first[s] + out.sn_ncol[s] - 1;
    if (parent[last] >= 0) { out.sn_parent[s] = sn_of[parent[last]]; sn_kids[out.sn_parent[s]].push_back(s); }
  }
  std::vector<int> smark(n, -1);
  for (int s = 0; s < ns; ++s) {
    const int f = out.sn_first[s], l = f + out.sn_ncol[s] - 1;
    std::vector<int>& R = out.sn_rows[s];
    for (int j = f; j <= l; ++j) { R.push_back(j); smark[j] = s; }
    for (int j = f; j <= l; ++j)
      for (int i : cols[j]) if (i > l && smark[i] != s) { smark[i] = s; R.push_back(i); }
    for (int c : sn_kids[s]) {
      const auto& Rc = out.sn_rows[c];
      for (size_t q = out.sn_ncol[c]; q < Rc.size(); ++q) {
        int i = Rc[q];
        if (i > l && smark[i] != s) { smark[i] = s; R.push_back(i); }
      }
    }
    std::sort(R.begin() + out.sn_ncol[s], R.end());
    if ((int)R.size() != rowsz[top_of[s]]) throw std::runtime_error("supernode structure disagrees with column counts");
  }
  out.pos = std::move(pos);
  out.parent = std::move(parent);
  out.colcount = std::move(count);
}

}  // namespace

// Run f(0 .. n-1) on up to hardware_concurrency host threads; the first
// exception thrown by any task is rethrown after all threads have joined.
void parallel_for(int n, const std::function<void(int)>& f) {
  const int nt = std::max(1, std::min<int>(n, (int)std::thread::hardware_concurrency()));
  std::atomic<int> next{0};
  std::mutex mu;
  std::exception_ptr err;
  auto work = [&] {
    for (;;) {
      const int q = next.fetch_add(1);
      if (q >= n) return;
      try {
        f(q);
      } catch (...) {
        std::lock_guard<std::mutex> lock(mu);
        if (!err) err = std::current_exception();
      }
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
  if (err) std::rethrow_exception(err);
}

std::string analyze(const ProblemSpec& sp, Analysis& A) {
  auto t0 = std::chrono::steady_clock::now();
  try {
    const int ni = (int)sp.T.size();
    if (ni < 1) return "n_instances must be >= 1";
    if (sp.amalgamation < 0 || sp.amalgamation > 2) return "amalgamation must be 0, 1 or 2";
    ModelConst& mc = A.mc;
    mc = ModelConst{};
    mc.model = sp.model;
    if (sp.model == MODEL_DISTILL) {
      if (sp.N < 3 || sp.Nf < 2 || sp.Nf > sp.N - 1) return "distillation needs N >= 3 and 2 <= Nf <= N-1";
      mc.nx = sp.N; mc.nu = 1; mc.WH = 5; mc.WS = 2 * sp.N + 2;
    } else if (sp.model == MODEL_PLATE) {
      if (sp.g < 2 || sp.S < 4 || sp.S % 4 || sp.g % (sp.S / 4)) return "plate needs g >= 2, S % 4 == 0, g % (S/4) == 0";
      mc.nx = sp.g * sp.g; mc.nu = sp.S; mc.WH = 8; mc.WS = sp.g * sp.g + sp.S;
    } else if (sp.model == MODEL_TOY) {
      mc.nx = 1; mc.nu = 1; mc.WH = 3; mc.WS = 2;
    } else if (sp.model == MODEL_PPLATE) {
      if (sp.g < 4) return "the paper's plate needs g >= 4 grid points per side";
      mc.nx = (sp.g - 2) * (sp.g - 2); mc.nu = 1; mc.WH = 7; mc.WS = mc.nx + 1;
    } else if (sp.model == MODEL_DDAE) {
      if (sp.N < 3 || sp.Nf < 2 || sp.Nf > sp.N - 1) return "distillation needs N >= 3 and 2 <= Nf <= N-1";
      mc.nx = sp.N; mc.nu = sp.N + 4; mc.WH = 8; mc.WS = 3 * sp.N + 1;
    } else {
      return "unknown model";
    }
    mc.N = sp.N; mc.Nf = sp.Nf; mc.g = sp.g; mc.S = sp.S;
    mc.dt = sp.dt; mc.alpha = sp.alpha; mc.D = sp.D; mc.F = sp.F; mc.xF = sp.xF;
    mc.Ac = sp.Ac; mc.At = sp.At; mc.Ar = sp.Ar; mc.wdu = sp.wdu;
    mc.kappa = sp.kappa; mc.cq = sp.cq; mc.rho_u = sp.rho_u;
    mc.xlo = sp.xlo; mc.xhi = sp.xhi; mc.ulo = sp.ulo; mc.uhi = sp.uhi;
    mc.wu = sp.wu; mc.ubar = sp.ubar;
    mc.inv_Ac = 1.0 / sp.Ac; mc.inv_At = 1.0 / sp.At; mc.inv_Ar = 1.0 / sp.Ar;
    mc.gamma = sp.gamma; mc.tol = sp.tol; mc.pivtol = sp.pivtol; mc.dw_max = sp.dw_max;
    mc.Tb = sp.Tb; mc.qloss = sp.qloss;
    mc.nr = (sp.model == MODEL_DDAE) ? 2 * sp.N + 3 : mc.nx;
    const int nx = mc.nx, nu = mc.nu, WH = mc.WH, WS = mc.WS;
    A.n_inst = ni;
    A.sp_stride = (sp.model == MODEL_PLATE) ? nx : *std::max_element(sp.T.begin(), sp.T.end());
    A.inst_T = sp.T;
    A.inst_voff.resize(ni); A.inst_roff.resize(ni); A.inst_woff.resize(ni);
    A.inst_n.resize(ni); A.inst_m.resize(ni); A.inst_nz.resize(ni);
    long long n = 0, m = 0, nW = 0;
    for (int i = 0; i < ni; ++i) {
      if (sp.T[i] < 1) return "horizons must be >= 1";
      Layout L{nx, nu, sp.T[i], mc.nr};
      A.inst_voff[i] = (int)n; A.inst_roff[i] = (int)m; A.inst_woff[i] = (int)nW;
      A.inst_n[i] = L.n(); A.inst_m[i] = L.m();
      n += L.n(); m += L.m(); nW += (long long)sp.T[i] * WS;
    }
    if (n > (1LL << 30) || m * WH > (1LL << 31) - 1 || nW > (1LL << 31) - 1) return "problem too large for 32-bit vector indices";
    A.n = (int)n; A.m = (int)m; A.nW = (int)nW;
    A.var_inst.resize(n); A.row_inst.resize(m);
    A.yL.resize(n); A.yU.resize(n);
    A.Hcol.assign((size_t)m * WH, -1);
    std::vector<int> Wi((size_t)nW, -1), Wj((size_t)nW, -1);
    A.perm.resize(n); A.iperm.resize(n);

    std::vector<InstSym> syms(ni);
    for (int i = 0; i < ni; ++i) {
      Layout L{nx, nu, sp.T[i], mc.nr};
      const int vo = A.inst_voff[i], ro = A.inst_roff[i], wo = A.inst_woff[i];
      const int nl = L.n(), ml = L.m();
      for (int v = 0; v < nl; ++v) A.var_inst[vo + v] = i;
      for (int r = 0; r < ml; ++r) A.row_inst[ro + r] = i;
      // bounds: x_0 free, stages 1..T bounded
      int nz = 2 * ml;
      for (int v = 0; v < nx; ++v) { A.yL[vo + v] = -INFINITY; A.yU[vo + v] = INFINITY; }
      for (int k = 1; k <= L.T; ++k) {
        for (int q = 0; q < nx; ++q) { A.yL[vo + L.offx(k) + q] = sp.xlo; A.yU[vo + L.offx(k) + q] = sp.xhi; }
        for (int q = 0; q < nu; ++q) { A.yL[vo + L.offu(k) + q] = sp.ulo; A.yU[vo + L.offu(k) + q] = sp.uhi; }
        if (sp.model == MODEL_DDAE) {  // y in [0, 1], u as given, L, V, S in [0, 10] (eq. distill-ocp)
          for (int q = 0; q < nx; ++q) { A.yL[vo + L.offu(k) + q] = 0.0; A.yU[vo + L.offu(k) + q] = 1.0; }
          for (int q = nx + 1; q < nu; ++q) { A.yL[vo + L.offu(k) + q] = 0.0; A.yU[vo + L.offu(k) + q] = 10.0; }
        }
      }
      for (int v = 0; v < nl; ++v) nz += std::isfinite(A.yL[vo + v]) + std::isfinite(A.yU[vo + v]);
      A.inst_nz[i] = nz;
      // Jacobian slots (local columns, -1 unused)
      auto hc = [&](int r, int s) -> int& { return A.Hcol[(size_t)(ro + r) * WH + s]; };
      for (int q = 0; q < nx; ++q) hc(q, 0) = q;
      for (int k = 0; k < L.T; ++k) {
        if (sp.model == MODEL_DDAE) {
          // balance of tray i: [x_k,i | x_{k+1},i-1 | x_{k+1},i | y_{k+1},i | y_{k+1},i+1 | L | V | S]
          const int N = sp.N, Nf = sp.Nf, bx = L.offx(k + 1), bu = L.offu(k + 1);
          for (int i = 1; i <= N; ++i) {
            const int r = L.row(k, i - 1);
            hc(r, 0) = L.offx(k) + i - 1;
            if (i >= 2) hc(r, 1) = bx + i - 2;
            hc(r, 2) = bx + i - 1;
            if (i >= 2) hc(r, 3) = bu + i - 1;
            if (i <= N - 1) hc(r, 4) = bu + i;
            if (i >= 2 && i <= Nf) hc(r, 5) = bu + N + 1;
            hc(r, 6) = bu + N + 2;
            if (i >= Nf) hc(r, 7) = bu + N + 3;
          }
          for (int i = 0; i < N; ++i) {  // equilibrium: [x_{k+1},i | y_{k+1},i]
            hc(L.row(k, N + i), 0) = bx + i;
            hc(L.row(k, N + i), 1) = bu + i;
          }
          hc(L.row(k, 2 * N), 0) = bu + N;          // L - u D: [u | L]
          hc(L.row(k, 2 * N), 1) = bu + N + 1;
          hc(L.row(k, 2 * N + 1), 0) = bu + N + 1;  // V - L - D: [L | V]
          hc(L.row(k, 2 * N + 1), 1) = bu + N + 2;
          hc(L.row(k, 2 * N + 2), 0) = bu + N + 1;  // S - L - F: [L | S]
          hc(L.row(k, 2 * N + 2), 1) = bu + N + 3;
          continue;
        }
        for (int q = 0; q < nx; ++q) {
          const int r = L.row(k, q);
          hc(r, 0) = L.offx(k) + q;
          if (sp.model == MODEL_DISTILL) {
            if (q > 0) hc(r, 1) = L.offx(k + 1) + q - 1;
            hc(r, 2) = L.offx(k + 1) + q;
            if (q < nx - 1) hc(r, 3) = L.offx(k + 1) + q + 1;
            hc(r, 4) = L.offu(k + 1);
          } else if (sp.model == MODEL_PLATE) {
            const int g = sp.g, ci = q % g, cj = q / g, b = L.offx(k + 1);
            if (cj > 0) hc(r, 1) = b + q - g;
            if (ci > 0) hc(r, 2) = b + q - 1;
            hc(r, 3) = b + q;
            if (ci < g - 1) hc(r, 4) = b + q + 1;
            if (cj < g - 1) hc(r, 5) = b + q + g;
            int segs[2];
            int ns = plate_segments(g, sp.S, ci, cj, segs);
            for (int t = 0; t < ns; ++t) hc(r, 6 + t) = L.offu(k + 1) + segs[t];
          } else if (sp.model == MODEL_PPLATE) {
            const int mm = sp.g - 2, ci = q % mm, cj = q / mm, b = L.offx(k + 1);
            if (cj > 0) hc(r, 1) = b + q - mm;
            if (ci > 0) hc(r, 2) = b + q - 1;
            hc(r, 3) = b + q;
            if (ci < mm - 1) hc(r, 4) = b + q + 1;
            if (cj < mm - 1) hc(r, 5) = b + q + mm;
            if (ci == 0 || cj == 0) hc(r, 6) = L.offu(k + 1);
          } else {
            hc(r, 1) = L.offx(k + 1);
            hc(r, 2) = L.offu(k + 1);
          }
        }
      }
      // Hessian slots (local indices, lower triangle)
      for (int k = 1; k <= L.T; ++k) {
        const size_t base = (size_t)wo + (size_t)(k - 1) * WS;
        auto ws = [&](int s, int a, int b) { Wi[base + s] = std::max(a, b); Wj[base + s] = std::min(a, b); };
        if (sp.model == MODEL_DISTILL) {
          for (int q = 0; q < nx; ++q) { ws(q, L.offx(k) + q, L.offx(k) + q); ws(nx + q, L.offu(k), L.offx(k) + q); }
          ws(2 * nx, L.offu(k), L.offu(k));
          if (k >= 2) ws(2 * nx + 1, L.offu(k), L.offu(k - 1));
        } else if (sp.model == MODEL_DDAE) {
          // [x_j diag (N) | (L or S, x_j), j < N (N-1) | (V, x_1) | (V, y_j), j >= 2 (N-1) | u diag | (u, u_prev)]
          const int N = sp.N, Nf = sp.Nf, bx = L.offx(k), bu = L.offu(k);
          for (int j = 0; j < N; ++j) ws(j, bx + j, bx + j);
          for (int j = 1; j <= N - 1; ++j) ws(N + j - 1, bu + N + (j < Nf ? 1 : 3), bx + j - 1);
          ws(2 * N - 1, bu + N + 2, bx);
          for (int j = 2; j <= N; ++j) ws(2 * N + j - 2, bu + N + 2, bu + j - 1);
          ws(3 * N - 1, bu + N, bu + N);
          if (k >= 2) ws(3 * N, bu + N, L.offu(k - 1) + N);
        } else if (sp.model == MODEL_PLATE || sp.model == MODEL_PPLATE) {
          for (int q = 0; q < nx; ++q) ws(q, L.offx(k) + q, L.offx(k) + q);
          for (int q = 0; q < nu; ++q) ws(nx + q, L.offu(k) + q, L.offu(k) + q);
        } else {
          ws(0, L.offx(k), L.offx(k));
          ws(1, L.offu(k), L.offu(k));
        }
      }
    }
    // The symbolic analysis of an instance (condensed pattern, ordering,
    // elimination tree, supernodes) depends only on its horizon: it runs once
    // per distinct horizon, for the first instance that has it, on several
    // host threads, and the other instances copy it.
    auto ord_of = [&](int T) { return sp.ordering != 0 ? sp.ordering : (T < 8 ? 1 : 2); };  // short horizons: a chain
    std::vector<int> rep_of(ni), reps;
    {
      std::vector<std::pair<int, int>> firsts;  // (T, first instance), sorted by T
      for (int i = 0; i < ni; ++i) {
        auto it = std::lower_bound(firsts.begin(), firsts.end(), std::make_pair(sp.T[i], -1));
        if (it != firsts.end() && it->first == sp.T[i]) {
          rep_of[i] = it->second;
        } else {
          firsts.insert(it, {sp.T[i], i});
          rep_of[i] = i;
          reps.push_back(i);
        }
      }
    }
    auto symbolic_of = [&](int i) {
      Layout L{nx, nu, sp.T[i], mc.nr};
      const int wo = A.inst_woff[i], ro = A.inst_roff[i];
      const int nl = L.n(), ml = L.m();
      auto hc = [&](int r, int s) -> int { return A.Hcol[(size_t)(ro + r) * WH + s]; };
      // condensed pattern K_c = W + Sigma + H^T D H (local lower edges)
      std::vector<std::pair<int, int>> edges;
      edges.reserve((size_t)ml * WH * (WH + 1) / 2 + (size_t)L.T * WS + nl);
      for (int v = 0; v < nl; ++v) edges.push_back({v, v});
      for (int s = 0; s < L.T * WS; ++s)
        if (Wi[wo + s] >= 0) edges.push_back({Wi[wo + s], Wj[wo + s]});
      for (int r = 0; r < ml; ++r)
        for (int a = 0; a < WH; ++a) {
          int ca = hc(r, a);
          if (ca < 0) continue;
          for (int b = 0; b <= a; ++b) {
            int cb = hc(r, b);
            if (cb < 0) continue;
            edges.push_back({std::max(ca, cb), std::min(ca, cb)});
          }
        }
      std::sort(edges.begin(), edges.end());
      edges.erase(std::unique(edges.begin(), edges.end()), edges.end());
      // ordering
      const int ord = ord_of(L.T);
      std::vector<int> order(nl);
      if (ord == 1) {
        std::iota(order.begin(), order.end(), 0);
      } else {
        std::vector<std::vector<int>> adj(nl);
        for (auto& e : edges) if (e.first != e.second) { adj[e.first].push_back(e.second); adj[e.second].push_back(e.first); }
        std::vector<std::array<int, 3>> coord(nl, {0, 0, 0});
        for (int k = 0; k <= L.T; ++k) {
          for (int q = 0; q < nx; ++q) {
            auto& c = coord[L.offx(k) + q];
            c[0] = k;
            if (sp.model == MODEL_PLATE) { c[1] = q % sp.g; c[2] = q / sp.g; }
            if (sp.model == MODEL_PPLATE) { c[1] = q % (sp.g - 2); c[2] = q / (sp.g - 2); }
          }
          if (k >= 1)
            for (int q = 0; q < nu; ++q) {
              auto& c = coord[L.offu(k) + q];
              c[0] = k;
              if (sp.model == MODEL_PLATE) {
                // segment midpoint on its side
                const int per = sp.S / 4, run = sp.g / per, side = q / per, mid = (q % per) * run + run / 2;
                const int xs[4] = {mid, sp.g - 1, mid, 0}, ys[4] = {0, mid, sp.g - 1, mid};
                c[1] = xs[side]; c[2] = ys[side];
              }
            }
        }
        int leaf = (sp.model == MODEL_PLATE || sp.model == MODEL_PPLATE) ? std::max(1, sp.nd_leaf) * 64
                                                                         : std::max(1, sp.nd_leaf) * (nx + nu);
        if (ord == 3 && sp.nd_leaf <= 1) leaf = nl;  // the whole horizon is one two-sided leaf
        NDOrder nd(adj, coord, leaf);
        nd.two_sided = ord == 3;
        std::vector<int> all(nl);
        std::iota(all.begin(), all.end(), 0);
        nd.run(all);
        order = nd.order;
        if ((int)order.size() != nl) throw std::runtime_error("nested dissection lost vertices");
      }
      // Automatic amalgamation: relaxed, unless every front of the relaxed
      // partition has at most AUTO_SMALL_FRONT_ROWS rows.  Such fronts are
      // factored in shared memory, and their time is set by the chain of
      // pivots of the widest front of each level, not by flops: there the
      // separators of nested dissection are kept apart (sibling-limited), so
      // that no level waits on a separator merged with one below it.
      int am = sp.amalgamation;
      if (am != 0) {
        symbolic_instance(nl, edges, order, am, syms[i]);
      } else {
        am = 1;
        symbolic_instance(nl, edges, order, am, syms[i]);
        size_t rows = 0;
        for (const auto& R : syms[i].sn_rows) rows = std::max(rows, R.size());
        if (rows <= (size_t)AUTO_SMALL_FRONT_ROWS) {
          am = 2;
          symbolic_instance(nl, edges, order, am, syms[i]);
        }
      }
      syms[i].amalg = am;
    };
    parallel_for((int)reps.size(), [&](int q) { symbolic_of(reps[q]); });
    for (int i = 0; i < ni; ++i)
      if (rep_of[i] != i) syms[i] = syms[rep_of[i]];
    A.ordering_used = ord_of(sp.T[ni - 1]);
    A.amalgamation_used = syms[ni - 1].amalg;
    for (int i = 0; i < ni; ++i) {
      Layout L{nx, nu, sp.T[i], mc.nr};
      const int vo = A.inst_voff[i], ro = A.inst_roff[i], wo = A.inst_woff[i];
      const int nl = L.n(), ml = L.m();
      auto hc = [&](int r, int s) -> int& { return A.Hcol[(size_t)(ro + r) * WH + s]; };
      for (int v = 0; v < nl; ++v) { A.perm[vo + v] = vo + syms[i].pos[v]; A.iperm[vo + syms[i].pos[v]] = vo + v; }
      // convert H columns to global indices
      for (int r = 0; r < ml; ++r)
        for (int s = 0; s < WH; ++s) if (hc(r, s) >= 0) hc(r, s) += vo;
      for (int s = 0; s < L.T * WS; ++s)
        if (Wi[wo + s] >= 0) { Wi[wo + s] += vo; Wj[wo + s] += vo; }
    }

    // H column lists (CSC over slots) for H^T v products
    A.Hcsc_ptr.assign(n + 1, 0);
    for (size_t s = 0; s < A.Hcol.size(); ++s) if (A.Hcol[s] >= 0) A.Hcsc_ptr[A.Hcol[s] + 1]++;
    for (int v = 0; v < n; ++v) A.Hcsc_ptr[v + 1] += A.Hcsc_ptr[v];
    A.Hcsc_slot.resize(A.Hcsc_ptr[n]);
    {
      std::vector<int> fill(A.Hcsc_ptr.begin(), A.Hcsc_ptr.end() - 1);
      for (size_t s = 0; s < A.Hcol.size(); ++s) if (A.Hcol[s] >= 0) A.Hcsc_slot[fill[A.Hcol[s]]++] = (int)s;
    }

    // per-variable adjacency of the Hessian slots (both triangles), for K x
    A.Wadj_ptr.assign(n + 1, 0);
    for (long long q = 0; q < nW; ++q)
      if (Wi[q] >= 0) { A.Wadj_ptr[Wi[q] + 1]++; if (Wj[q] != Wi[q]) A.Wadj_ptr[Wj[q] + 1]++; }
    for (int v = 0; v < n; ++v) A.Wadj_ptr[v + 1] += A.Wadj_ptr[v];
    A.Wadj_slot.resize(A.Wadj_ptr[n]);
    A.Wadj_other.resize(A.Wadj_ptr[n]);
    {
      std::vector<int> fill(A.Wadj_ptr.begin(), A.Wadj_ptr.end() - 1);
      for (long long q = 0; q < nW; ++q) {
        if (Wi[q] < 0) continue;
        A.Wadj_slot[fill[Wi[q]]] = (int)q; A.Wadj_other[fill[Wi[q]]++] = Wj[q];
        if (Wj[q] != Wi[q]) { A.Wadj_slot[fill[Wj[q]]] = (int)q; A.Wadj_other[fill[Wj[q]]++] = Wi[q]; }
      }
    }

    // global supernodes
    A.sn_first.clear();
    std::vector<int> sn_base(ni);
    for (int i = 0; i < ni; ++i) {
      const InstSym& S = syms[i];
      sn_base[i] = (int)A.sn_first.size();
      for (size_t s = 0; s < S.sn_first.size(); ++s) {
        A.sn_first.push_back(A.inst_voff[i] + S.sn_first[s]);
        A.sn_ncol.push_back(S.sn_ncol[s]);
        A.sn_nrow.push_back((int)S.sn_rows[s].size());
        A.sn_inst.push_back(i);
        A.sn_parent.push_back(S.sn_parent[s] < 0 ? -1 : sn_base[i] + S.sn_parent[s]);
      }
    }
    const int ns = (int)A.sn_first.size();
    A.sn_rowptr.assign(ns + 1, 0);
    A.sn_Lptr.assign(ns + 1, 0); A.sn_Uptr.assign(ns + 1, 0); A.sn_uvptr.assign(ns + 1, 0);
    A.factor_flops = 0; A.nnzL_true = 0; A.max_front = 0;
    for (int s = 0; s < ns; ++s) {
      const long long c = A.sn_ncol[s], r = A.sn_nrow[s];
      A.sn_rowptr[s + 1] = A.sn_rowptr[s] + r;
      A.sn_Lptr[s + 1] = A.sn_Lptr[s] + (((long long)r * c + 1) & ~1LL);  // panels start on 16-byte boundaries
      A.sn_Uptr[s + 1] = A.sn_Uptr[s] + (r - c) * (r - c);
      A.sn_uvptr[s + 1] = A.sn_uvptr[s] + (r - c);
      for (long long j = 0; j < c; ++j) {
        const double cj = (double)(r - j);
        A.factor_flops += cj * cj;
        A.nnzL_true += r - j;
      }
      A.max_front = std::max(A.max_front, (int)r);
    }
    A.nnzL = A.sn_Lptr[ns]; A.nU = A.sn_Uptr[ns]; A.nuv = A.sn_uvptr[ns];
    A.solve_flops = 4.0 * (double)A.nnzL_true;
    A.sn_rows.resize(A.sn_rowptr[ns]);
    for (int i = 0; i < ni; ++i) {
      const InstSym& S = syms[i];
      for (size_t s = 0; s < S.sn_first.size(); ++s) {
        const int gs = sn_base[i] + (int)s;
        const auto& R = S.sn_rows[s];
        for (size_t q = 0; q < R.size(); ++q) A.sn_rows[A.sn_rowptr[gs] + q] = A.inst_voff[i] + R[q];
      }
    }
    // children lists and relative positions of each child's update rows in its parent
    A.sn_child_ptr.assign(ns + 1, 0);
    for (int s = 0; s < ns; ++s) if (A.sn_parent[s] >= 0) A.sn_child_ptr[A.sn_parent[s] + 1]++;
    for (int s = 0; s < ns; ++s) A.sn_child_ptr[s + 1] += A.sn_child_ptr[s];
    A.sn_child.resize(A.sn_child_ptr[ns]);
    {
      std::vector<int> fill(A.sn_child_ptr.begin(), A.sn_child_ptr.end() - 1);
      for (int s = 0; s < ns; ++s) if (A.sn_parent[s] >= 0) A.sn_child[fill[A.sn_parent[s]]++] = s;
    }
    A.sn_relptr.assign(ns + 1, 0);
    for (int s = 0; s < ns; ++s) A.sn_relptr[s + 1] = A.sn_relptr[s] + (A.sn_nrow[s] - A.sn_ncol[s]);
    A.sn_rel.resize(A.sn_relptr[ns]);
    for (int s = 0; s < ns; ++s) {
      const int p = A.sn_parent[s];
      const int nupd = A.sn_nrow[s] - A.sn_ncol[s];
      if (nupd > 0 && p < 0) throw std::runtime_error("root supernode with update rows");
      const int* Rp = A.sn_rows.data() + A.sn_rowptr[p < 0 ? s : p];
      const int np_ = A.sn_nrow[p < 0 ? s : p];
      for (int q = 0; q < nupd; ++q) {
        const int row = A.sn_rows[A.sn_rowptr[s] + A.sn_ncol[s] + q];
        const int* it = std::lower_bound(Rp, Rp + np_, row);
        if (it == Rp + np_ || *it != row) throw std::runtime_error("update row missing from parent structure");
        A.sn_rel[A.sn_relptr[s] + q] = (int)(it - Rp);
      }
    }
    // level sets by height in the supernodal elimination forest
    std::vector<int> height(ns, 0);
    int nlev = 0;
    for (int s = 0; s < ns; ++s) {  // children precede parents
      for (int q = A.sn_child_ptr[s]; q < A.sn_child_ptr[s + 1]; ++q) height[s] = std::max(height[s], height[A.sn_child[q]] + 1);
      nlev = std::max(nlev, height[s] + 1);
    }
    A.level_ptr.assign(nlev + 1, 0);
    for (int s = 0; s < ns; ++s) A.level_ptr[height[s] + 1]++;
    for (int l = 0; l < nlev; ++l) A.level_ptr[l + 1] += A.level_ptr[l];
    A.level_sn.resize(ns);
    {
      std::vector<int> fill(A.level_ptr.begin(), A.level_ptr.end() - 1);
      for (int s = 0; s < ns; ++s) A.level_sn[fill[height[s]]++] = s;
    }
    // supernode of each factor column
    std::vector<int> sn_of_col(n);
    for (int s = 0; s < ns; ++s)
      for (int j = 0; j < A.sn_ncol[s]; ++j) sn_of_col[A.sn_first[s] + j] = s;
    auto lidx = [&](int vi, int vj) -> long long {
      int r = A.perm[vi], c = A.perm[vj];
      if (r < c) std::swap(r, c);
      const int s = sn_of_col[c];
      const int* R = A.sn_rows.data() + A.sn_rowptr[s];
      const int* it = std::lower_bound(R, R + A.sn_nrow[s], r);
      if (it == R + A.sn_nrow[s] || *it != r) throw std::runtime_error("matrix entry outside the factor pattern");
      return A.sn_Lptr[s] + (long long)(c - A.sn_first[s]) * A.sn_nrow[s] + (it - R);
    };
    // assembly map: every stored term of K_c, grouped by its factor position.
    // Each instance's terms land in its own panels, which follow the previous
    // instance's, so the map is built per instance (on several host threads)
    // and the instances' parts are concatenated in order.
    struct Term { long long L; int type, a, b; };  // type 0 diag (a = var), 1 W (a = slot), 2 HDH (a, b slots)
    struct MapPart {
      std::vector<long long> tgt_L;
      std::vector<int> tgt_diag, tw_cnt, tw_idx, th_cnt, th_a, th_b;
    };
    std::vector<MapPart> parts(ni);
    parallel_for(ni, [&](int i) {
      const int vo = A.inst_voff[i], nl = A.inst_n[i];
      const long long wo = A.inst_woff[i], nWi = (long long)sp.T[i] * WS;
      const long long ro = A.inst_roff[i], ml = A.inst_m[i];
      std::vector<Term> terms;
      terms.reserve((size_t)nl + nWi + (size_t)ml * WH * 3);
      for (int v = vo; v < vo + nl; ++v) terms.push_back({lidx(v, v), 0, v, -1});
      for (long long s = wo; s < wo + nWi; ++s) if (Wi[s] >= 0) terms.push_back({lidx(Wi[s], Wj[s]), 1, (int)s, -1});
      for (long long r = ro; r < ro + ml; ++r)
        for (int a = 0; a < WH; ++a) {
          const int ca = A.Hcol[r * WH + a];
          if (ca < 0) continue;
          for (int b = 0; b <= a; ++b) {
            const int cb = A.Hcol[r * WH + b];
            if (cb < 0) continue;
            terms.push_back({lidx(ca, cb), 2, (int)(r * WH + a), (int)(r * WH + b)});
          }
        }
      std::stable_sort(terms.begin(), terms.end(), [](const Term& x, const Term& y) {
        return x.L < y.L || (x.L == y.L && x.type < y.type);
      });
      MapPart& P = parts[i];
      for (size_t q = 0; q < terms.size();) {
        const long long L = terms[q].L;
        P.tgt_L.push_back(L);
        int diag = -1, nw = 0, nh = 0;
        for (; q < terms.size() && terms[q].L == L; ++q) {
          const Term& t = terms[q];
          if (t.type == 0) diag = t.a;
          else if (t.type == 1) { P.tw_idx.push_back(t.a); ++nw; }
          else { P.th_a.push_back(t.a); P.th_b.push_back(t.b); ++nh; }
        }
        P.tgt_diag.push_back(diag);
        P.tw_cnt.push_back(nw);
        P.th_cnt.push_back(nh);
      }
    });
    A.tgt_L.clear(); A.tgt_diag.clear(); A.tw_idx.clear(); A.th_a.clear(); A.th_b.clear();
    A.tw_ptr.assign(1, 0); A.th_ptr.assign(1, 0);
    for (const MapPart& P : parts) {
      A.tgt_L.insert(A.tgt_L.end(), P.tgt_L.begin(), P.tgt_L.end());
      A.tgt_diag.insert(A.tgt_diag.end(), P.tgt_diag.begin(), P.tgt_diag.end());
      A.tw_idx.insert(A.tw_idx.end(), P.tw_idx.begin(), P.tw_idx.end());
      A.th_a.insert(A.th_a.end(), P.th_a.begin(), P.th_a.end());
      A.th_b.insert(A.th_b.end(), P.th_b.begin(), P.th_b.end());
      for (size_t t = 0; t < P.tgt_L.size(); ++t) {
        A.tw_ptr.push_back(A.tw_ptr.back() + P.tw_cnt[t]);
        A.th_ptr.push_back(A.th_ptr.back() + P.th_cnt[t]);
      }
    }
    // Reduction chunks (never crossing an instance).  A block reduces one
    // chunk, RED_CHUNK threads striding over it; a chunk holds RED_CHUNK x E
    // elements with E chosen so that the whole problem still gives about
    // RED_TARGET_BLOCKS blocks (E = 1 for a single small instance, whose
    // reductions are latency-bound; up to 16 for wide batches, where the tree
    // reduction of a 128-element chunk would cost more than its elements).
    long long tot_el = 0;
    for (int i = 0; i < ni; ++i) tot_el += (long long)A.inst_n[i] + A.inst_m[i];
    const int E = (int)std::max(1LL, std::min(16LL, tot_el / ((long long)RED_TARGET_BLOCKS * RED_CHUNK)));
    const int CH = RED_CHUNK * E;
    A.red_chunk_elems = CH;
    A.chunks.clear();
    A.inst_chunk_ptr.assign(ni + 1, 0);
    for (int i = 0; i < ni; ++i) {
      for (int b = 0; b < A.inst_n[i]; b += CH)
        A.chunks.push_back({i, 0, A.inst_voff[i] + b, A.inst_voff[i] + std::min(A.inst_n[i], b + CH)});
      for (int b = 0; b < A.inst_m[i]; b += CH)
        A.chunks.push_back({i, 1, A.inst_roff[i] + b, A.inst_roff[i] + std::min(A.inst_m[i], b + CH)});
      A.inst_chunk_ptr[i + 1] = (int)A.chunks.size();
    }
    // Within each variable chunk, variables by descending column length of H
    // (stable): the H^T products loop over a column, and a warp runs as many
    // FP64 iterations as its longest column, whatever the other lanes need.
    A.red_var.resize(A.n);
    std::iota(A.red_var.begin(), A.red_var.end(), 0);
    for (const Chunk& c : A.chunks) {
      if (c.kind != 0) continue;
      std::stable_sort(A.red_var.begin() + c.begin, A.red_var.begin() + c.end, [&](int a, int b) {
        return A.Hcsc_ptr[a + 1] - A.Hcsc_ptr[a] > A.Hcsc_ptr[b + 1] - A.Hcsc_ptr[b];
      });
    }
    A.inst_chunk_list.resize(A.chunks.size());
    std::iota(A.inst_chunk_list.begin(), A.inst_chunk_list.end(), 0);
  } catch (const std::exception& e) {
    return std::string("structure analysis failed: ") + e.what();
  }
  A.analysis_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return "";
}

}  // namespace nmpc
