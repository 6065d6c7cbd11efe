// One-time structure analysis on the host (Sec. 3.2.3 SymCholesky plus the
// transcription's sparsity patterns).  Produces everything the device needs
// to re-run the numeric work of Algorithm 2 without touching structure again.
#pragma once
#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "nmpc_internal.h"

namespace nmpc {

struct ProblemSpec {
  int model = 0;
  std::vector<int> T;  // horizon per instance
  int N = 0, Nf = 0, g = 0, S = 0;
  double dt = 1.0;
  double alpha = 1.6, D = 0.2, F = 0.4, xF = 0.5, Ac = 1, At = 1, Ar = 1, wdu = 0.01;
  double kappa = 0.01, cq = 0.01, rho_u = 1e-3;
  double xlo = 0, xhi = 1, ulo = 1, uhi = 5;
  double wu = 0, ubar = 0;
  double Tb = 50.0, qloss = 10.0;
  double gamma = 1e-8, tol = 1e-8, pivtol = 1e-12, dw_max = 1e40;
  int ordering = 0;  // 0 auto, 1 natural, 2 nested dissection
  int nd_leaf = 1;
  int amalgamation = 0;
};

struct Analysis {
  ModelConst mc{};
  int n_inst = 0, n = 0, m = 0, nW = 0, sp_stride = 0;
  std::vector<int> inst_T, inst_voff, inst_roff, inst_woff, inst_n, inst_m, inst_nz;
  std::vector<int> var_inst, row_inst;
  std::vector<double> yL, yU;
  std::vector<int> Hcol;                    // m * WH
  std::vector<int> Hcsc_ptr, Hcsc_slot;     // column lists of H slots
  std::vector<int> Wadj_ptr, Wadj_slot, Wadj_other;  // per variable: W slots it takes part in, and the partner
  std::vector<int> perm, iperm;             // global: perm[var] = factor position
  // supernodes (global, instance after instance, each in postorder)
  std::vector<int> sn_first, sn_ncol, sn_nrow, sn_inst, sn_parent;
  std::vector<long long> sn_Lptr, sn_Uptr, sn_uvptr, sn_rowptr, sn_relptr;
  std::vector<int> sn_rows, sn_rel;
  std::vector<int> sn_child_ptr, sn_child;
  std::vector<int> level_ptr, level_sn;
  long long nnzL = 0, nU = 0, nuv = 0;
  // assembly map
  std::vector<long long> tgt_L;
  std::vector<int> tgt_diag, tw_ptr, tw_idx, th_ptr, th_a, th_b;
  // reduction chunks, and the variables of each variable chunk ordered by
  // their number of Jacobian entries (longest first)
  std::vector<Chunk> chunks;
  std::vector<int> inst_chunk_ptr, inst_chunk_list;
  std::vector<int> red_var;
  int red_chunk_elems = 0;
  // stats
  double factor_flops = 0, solve_flops = 0, analysis_ms = 0;
  long long nnzL_true = 0;
  int max_front = 0, ordering_used = 0, amalgamation_used = 0;
};

// Returns an empty string on success, else an error message.
std::string analyze(const ProblemSpec& spec, Analysis& out);

// Run f(0 .. n-1) on up to hardware_concurrency host threads (the first
// exception thrown by a task is rethrown after all threads have joined).
void parallel_for(int n, const std::function<void(int)>& f);

}  // namespace nmpc
