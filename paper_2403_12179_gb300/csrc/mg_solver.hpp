// Multigrid hierarchy shared by the single-solve driver (mg_solver.cu) and the batched /
// served drivers (mg_batch.cu).
#pragma once

#include "mg_runtime.hpp"

namespace gbmg {

struct LevelData {
  std::shared_ptr<BoxArrayObj> bao;
  double h = 1.0;
  std::shared_ptr<FabObj> phi, rhs;
  OpTable smooth, rr, prolong, zero;
  // the stencil tables read neighbouring boxes directly (no ghost fill before them)
  bool direct = false;
  // fused sweeps ping-pong between phi and phi2 (same layout)
  bool fused = false;
  std::shared_ptr<FabObj> phi2;
  FusedTable f_ab, f_ba;
};

struct Hierarchy {
  // cache key
  int64_t rhs_id = 0, phi_id = 0;
  int bc_key = 0;
  SolveParams p;
  mg_bc bc{};
  int dt = DT_F64;  // inner precision
  bool mixed = false;
  std::vector<LevelData> L;
  std::shared_ptr<FabObj> phi0, rhs0;  // the caller's fabs (FP64)
  std::shared_ptr<FabObj> r0;          // mixed: FP64 residual stored by each norm check
  bool direct0 = false;                // the norm check reads neighbouring boxes directly
  OpTable resid0, rhsabs0, scale0, correct0, zero0_64;
  DevBufP Mt, offr, offp, job;
  int N = 0;
  // levels [lc, L.size()) run as one coarse-cycle launch; lc == L.size(): not used
  int lc = 0;
  size_t csmem = 0;
  DevBufP cjob, coff;
  CoarseJob cjob_host{};
  DevBufP dnorm;  // [0] residual norm bits, [1] rhs norm bits
  unsigned long long* hnorm = nullptr;
  BottomJob job_host{};
  cudaGraphExec_t step_graph = nullptr;
  cudaStream_t graph_stream = nullptr;
  long long graph_kernels = 0;
  bool graph_timed = false;                  // the step graph records sweep_ev
  cudaEvent_t sweep_ev[2] = {nullptr, nullptr};
  ~Hierarchy() {
    if (step_graph) cudaGraphExecDestroy(step_graph);
    if (hnorm) cudaFreeHost(hnorm);
    for (cudaEvent_t e : sweep_ev)
      if (e) cudaEventDestroy(e);
  }
};


// Cached per (rhs fab, phi fab, bc, options); builds coarse levels, tables and plans.
Hierarchy& get_hierarchy(Ctx& c, FabObj& rhs, FabObj& phi, const mg_bc* bc, const SolveParams& p);

}  // namespace gbmg
