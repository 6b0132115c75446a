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
  // FP64 solves whose finest level starts each V-cycle with a red half-sweep: that
  // half-sweep of the next cycle also takes the red cells' residual norm of the current
  // iterate (it computes the same neighbour sums), replacing a separate residual pass; it
  // runs speculatively at the end of each step, saving the red values it replaces in save0
  // (null when the solve does not speculate), and is undone if the stop test ends the solve.
  // res0 holds, within each V-cycle, the black cells' residuals that the last pre-smoothing
  // half-sweep stores for the residual + restriction (stored0: level 0's residual +
  // restriction table reads them; store0 is that half-sweep's table).  Both are one-colour
  // arrays (half a row per row, see launch_rbgs_half).
  DevBufP save0, res0;
  OpTable store0;
  bool stored0 = false;
  // step graphs: [0] plain step, [1] first step of a speculating solve (a whole V-cycle,
  // then the next one's red half-sweep), [2] later steps (the V-cycle without that red
  // half-sweep, then the next one's)
  cudaGraphExec_t step_graph[3] = {nullptr, nullptr, nullptr};
  long long graph_kernels[3] = {0, 0, 0};
  cudaStream_t graph_stream = nullptr;
  bool graph_timed = false;                  // the step graphs record sweep_ev
  cudaEvent_t sweep_ev[2] = {nullptr, nullptr};
  ~Hierarchy() {
    for (cudaGraphExec_t g : step_graph)
      if (g) cudaGraphExecDestroy(g);
    if (hnorm) cudaFreeHost(hnorm);
    for (cudaEvent_t e : sweep_ev)
      if (e) cudaEventDestroy(e);
  }
};


// Cached per (rhs fab, phi fab, bc, options); builds coarse levels, tables and plans.
Hierarchy& get_hierarchy(Ctx& c, FabObj& rhs, FabObj& phi, const mg_bc* bc, const SolveParams& p);

// One V-cycle for the hierarchy's problem from a zero guess: phi (the caller's level-0 fab,
// ghosts included) is zeroed, then the cycle is enqueued on s; no norm is taken.
void enqueue_correction_cycle(Ctx& c, Hierarchy& H, cudaStream_t s);

}  // namespace gbmg
