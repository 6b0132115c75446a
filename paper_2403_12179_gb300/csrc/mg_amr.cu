// Two-level AMR composite Poisson solve (coarse level over the domain, one refined box region,
// refinement ratio 2) on sm_103a.
//
// The AMReX/pyAMReX review (Sec. 1, Sec. 2) describes the block-structured AMR hierarchy --
// a coarse level covering the domain, finer levels covering sub-regions, inter-level
// operations between them and cached communication patterns -- and the framework's linear
// solvers for cell-centered data.  The composite discretisation here is the reading this
// library documents in gbmg.h (mg_amr2_solve):
//   * fine ghost cells across the coarse/fine boundary come from quadratic interpolation:
//     tangentially over the 3 x 3 coarse cells of the layer outside the fine region (3-point
//     Lagrange weights at the fine centre's offset of -1/4 or +1/4 coarse cells), then along
//     the normal through that value and the first two fine cells inside
//     (g = 8/15 c + 2/3 f1 - 1/5 f2);
//   * a coarse cell next to the fine region takes, on the shared face, the mean of the four
//     fine fluxes through it (flux matching), so the composite operator is conservative.
// Both are inter-level "tag lists" built once on the host, like the ghost fill's copy tags:
// one entry per coarse/fine ghost cell (its destination, the two fine cells and the nine
// coarse cells it reads) and one per coarse cell on the interface.
//
// The solve iterates on the composite residual r = f - A phi (stop test before each
// iteration, max over fine cells and uncovered coarse cells):
//   1. coarse correction: rhs = r on uncovered coarse cells and the mean of the fine residual
//      on covered ones; e0 = one V(nu1, nu2) cycle of the single-level solver from 0;
//      phi0 += e0, and every fine cell adds its parent's e0;
//   2. nu1 + nu2 red-black sweeps on the fine level, the coarse/fine ghosts refreshed from
//      phi0 before each colour;
//   3. covered coarse cells take the mean of their 8 fine children.
// Every step is one launch over all boxes of its level (Sec. 3.2).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "mg_runtime.hpp"
#include "mg_solver.hpp"

namespace gbmg {

namespace {

// One coarse/fine ghost cell: element offsets into the fine phi fab (the ghost, the first and
// second fine cells inside along the normal) and into the coarse phi fab (c[3q + p]: tangential
// offsets p - 1 along the lower tangential dimension, q - 1 along the other); par bit 0 / 1:
// the fine cell sits in the upper half of its parent along the lower / other tangential
// dimension (weights at +1/4), else the lower half (-1/4).
struct CFGhost {
  long long dst, f1, f2;
  long long c[9];
  int par;
  int pad_;
};

// One coarse cell beside the fine region: its residual (offset into the coarse residual fab),
// its phi and the covered neighbour's phi (coarse phi fab), and the four fine cells across the
// shared face with their coarse/fine ghosts (fine phi fab).
struct RefluxCell {
  long long r, pc, pn;
  long long f[4], g[4];
};

__constant__ double kWLo[3] = {5.0 / 32.0, 15.0 / 16.0, -3.0 / 32.0};  // offset -1/4
__constant__ double kWHi[3] = {-3.0 / 32.0, 15.0 / 16.0, 5.0 / 32.0};  // offset +1/4
constexpr double kN0 = 8.0 / 15.0, kN1 = 2.0 / 3.0, kN2 = -1.0 / 5.0;

// g = 8/15 c + 2/3 f1 - 1/5 f2 with c = sum_q w1[q] (sum_p w0[p] C[p, q]), each sum in
// index order as fused multiply-adds.
__global__ void __launch_bounds__(256) k_cf_ghosts(const CFGhost* __restrict__ T, int n,
                                                   double* __restrict__ fine,
                                                   const double* __restrict__ coarse) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const CFGhost& e = T[i];
  const double* w0 = (e.par & 1) ? kWHi : kWLo;
  const double* w1 = (e.par & 2) ? kWHi : kWLo;
  double c = 0.0;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    double cq = __dmul_rn(w0[0], coarse[e.c[3 * q]]);
    cq = __fma_rn(w0[1], coarse[e.c[3 * q + 1]], cq);
    cq = __fma_rn(w0[2], coarse[e.c[3 * q + 2]], cq);
    c = q == 0 ? __dmul_rn(w1[0], cq) : __fma_rn(w1[q], cq, c);
  }
  const double f1 = fine[e.f1], f2 = fine[e.f2];
  fine[e.dst] = __fma_rn(kN0, c, __fma_rn(kN1, f1, __dmul_rn(kN2, f2)));
}

// r += (F_coarse - F_fine) / h0 with the outward fluxes of the shared face:
// F_coarse = (phi_n - phi_c) / h0 (what the single-level residual used), F_fine = the mean of
// the four (phi_f - g_f) / h1.
__global__ void __launch_bounds__(256) k_reflux(const RefluxCell* __restrict__ T, int n,
                                                double* __restrict__ r,
                                                const double* __restrict__ coarse,
                                                const double* __restrict__ fine, double ih0,
                                                double ih1) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const RefluxCell& e = T[i];
  double s = __dsub_rn(fine[e.f[0]], fine[e.g[0]]);
#pragma unroll
  for (int k = 1; k < 4; ++k) s = __dadd_rn(s, __dsub_rn(fine[e.f[k]], fine[e.g[k]]));
  const double ff = __dmul_rn(s, 0.25 * ih1);
  const double fc = __dmul_rn(__dsub_rn(coarse[e.pn], coarse[e.pc]), ih0);
  r[e.r] = __fma_rn(__dsub_rn(fc, ff), ih0, r[e.r]);
}

// ---- host planning -------------------------------------------------------------------

struct AmrPlan {
  int64_t phi0 = 0, phi1 = 0, rhs0 = 0, rhs1 = 0;
  int bc_key = 0;
  double h_req = 0;  // the cell size asked for (0: default)
  int A[3], B[3];
  double h0 = 0, h1 = 0;
  mg_bc bc{}, fine_bc{};
  int64_t r0 = 0, e0 = 0, r1 = 0;  // work fabs (registered handles)
  std::shared_ptr<Hierarchy> H;    // single-level cycle on (r0, e0)
  DevBufP cf, rf;
  int ncf = 0, nrf = 0;
  bool fine_direct = false, coarse_direct = false;  // tables read neighbouring boxes directly
  OpTable fine_smooth, fine_resid, coarse_resid, coarse_copy_f, fine_copy_f, avg_down,
      restrict_r, prolong, add0, rmax0, rmax1;
  DevBufP dnorm;
  unsigned long long* hnorm = nullptr;
  // one composite iteration (correction, fine sweeps, average-down, residual + norm) as a
  // CUDA graph, captured on `graph_stream` with `graph_kernels` kernels
  cudaGraphExec_t step = nullptr;
  cudaStream_t graph_stream = nullptr;
  long long graph_kernels = 0;
  ~AmrPlan() {
    if (step) cudaGraphExecDestroy(step);
    if (hnorm) cudaFreeHost(hnorm);
  }
};

std::mutex g_amr_mu;
std::map<Ctx*, std::vector<std::shared_ptr<AmrPlan>>> g_plans;

// Element offset of global cell (x, y, z) of a fab (the box owning it).
struct Owner {
  const FabObj* f;
  std::map<std::array<int, 3>, int> cell_box;  // only the cells asked about, cached
  long long at(int x, int y, int z) {
    const BoxArray& ba = f->ba->ba;
    auto key = std::array<int, 3>{x, y, z};
    auto it = cell_box.find(key);
    int b = -1;
    if (it != cell_box.end()) {
      b = it->second;
    } else {
      for (size_t k = 0; k < ba.boxes.size(); ++k)
        if (contains(ba.boxes[k], x, y, z)) { b = (int)k; break; }
      if (b < 0) fail(MG_EINVAL, "internal: cell outside every box");
      cell_box[key] = b;
    }
    return f->lay.at(ba, b, x, y, z);
  }
};

DView sub_view(const FabObj& f, int b, const int lo[3]) {
  DView v = f.view(b);
  const Box& B = f.ba->ba.boxes[b];
  long long o = (long long)(lo[2] - B.lo[2]) * v.plane + (long long)(lo[1] - B.lo[1]) * v.pitch +
                (lo[0] - B.lo[0]);
  v.p = (char*)v.p + o * f.esize();
  return v;
}

// Pieces of the fine boxes whose parent cells lie in one coarse box each: (fine box, coarse
// box, fine piece).
struct Piece {
  int fb, cb;
  Box fine;
};
std::vector<Piece> pieces(const BoxArray& F, const BoxArray& C) {
  std::vector<Piece> out;
  for (size_t fb = 0; fb < F.boxes.size(); ++fb) {
    const Box& X = F.boxes[fb];
    Box par;
    for (int d = 0; d < 3; ++d) { par.lo[d] = fdiv2(X.lo[d]); par.hi[d] = fdiv2(X.hi[d]); }
    for (size_t cb = 0; cb < C.boxes.size(); ++cb) {
      Box s = intersect(par, C.boxes[cb]);
      if (s.empty()) continue;
      Box f;
      for (int d = 0; d < 3; ++d) { f.lo[d] = 2 * s.lo[d]; f.hi[d] = 2 * s.hi[d] + 1; }
      out.push_back({(int)fb, (int)cb, f});
    }
  }
  return out;
}

template <class V>
OpTable piece_table(Ctx& c, const std::vector<Piece>& P, const Box& fdom, int kind, V&& views,
                    cudaStream_t s) {
  BoxArray ba;
  ba.dom = fdom;
  for (const Piece& p : P) ba.boxes.push_back(p.fine);
  return make_table(c, ba, kind, 1.0, 0, [&](int i, DRow& R) { views(P[i], R); }, s);
}

AmrPlan& get_plan(Ctx& c, int64_t rhs0, int64_t phi0, int64_t rhs1, int64_t phi1, const mg_bc* bc,
                  const SolveParams& p) {
  int per[3];
  const int key = bc_code(bc, per);
  std::lock_guard<std::mutex> lk(g_amr_mu);
  auto same = [&](const SolveParams& a) {
    return a.nu1 == p.nu1 && a.nu2 == p.nu2 && a.smoother == p.smoother &&
           a.coarse_cells == p.coarse_cells && a.direct_reads == p.direct_reads &&
           a.prolong == p.prolong && a.use_graph == p.use_graph;
  };
  for (auto& P : g_plans[&c])
    if (P->phi0 == phi0 && P->phi1 == phi1 && P->rhs0 == rhs0 && P->rhs1 == rhs1 &&
        P->bc_key == key && same(P->H->p) && P->h_req == p.h)
      return *P;
  auto f0 = c.get_fab(phi0), f1 = c.get_fab(phi1), g0 = c.get_fab(rhs0), g1 = c.get_fab(rhs1);
  for (auto* f : {f0.get(), f1.get(), g0.get(), g1.get()})
    if (f->dtype != DT_F64 || f->lay.ncomp != 1)
      fail(MG_EINVAL, "mg_amr2_solve needs FP64 one-component fabs");
  if (f0->lay.g < 1 || f1->lay.g < 1) fail(MG_EINVAL, "phi fabs need at least one ghost layer");
  const BoxArray& C = f0->ba->ba;
  const BoxArray& F = f1->ba->ba;
  if (!aligned(F)) fail(MG_EINVAL, "fine boxes must have even bounds (whole 2x2x2 child groups)");
  if (g0->ba->ba.boxes.size() != C.boxes.size() || g1->ba->ba.boxes.size() != F.boxes.size() ||
      std::memcmp(g0->ba->ba.boxes.data(), C.boxes.data(), C.boxes.size() * sizeof(Box)) != 0 ||
      std::memcmp(g1->ba->ba.boxes.data(), F.boxes.data(), F.boxes.size() * sizeof(Box)) != 0)
    fail(MG_EINVAL, "rhs and phi of a level must share a box array");
  auto P = std::make_shared<AmrPlan>();
  P->phi0 = phi0; P->phi1 = phi1; P->rhs0 = rhs0; P->rhs1 = rhs1; P->bc_key = key; P->bc = *bc;
  P->h_req = p.h;
  int n0[3], n1[3];
  for (int d = 0; d < 3; ++d) {
    n0[d] = C.dom.len(d);
    n1[d] = F.dom.len(d);
    if (C.dom.lo[d] != 0) fail(MG_EINVAL, "the coarse domain must start at 0");
    if ((F.dom.lo[d] & 1) || (n1[d] & 1))
      fail(MG_EINVAL, "the fine domain must be a coarse box region refined by 2");
    P->A[d] = F.dom.lo[d] / 2;
    P->B[d] = P->A[d] + n1[d] / 2;
    if (P->A[d] < 1 || P->B[d] > n0[d] - 1)
      fail(MG_EINVAL, "the refined region must stay one coarse cell away from every domain face");
  }
  P->h0 = p.h > 0 ? p.h : 1.0 / n0[0];
  P->h1 = P->h0 / 2;
  for (int d = 0; d < 3; ++d) P->fine_bc.kind[d][0] = P->fine_bc.kind[d][1] = MG_BC_DIRICHLET0;
  cudaStream_t s = c.stream;
  // work fabs: the composite residual of both levels and the coarse correction
  P->r0 = add_pool_fab(c, f0->ba, f0->ba_id, 1, 0, DT_F64, s);
  P->e0 = add_pool_fab(c, f0->ba, f0->ba_id, 1, 1, DT_F64, s);
  P->r1 = add_pool_fab(c, f1->ba, f1->ba_id, 1, 0, DT_F64, s);
  auto r0 = c.get_fab(P->r0), e0 = c.get_fab(P->e0), r1 = c.get_fab(P->r1);
  SolveParams pc = p;
  pc.h = P->h0;
  pc.precision = MG_PREC_F64;
  {
    std::lock_guard<std::recursive_mutex> hl(c.hier_mu);
    Hierarchy& H = get_hierarchy(c, *r0, *e0, bc, pc);
    for (auto& h : c.hier)
      if (h.get() == &H) P->H = h;
  }
  // coarse/fine ghost list
  Owner of{f1.get(), {}}, oc{f0.get(), {}};
  std::vector<CFGhost> cf;
  for (int d = 0; d < 3; ++d) {
    const int t0 = d == 0 ? 1 : 0, t1 = d == 2 ? 1 : 2;
    for (int side = 0; side < 2; ++side) {
      const int X = side == 0 ? P->A[d] - 1 : P->B[d];
      const int fin1 = side == 0 ? F.dom.lo[d] : F.dom.hi[d];
      const int step = side == 0 ? 1 : -1;
      for (int j = F.dom.lo[t1]; j <= F.dom.hi[t1]; ++j)
        for (int i = F.dom.lo[t0]; i <= F.dom.hi[t0]; ++i) {
          CFGhost e{};
          int q1[3], q2[3];
          q1[d] = fin1;
          q2[d] = fin1 + step;
          q1[t0] = q2[t0] = i;
          q1[t1] = q2[t1] = j;
          e.f1 = of.at(q1[0], q1[1], q1[2]);
          e.f2 = of.at(q2[0], q2[1], q2[2]);
          // the ghost lives in the box of the first fine cell, one cell outside along d
          const int gb = of.cell_box[{q1[0], q1[1], q1[2]}];
          int gq[3] = {q1[0], q1[1], q1[2]};
          gq[d] -= step;
          e.dst = f1->lay.at(F, gb, gq[0], gq[1], gq[2]);
          const int P0 = fdiv2(i), P1 = fdiv2(j);
          for (int qq = 0; qq < 3; ++qq)
            for (int pp = 0; pp < 3; ++pp) {
              int cc[3];
              cc[d] = X;
              cc[t0] = P0 + pp - 1;
              cc[t1] = P1 + qq - 1;
              e.c[3 * qq + pp] = oc.at(cc[0], cc[1], cc[2]);
            }
          e.par = (i & 1) | ((j & 1) << 1);
          cf.push_back(e);
        }
    }
  }
  P->ncf = (int)cf.size();
  P->cf = c.upload(cf.data(), cf.size() * sizeof(CFGhost), s);
  // coarse cells beside the fine region, with the four fine faces of their shared face
  Owner orr{r0.get(), {}};
  std::vector<RefluxCell> rf;
  for (int d = 0; d < 3; ++d) {
    const int t0 = d == 0 ? 1 : 0, t1 = d == 2 ? 1 : 2;
    for (int side = 0; side < 2; ++side) {
      const int X = side == 0 ? P->A[d] - 1 : P->B[d];      // the uncovered coarse cell
      const int Xn = side == 0 ? P->A[d] : P->B[d] - 1;     // its covered neighbour
      const int fin1 = side == 0 ? F.dom.lo[d] : F.dom.hi[d];
      const int step = side == 0 ? 1 : -1;
      for (int J = P->A[t1]; J < P->B[t1]; ++J)
        for (int I = P->A[t0]; I < P->B[t0]; ++I) {
          RefluxCell e{};
          int cc[3], cn[3];
          cc[d] = X;
          cn[d] = Xn;
          cc[t0] = cn[t0] = I;
          cc[t1] = cn[t1] = J;
          e.r = orr.at(cc[0], cc[1], cc[2]);
          e.pc = oc.at(cc[0], cc[1], cc[2]);
          e.pn = oc.at(cn[0], cn[1], cn[2]);
          int k = 0;
          for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a, ++k) {
              int q[3];
              q[d] = fin1;
              q[t0] = 2 * I + a;
              q[t1] = 2 * J + b;
              e.f[k] = of.at(q[0], q[1], q[2]);
              const int gb = of.cell_box[{q[0], q[1], q[2]}];
              q[d] -= step;
              e.g[k] = f1->lay.at(F, gb, q[0], q[1], q[2]);
            }
          rf.push_back(e);
        }
    }
  }
  P->nrf = (int)rf.size();
  P->rf = c.upload(rf.data(), rf.size() * sizeof(RefluxCell), s);
  // level tables.  On a regular grid of fine boxes the fine stencils read neighbouring fine
  // boxes directly and only the coarse/fine ghosts of the region's faces (written by
  // k_cf_ghosts) as ghost cells; the coarse residual reads neighbouring boxes directly too.
  const int no_periodic[3] = {0, 0, 0};
  const FaceReads frf = direct_neighbours(*f1, no_periodic, true);
  const FaceReads frc = direct_neighbours(*f0, per);
  P->fine_direct = frf.ok();
  P->coarse_direct = frc.ok();
  P->fine_smooth = make_table(c, F, 0, P->h1, 0, [&](int b, DRow& R) {
    R.v[0] = f1->view(b);
    R.v[1] = g1->view(b);
    frf.apply(b, R);
  }, s);
  P->fine_resid = make_table(c, F, 0, P->h1, 0, [&](int b, DRow& R) {
    R.v[0] = f1->view(b);
    R.v[1] = g1->view(b);
    R.v[2] = r1->view(b);
    frf.apply(b, R);
  }, s);
  P->coarse_resid = make_table(c, C, 0, P->h0, 0, [&](int b, DRow& R) {
    R.v[0] = f0->view(b);
    R.v[1] = g0->view(b);
    R.v[2] = r0->view(b);
    frc.apply(b, R);
  }, s);
  P->coarse_copy_f = make_table(c, C, 0, P->h0, 0, [&](int b, DRow& R) {
    R.v[0] = r0->view(b);
    R.v[1] = g0->view(b);
  }, s);
  P->add0 = make_table(c, C, 0, P->h0, 0, [&](int b, DRow& R) {
    R.v[0] = f0->view(b);
    R.v[1] = e0->view(b);
  }, s);
  P->fine_copy_f = make_table(c, F, 0, P->h1, 0, [&](int b, DRow& R) {
    R.v[0] = r1->view(b);
    R.v[1] = g1->view(b);
  }, s);
  P->rmax0 = make_table(c, C, 0, P->h0, 0, [&](int b, DRow& R) { R.v[0] = r0->view(b); }, s);
  P->rmax1 = make_table(c, F, 0, P->h1, 0, [&](int b, DRow& R) { R.v[0] = r1->view(b); }, s);
  const std::vector<Piece> pcs = pieces(F, C);
  P->avg_down = piece_table(c, pcs, F.dom, 1, [&](const Piece& q, DRow& R) {
    R.v[0] = sub_view(*f1, q.fb, q.fine.lo);
    int clo[3] = {q.fine.lo[0] / 2, q.fine.lo[1] / 2, q.fine.lo[2] / 2};
    R.c[0] = sub_view(*f0, q.cb, clo);
  }, s);
  P->restrict_r = piece_table(c, pcs, F.dom, 1, [&](const Piece& q, DRow& R) {
    R.v[0] = sub_view(*r1, q.fb, q.fine.lo);
    int clo[3] = {q.fine.lo[0] / 2, q.fine.lo[1] / 2, q.fine.lo[2] / 2};
    R.c[0] = sub_view(*r0, q.cb, clo);
  }, s);
  P->prolong = piece_table(c, pcs, F.dom, 0, [&](const Piece& q, DRow& R) {
    R.v[0] = sub_view(*f1, q.fb, q.fine.lo);
    int clo[3] = {q.fine.lo[0] / 2, q.fine.lo[1] / 2, q.fine.lo[2] / 2};
    R.c[0] = sub_view(*e0, q.cb, clo);
  }, s);
  fill_plan(c, *f1, &P->fine_bc, 1);
  fill_plan(c, *f0, bc, 1);
  P->dnorm = c.alloc(16, s);
  MG_CK(cudaMallocHost(&P->hnorm, 16));
  MG_CK(cudaStreamSynchronize(s));
  g_plans[&c].push_back(P);
  return *P;
}

// Coarse/fine ghosts of phi1 from phi0 (after the fine level's own fill).
void fill_fine(Ctx& c, AmrPlan& P, FabObj& f0, FabObj& f1, cudaStream_t s) {
  if (!P.fine_direct) launch_fill(c, f1, &P.fine_bc, s, 1);
  if (P.ncf) {
    launch_k(k_cf_ghosts, (P.ncf + 255) / 256, 256, 0, s, (const CFGhost*)P.cf->p, P.ncf,
                                                    (double*)f1.base, (const double*)f0.base);
    count_launches(1);
    MG_CK(cudaGetLastError());
  }
}

// Composite residual into r0 (covered cells: the mean of the fine residual) and r1; its
// max-norm into dnorm[0] (bit pattern).
void enqueue_residual(Ctx& c, AmrPlan& P, cudaStream_t s) {
  auto f0 = c.get_fab(P.phi0), f1 = c.get_fab(P.phi1);
  auto r0 = c.get_fab(P.r0);
  unsigned long long* dn = (unsigned long long*)P.dnorm->p;
  fill_fine(c, P, *f0, *f1, s);
  MG_CK(launch_residual(DT_F64, P.fine_resid.rows(), P.fine_resid.nbox, P.fine_resid.nrows,
                        nullptr, s, P.fine_direct));
  if (!P.coarse_direct) launch_fill(c, *f0, &P.bc, s, 1);
  MG_CK(launch_residual(DT_F64, P.coarse_resid.rows(), P.coarse_resid.nbox,
                        P.coarse_resid.nrows, nullptr, s, P.coarse_direct));
  if (P.nrf) {
    launch_k(k_reflux, (P.nrf + 255) / 256, 256, 0, s, (const RefluxCell*)P.rf->p, P.nrf,
                                                  (double*)r0->base, (const double*)f0->base,
                                                  (const double*)f1->base, 1.0 / P.h0, 1.0 / P.h1);
    count_launches(1);
    MG_CK(cudaGetLastError());
  }
  MG_CK(launch_restrict(DT_F64, P.restrict_r.rows(), P.restrict_r.nbox, P.restrict_r.nrows, s));
  MG_CK(cudaMemsetAsync(dn, 0, 8, s));
  MG_CK(launch_maxabs(DT_F64, P.rmax0.rows(), P.rmax0.nbox, P.rmax0.nrows, dn, s));
  MG_CK(launch_maxabs(DT_F64, P.rmax1.rows(), P.rmax1.nbox, P.rmax1.nrows, dn, s));
}

double bits2d(unsigned long long b) {
  double d;
  std::memcpy(&d, &b, 8);
  return d;
}

}  // namespace

namespace {
void release_plan(Ctx& c, AmrPlan& P) {
  cudaStreamSynchronize(c.stream);
  if (P.step) {
    cudaGraphExecDestroy(P.step);
    P.step = nullptr;
  }
  if (P.H) {
    std::lock_guard<std::recursive_mutex> hl(c.hier_mu);
    std::vector<std::shared_ptr<Hierarchy>> rest;
    for (auto& h : c.hier)
      if (h != P.H) rest.push_back(h);
    c.hier.swap(rest);
    P.H.reset();
  }
  for (int64_t id : {P.r0, P.e0, P.r1})
    if (id) release_fab(c, id, c.stream);
}
}  // namespace

void amr_drop_plans(Ctx& c, int64_t fab) {
  std::vector<std::shared_ptr<AmrPlan>> gone;
  {
    std::lock_guard<std::mutex> lk(g_amr_mu);
    auto it = g_plans.find(&c);
    if (it == g_plans.end()) return;
    std::vector<std::shared_ptr<AmrPlan>> keep;
    for (auto& P : it->second) {
      const bool uses = fab == 0 || P->phi0 == fab || P->phi1 == fab || P->rhs0 == fab ||
                        P->rhs1 == fab;
      (uses ? gone : keep).push_back(P);
    }
    if (keep.empty()) g_plans.erase(it);
    else it->second.swap(keep);
  }
  for (auto& P : gone) release_plan(c, *P);
}

}  // namespace gbmg

using namespace gbmg;

extern "C" {

int mg_amr2_residual(mg_ctx_t h, mg_fab_t rhs0, mg_fab_t phi0, mg_fab_t rhs1, mg_fab_t phi1,
                     const mg_bc* bc, double hh, mg_fab_t r0, mg_fab_t r1, double* norm) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    c->require_device();
    SolveParams p;
    p.h = hh;
    AmrPlan& P = get_plan(*c, rhs0, phi0, rhs1, phi1, bc, p);
    cudaStream_t s = c->stream;
    // covered coarse cells first take the mean of their fine children (the composite
    // unknowns are the fine cells and the uncovered coarse cells)
    MG_CK(launch_restrict(DT_F64, P.avg_down.rows(), P.avg_down.nbox, P.avg_down.nrows, s));
    enqueue_residual(*c, P, s);
    MG_CK(cudaMemcpyAsync(P.hnorm, P.dnorm->p, 8, cudaMemcpyDeviceToHost, s));
    auto w0 = c->get_fab(P.r0), w1 = c->get_fab(P.r1);
    auto o0 = r0 ? c->get_fab(r0) : nullptr, o1 = r1 ? c->get_fab(r1) : nullptr;
    if (o0) {
      if (o0->bytes < w0->bytes || o0->lay.g != 0) fail(MG_EINVAL, "r0 must match rhs0 without ghosts");
      MG_CK(cudaMemcpyAsync(o0->base, w0->base, w0->bytes, cudaMemcpyDeviceToDevice, s));
    }
    if (o1) {
      if (o1->bytes < w1->bytes || o1->lay.g != 0) fail(MG_EINVAL, "r1 must match rhs1 without ghosts");
      MG_CK(cudaMemcpyAsync(o1->base, w1->base, w1->bytes, cudaMemcpyDeviceToDevice, s));
    }
    MG_CK(cudaStreamSynchronize(s));
    if (norm) *norm = bits2d(P.hnorm[0]);
    return MG_OK;
  });
}

int mg_amr2_solve(mg_ctx_t h, mg_fab_t rhs0, mg_fab_t phi0, mg_fab_t rhs1, mg_fab_t phi1,
                  const mg_bc* bc, double tol, const mg_options* opt, mg_result* res) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    c->require_device();
    if (!(tol >= 0)) fail(MG_EINVAL, "tol must be >= 0");
    auto f0 = c->get_fab(phi0), f1 = c->get_fab(phi1);
    SolveParams p = params_from(opt, f0->ba->ba);
    if (p.precision != MG_PREC_F64) fail(MG_EINVAL, "mg_amr2_solve runs in FP64");
    const double t_start = c->now();
    AmrPlan& P = get_plan(*c, rhs0, phi0, rhs1, phi1, bc, p);
    cudaStream_t s = c->stream;
    unsigned long long* dn = (unsigned long long*)P.dnorm->p;
    // ||f||_inf over the composite cells: r0 <- rhs0 and r1 <- rhs1, then the covered part of
    // r0 <- the mean of r1 (a mean of fine values cannot raise the maximum).  The covered
    // coarse phi takes the mean of the fine phi (the composite unknowns are the fine cells
    // and the uncovered coarse cells).
    MG_CK(cudaMemsetAsync(dn, 0, 8, s));
    MG_CK(launch_set_valid(DT_F64, P.rmax0.rows(), P.rmax0.nbox, P.rmax0.nrows, 0.0, s));
    MG_CK(launch_add_valid(DT_F64, P.coarse_copy_f.rows(), P.coarse_copy_f.nbox,
                           P.coarse_copy_f.nrows, s));
    MG_CK(launch_set_valid(DT_F64, P.rmax1.rows(), P.rmax1.nbox, P.rmax1.nrows, 0.0, s));
    MG_CK(launch_add_valid(DT_F64, P.fine_copy_f.rows(), P.fine_copy_f.nbox, P.fine_copy_f.nrows,
                           s));
    MG_CK(launch_restrict(DT_F64, P.restrict_r.rows(), P.restrict_r.nbox, P.restrict_r.nrows, s));
    MG_CK(launch_maxabs(DT_F64, P.rmax0.rows(), P.rmax0.nbox, P.rmax0.nrows, dn, s));
    MG_CK(launch_maxabs(DT_F64, P.rmax1.rows(), P.rmax1.nbox, P.rmax1.nrows, dn, s));
    MG_CK(launch_restrict(DT_F64, P.avg_down.rows(), P.avg_down.nbox, P.avg_down.nrows, s));
    MG_CK(cudaMemcpyAsync(P.hnorm, dn, 8, cudaMemcpyDeviceToHost, s));
    MG_CK(cudaStreamSynchronize(s));
    const double rhsnorm = bits2d(P.hnorm[0]);
    mg_result r{};
    r.t_start = t_start;
    int status = MG_OK, it = 0;
    double rn = 0.0;
    if (std::isnan(rhsnorm) || std::isinf(rhsnorm)) {
      status = MG_ENAN;
    } else {
      // one iteration after the stop test: coarse correction from the composite residual
      // (r0 is its right-hand side), fine sweeps with coarse/fine ghosts from the corrected
      // coarse level, average-down; then the composite residual and its norm
      auto body = [&] {
        enqueue_correction_cycle(*c, *P.H, s);
        MG_CK(launch_add_valid(DT_F64, P.add0.rows(), P.add0.nbox, P.add0.nrows, s));
        MG_CK(launch_prolong_add(DT_F64, P.prolong.rows(), P.prolong.nbox, P.prolong.nrows, s,
                                 P.prolong.width));
        for (int k = 0; k < p.nu1 + p.nu2; ++k)
          for (int color = 0; color < 2; ++color) {
            fill_fine(*c, P, *f0, *f1, s);
            MG_CK(launch_rbgs_half(DT_F64, P.fine_smooth.rows(), P.fine_smooth.nbox,
                                   P.fine_smooth.nrows, color, s, P.fine_direct, nullptr,
                                   P.fine_smooth.width));
          }
        MG_CK(launch_restrict(DT_F64, P.avg_down.rows(), P.avg_down.nbox, P.avg_down.nrows, s));
        enqueue_residual(*c, P, s);
        MG_CK(cudaMemcpyAsync(P.hnorm, dn, 8, cudaMemcpyDeviceToHost, s));
      };
      // replayed as a graph from the second iteration on (the first, eager, builds every
      // cached table the iteration uses)
      const bool graph = p.use_graph && s != nullptr && s != cudaStreamLegacy &&
                         s != cudaStreamPerThread;
      if (P.step && P.graph_stream != s) {
        cudaGraphExecDestroy(P.step);
        P.step = nullptr;
      }
      enqueue_residual(*c, P, s);
      MG_CK(cudaMemcpyAsync(P.hnorm, dn, 8, cudaMemcpyDeviceToHost, s));
      MG_CK(cudaStreamSynchronize(s));
      for (;;) {
        rn = bits2d(P.hnorm[0]);
        if (std::isnan(rn) || std::isinf(rn)) { status = MG_ENAN; break; }
        if (p.fixed_vcycles >= 0) {
          if (it == p.fixed_vcycles) break;
        } else {
          if (rn <= tol * rhsnorm) break;
          if (it == p.max_iter) { status = MG_NOT_CONVERGED; break; }
        }
        if (graph && it >= 1) {
          if (!P.step) {
            cudaGraph_t g = nullptr;
            const long long before = launches_so_far();
            MG_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            try {
              body();
            } catch (...) {
              cudaStreamEndCapture(s, &g);
              if (g) cudaGraphDestroy(g);
              count_launches(before - launches_so_far());
              throw;
            }
            MG_CK(cudaStreamEndCapture(s, &g));
            P.graph_kernels = launches_so_far() - before;  // captured, not executed
            count_launches(-P.graph_kernels);
            cudaError_t e = cudaGraphInstantiate(&P.step, g, 0);
            cudaGraphDestroy(g);
            MG_CK(e);
            P.graph_stream = s;
          }
          MG_CK(cudaGraphLaunch(P.step, s));
          count_launches(P.graph_kernels);
        } else {
          body();
        }
        MG_CK(cudaStreamSynchronize(s));
        ++it;
      }
    }
    // covered coarse cells: the mean of their fine children
    MG_CK(launch_restrict(DT_F64, P.avg_down.rows(), P.avg_down.nbox, P.avg_down.nrows, s));
    MG_CK(cudaStreamSynchronize(s));
    check_device_error(*c);
    r.status = status;
    r.vcycles = it;
    r.rel_resid = rhsnorm > 0 ? rn / rhsnorm : 0.0;
    r.t_end = c->now();
    r.seconds = r.t_end - t_start;
    if (res) *res = r;
    return status;
  });
}

}  // extern "C"
