// Multigrid hierarchy and V-cycle driver.
//
// The paper (Sec. 2) only names a cell-centered linear solver; the cycle here is the one
// this library documents in gbmg.h: V(nu1, nu2) with red-black Gauss-Seidel, fused
// residual + restriction, piecewise-constant prolongation and an exact bottom solve, the
// stop test ||rhs - A phi||_inf <= tol ||rhs||_inf before each cycle.  Each stage is one
// launch over all boxes of a level; a whole cycle plus the next norm check is replayed as
// one CUDA graph.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "mg_runtime.hpp"
#include "mg_solver.hpp"

namespace gbmg {

namespace {

std::shared_ptr<FabObj> internal_fab(Ctx& c, std::shared_ptr<BoxArrayObj> ba, int g, int dt) {
  auto f = std::make_shared<FabObj>();
  f->ba = std::move(ba);
  f->dtype = dt;
  f->lay = make_layout(f->ba->ba, 1, g, f->esize());
  f->bytes = (size_t)f->lay.total * f->esize();
  f->own = c.alloc(f->bytes, c.stream);
  f->base = f->own->p;
  MG_CK(cudaMemsetAsync(f->base, 0, f->bytes, c.stream));
  return f;
}

bool same_boxes(const BoxArray& a, const BoxArray& b) {
  return a.boxes.size() == b.boxes.size() &&
         std::memcmp(a.boxes.data(), b.boxes.data(), a.boxes.size() * sizeof(Box)) == 0 &&
         std::memcmp(&a.dom, &b.dom, sizeof(Box)) == 0;
}

DView coarse_view_of(const FabObj& coarse, const Box& fine_box) {
  const BoxArray& C = coarse.ba->ba;
  Box p;
  for (int d = 0; d < 3; ++d) { p.lo[d] = fdiv2(fine_box.lo[d]); p.hi[d] = fdiv2(fine_box.hi[d]); }
  for (size_t cb = 0; cb < C.boxes.size(); ++cb) {
    if (intersect(p, C.boxes[cb]).npts() != p.npts()) continue;
    DView v = coarse.view((int)cb);
    const Box& B = C.boxes[cb];
    long long o = (long long)(p.lo[2] - B.lo[2]) * v.plane + (long long)(p.lo[1] - B.lo[1]) * v.pitch +
                  (p.lo[0] - B.lo[0]);
    v.p = (char*)v.p + o * coarse.esize();
    return v;
  }
  fail(MG_EINVAL, "internal: parent cells span several coarse boxes");
}

}  // namespace

namespace {

// Smallest level (cells) that the automatic smoother choice runs with the fused sweep (FP32).
// Measured on GB300 (mixed 256^3 / 512^3 solves, 512 batched solves): 256^3 beats 2^18, 2^21,
// 2^25 and fusing every level.
constexpr long long kFusedMinCells = 1ll << 24;

void build_tables(Ctx& c, Hierarchy& H, cudaStream_t s) {
  const int nl = (int)H.L.size();
  int per[3];
  bc_code(&H.bc, per);
  for (int l = 0; l < nl; ++l) {
    LevelData& D = H.L[l];
    const BoxArray& ba = D.bao->ba;
    // levels smoothed by half-sweeps may read neighbouring boxes instead of ghost cells
    FaceReads fr;
    if (H.p.direct_reads && !D.fused) fr = direct_neighbours(*D.phi, per);
    D.direct = fr.ok();
    D.smooth = make_table(c, ba, 0, D.h, 0, [&](int b, DRow& R) {
      R.v[0] = D.phi->view(b);
      R.v[1] = D.rhs->view(b);
      fr.apply(b, R);
    }, s);
    D.smooth.direct = D.direct;
    D.zero = make_table(c, ba, 0, D.h, 0, [&](int b, DRow& R) { R.v[0] = D.phi->view(b); }, s);
    if (D.fused) {
      D.f_ab = make_fused(c, ba, D.h, *D.phi, *D.rhs, *D.phi2, per, s);
      D.f_ba = make_fused(c, ba, D.h, *D.phi2, *D.rhs, *D.phi, per, s);
      if (!D.f_ab.ok || !D.f_ba.ok) D.fused = false;
    }
    if (l + 1 < nl) {
      const LevelData& C = H.L[l + 1];
      D.rr = make_table(c, ba, 1, D.h, 0, [&](int b, DRow& R) {
        R.v[0] = D.phi->view(b);
        R.v[1] = D.rhs->view(b);
        R.c[0] = coarse_view_of(*C.rhs, ba.boxes[b]);
        R.c[1] = coarse_view_of(*C.phi, ba.boxes[b]);
        fr.apply(b, R);
      }, s);
      D.rr.direct = D.direct;
      D.prolong = make_table(c, ba, 0, D.h, 0, [&](int b, DRow& R) {
        R.v[0] = D.phi->view(b);
        R.c[0] = coarse_view_of(*C.phi, ba.boxes[b]);
      }, s);
    }
  }
  // level-0 FP64 tables: norm check (and the mixed-precision scale / correction)
  const BoxArray& ba0 = H.L[0].bao->ba;
  const double h0 = H.L[0].h;
  FaceReads fr0;
  if (H.p.direct_reads) fr0 = direct_neighbours(*H.phi0, per);
  H.direct0 = fr0.ok();
  H.resid0 = make_table(c, ba0, 0, h0, 0, [&](int b, DRow& R) {
    R.v[0] = H.phi0->view(b);
    R.v[1] = H.rhs0->view(b);
    if (H.mixed) R.v[2] = H.r0->view(b);  // kept for the next outer iteration's scaling
    fr0.apply(b, R);
  }, s);
  H.resid0.direct = H.direct0;
  H.rhsabs0 = make_table(c, ba0, 0, h0, 1, [&](int b, DRow& R) { R.v[0] = H.rhs0->view(b); }, s);
  H.zero0_64 = make_table(c, ba0, 0, h0, 0, [&](int b, DRow& R) { R.v[0] = H.phi0->view(b); }, s);
  if (H.mixed) {
    H.scale0 = make_table(c, ba0, 0, h0, 0, [&](int b, DRow& R) {
      R.v[0] = H.r0->view(b);
      R.c[0] = H.L[0].rhs->view(b);
      R.c[1] = H.L[0].phi->view(b);
    }, s);
    H.correct0 = make_table(c, ba0, 0, h0, 0, [&](int b, DRow& R) {
      R.v[0] = H.phi0->view(b);
      R.c[0] = H.L[0].phi->view(b);
    }, s);
  }
  // bottom
  const LevelData& B = H.L.back();
  const BoxArray& bb = B.bao->ba;
  int n[3] = {bb.dom.len(0), bb.dom.len(1), bb.dom.len(2)};
  const std::vector<double>& Mt = bottom_matrix_t(c, n, per, B.h);
  long long N = bb.dom.npts();
  std::vector<long long> orhs(N), ophi(N);
  for (size_t b = 0; b < bb.boxes.size(); ++b) {
    const Box& X = bb.boxes[b];
    for (int z = X.lo[2]; z <= X.hi[2]; ++z)
      for (int y = X.lo[1]; y <= X.hi[1]; ++y)
        for (int x = X.lo[0]; x <= X.hi[0]; ++x) {
          long long i = ((long long)(z - bb.dom.lo[2]) * n[1] + (y - bb.dom.lo[1])) * n[0] +
                        (x - bb.dom.lo[0]);
          orhs[i] = B.rhs->lay.at(bb, (int)b, x, y, z);
          ophi[i] = B.phi->lay.at(bb, (int)b, x, y, z);
        }
  }
  H.N = (int)N;
  H.Mt = c.upload(Mt.data(), Mt.size() * 8, s);
  H.offr = c.upload(orhs.data(), N * 8, s);
  H.offp = c.upload(ophi.data(), N * 8, s);
  BottomJob J{};
  J.Mt = (const double*)H.Mt->p;
  J.off_rhs = (const long long*)H.offr->p;
  J.off_phi = (const long long*)H.offp->p;
  J.rhs = B.rhs->base;
  J.phi = B.phi->base;
  J.N = (int)N;
  H.job = c.upload(&J, sizeof J, s);
  H.job_host = J;
  // The coarse end of the cycle as one launch: from the first level with at most
  // `limit` cells whose levels (down to the bottom) fit into shared memory.
  H.lc = nl;
  const int limit = H.p.coarse_cells != 0 ? H.p.coarse_cells : (H.dt == DT_F64 ? 512 : 4096);
  // (the coarse-cycle kernel prolongs by injection: the trilinear form runs level by level)
  const bool one_launch = H.p.coarse_cells >= 0 && H.p.prolong == MG_PROLONG_CONSTANT;
  for (int l = std::max(0, nl - kMaxCoarseLevels); one_launch && l + 1 < nl; ++l) {
    if (H.L[l].bao->ba.dom.npts() > limit) continue;
    int ext[kMaxCoarseLevels][3];
    for (int k = l; k < nl; ++k)
      for (int d = 0; d < 3; ++d) ext[k - l][d] = H.L[k].bao->ba.dom.len(d);
    const size_t smem = coarse_smem_bytes(H.dt, ext, nl - l);
    if (smem > kCoarseSmemMax) continue;
    // level l's cells, dense and x fastest, in its phi and rhs fabs
    const LevelData& T = H.L[l];
    const BoxArray& tb = T.bao->ba;
    const long long nt = tb.dom.npts();
    std::vector<long long> offs(2 * nt);
    for (size_t b = 0; b < tb.boxes.size(); ++b) {
      const Box& X = tb.boxes[b];
      for (int z = X.lo[2]; z <= X.hi[2]; ++z)
        for (int y = X.lo[1]; y <= X.hi[1]; ++y)
          for (int x = X.lo[0]; x <= X.hi[0]; ++x) {
            long long i = ((long long)(z - tb.dom.lo[2]) * ext[0][1] + (y - tb.dom.lo[1])) *
                              ext[0][0] + (x - tb.dom.lo[0]);
            offs[i] = T.phi->lay.at(tb, (int)b, x, y, z);
            offs[nt + i] = T.rhs->lay.at(tb, (int)b, x, y, z);
          }
    }
    H.coff = c.upload(offs.data(), offs.size() * 8, s);
    CoarseJob& C = H.cjob_host;
    C = CoarseJob{};
    C.off_phi = (const long long*)H.coff->p;
    C.off_rhs = C.off_phi + nt;
    C.phi = T.phi->base;
    C.rhs = T.rhs->base;
    C.Mt = J.Mt;
    C.N = J.N;
    C.nlev = nl - l;
    C.nu1 = H.p.nu1;
    C.nu2 = H.p.nu2;
    for (int d = 0; d < 3; ++d) C.periodic[d] = per[d];
    int off = 0;
    for (int k = 0; k < C.nlev; ++k) {
      const LevelData& D = H.L[l + k];
      CoarseLevel& V = C.lev[k];
      for (int d = 0; d < 3; ++d) {
        V.n[d] = ext[k][d];
        V.lo[d] = D.bao->ba.dom.lo[d];
      }
      V.h2 = D.h * D.h;
      V.ih2 = 1.0 / (D.h * D.h);
      V.off_phi = off;
      off += (V.n[0] + 2) * (V.n[1] + 2) * (V.n[2] + 2);
      V.off_rhs = off;
      off += V.n[0] * V.n[1] * V.n[2];
    }
    H.csmem = smem;
    MG_CK(coarse_opt_in(H.dt, smem));
    H.cjob = c.upload(&C, sizeof C, s);
    H.lc = l;
    break;
  }
  // fill plans must exist before any graph capture
  for (auto& D : H.L) {
    fill_plan(c, *D.phi, &H.bc, 1);
    if (D.fused) {
      fill_plan(c, *D.phi, &H.bc, 2);
      fill_plan(c, *D.phi2, &H.bc, 2);
      fill_plan(c, *D.rhs, &H.bc, 1);
    }
  }
  fill_plan(c, *H.phi0, &H.bc, 1);
}

}  // namespace

Hierarchy& get_hierarchy(Ctx& c, FabObj& rhs, FabObj& phi, const mg_bc* bc, const SolveParams& p) {
  std::lock_guard<std::recursive_mutex> lk(c.hier_mu);
  int per[3];
  int key = bc_code(bc, per);
  for (auto& h : c.hier) {
    if (h->rhs_id == rhs.id && h->phi_id == phi.id && h->bc_key == key &&
        h->p.nu1 == p.nu1 && h->p.nu2 == p.nu2 && h->p.precision == p.precision &&
        h->p.smoother == p.smoother && h->p.h == p.h &&
        h->p.coarse_cells == p.coarse_cells && h->p.direct_reads == p.direct_reads &&
        h->p.prolong == p.prolong && h->p.inner == p.inner)
      return *h;
  }
  if (rhs.dtype != DT_F64 || phi.dtype != DT_F64) fail(MG_EINVAL, "mg_solve needs FP64 fabs");
  if (rhs.lay.ncomp != 1 || phi.lay.ncomp != 1) fail(MG_EINVAL, "mg_solve needs 1-component fabs");
  if (!same_boxes(rhs.ba->ba, phi.ba->ba)) fail(MG_EINVAL, "rhs and phi are on different box arrays");
  if (phi.lay.g < 1) fail(MG_EINVAL, "phi needs at least one ghost cell");
  const std::vector<BoxArray>& lev = phi.ba->hierarchy();
  for (size_t l = 0; l + 1 < lev.size(); ++l)
    if (!aligned(lev[l]))
      fail(MG_EINVAL, "box array not supported by the solver: a level has boxes with odd bounds");
  std::unique_ptr<Hierarchy> H(new Hierarchy);
  H->rhs_id = rhs.id;
  H->phi_id = phi.id;
  H->bc_key = key;
  H->p = p;
  H->bc = *bc;
  H->mixed = p.precision == MG_PREC_MIXED;
  H->dt = H->mixed ? DT_F32 : DT_F64;
  H->phi0 = c.get_fab(phi.id);
  H->rhs0 = c.get_fab(rhs.id);
  cudaStream_t s = c.stream;
  const int nl = (int)lev.size();
  H->L.resize(nl);
  double h = p.h;
  for (int l = 0; l < nl; ++l) {
    LevelData& D = H->L[l];
    D.h = h;
    h *= 2.0;
    if (l == 0) D.bao = phi.ba;
    else {
      D.bao = std::make_shared<BoxArrayObj>();
      D.bao->ba = lev[l];
    }
    // FP64 levels default to half-sweeps: on GB300 they are bound by the FP64 pipe, and the
    // fused sweep's redundant ring updates add FP64 work; large FP32 levels are bound by HBM
    // bandwidth, where the fused sweep halves the traffic.  Small levels are latency-bound:
    // there half-sweeps reading neighbour boxes directly need no ghost fills at all.
    const bool big = lev[l].dom.npts() >= kFusedMinCells;
    const bool want_fused = l + 1 < nl && (p.smoother == MG_SMOOTH_FUSED ||
                                           (p.smoother == MG_SMOOTH_AUTO && H->dt == DT_F32 && big));
    if (l == 0 && !H->mixed) {
      D.phi = H->phi0;
      D.rhs = H->rhs0;
      D.fused = want_fused && fused_eligible(*D.phi, *D.rhs);
      if (p.smoother == MG_SMOOTH_FUSED && want_fused && !D.fused)
        fail(MG_EINVAL, "fused smoother needs phi nghost >= 2 and rhs nghost >= 1");
    } else {
      D.phi = internal_fab(c, D.bao, want_fused ? 2 : 1, H->dt);
      D.rhs = internal_fab(c, D.bao, want_fused ? 1 : 0, H->dt);
      D.fused = want_fused;
    }
    if (D.fused) D.phi2 = internal_fab(c, D.bao, D.phi->lay.g, H->dt);
  }
  if (H->mixed) H->r0 = internal_fab(c, phi.ba, 0, DT_F64);
  build_tables(c, *H, s);
  {
    // speculative red half-sweep with the norm check (see Hierarchy::save0): FP64, the
    // finest level smoothed by half-sweeps of its own (not inside the coarse-cycle kernel)
    // that read neighbours directly, pre- and post-smoothing present, even periodic extents
    // (an odd one maps a cell onto its own colour)
    int per[3];
    bc_code(bc, per);
    bool ok = !H->mixed && H->lc > 0 && p.nu1 >= 1 && p.nu2 >= 1 && !H->L[0].fused &&
              H->L[0].direct && H->direct0;
    for (int d = 0; d < 3; ++d)
      if (per[d] && (lev[0].dom.len(d) & 1)) ok = false;
    LevelData& D = H->L[0];
    const BoxArray& ba = D.bao->ba;
    // one-colour arrays over the level-0 boxes: (nx + 1) / 2 elements a row, rows dense
    std::vector<long long> off(ba.boxes.size() + 1, 0);
    for (size_t b = 0; b < ba.boxes.size(); ++b) {
      const Box& B = ba.boxes[b];
      off[b + 1] = off[b] + (long long)((B.len(0) + 1) / 2) * B.len(1) * B.len(2);
    }
    auto half_view = [&](const DevBufP& buf, int b) {
      const Box& B = ba.boxes[b];
      DView v{};
      v.pitch = (B.len(0) + 1) / 2;
      v.plane = (long long)v.pitch * B.len(1);
      v.cstride = v.plane * B.len(2);
      v.p = (double*)buf->p + off[b];
      return v;
    };
    if (ok) {
      H->save0 = c.alloc((size_t)off.back() * 8, s);
      FaceReads fr = direct_neighbours(*D.phi, per);
      D.smooth.d->reset(s);
      D.smooth = make_table(c, ba, 0, D.h, 0, [&](int b, DRow& R) {
        R.v[0] = D.phi->view(b);
        R.v[1] = D.rhs->view(b);
        R.v[2] = half_view(H->save0, b);
        fr.apply(b, R);
      }, s);
      D.smooth.direct = true;
    }
    // the last pre-smoothing half-sweep stores the black cells' residuals for the residual +
    // restriction, when level 0 is restricted by a stage kernel (not the bottom solve's level)
    if (ok && std::min(H->lc, nl - 1) >= 1) {
      H->res0 = c.alloc((size_t)off.back() * 8, s);
      FaceReads fr = direct_neighbours(*D.phi, per);
      const LevelData& C = H->L[1];
      H->store0 = make_table(c, ba, 0, D.h, 0, [&](int b, DRow& R) {
        R.v[0] = D.phi->view(b);
        R.v[1] = D.rhs->view(b);
        R.v[2] = half_view(H->res0, b);
        fr.apply(b, R);
      }, s);
      H->store0.direct = true;
      D.rr.d->reset(s);
      D.rr = make_table(c, ba, 1, D.h, 0, [&](int b, DRow& R) {
        R.v[0] = D.phi->view(b);
        R.v[1] = D.rhs->view(b);
        R.v[2] = half_view(H->res0, b);
        R.c[0] = coarse_view_of(*C.rhs, ba.boxes[b]);
        R.c[1] = coarse_view_of(*C.phi, ba.boxes[b]);
        fr.apply(b, R);
      }, s);
      D.rr.direct = true;
      H->stored0 = true;
    }
  }
  H->dnorm = c.alloc(16, s);
  MG_CK(cudaStreamSynchronize(s));
  c.hier.push_back(std::move(H));
  return *c.hier.back();
}

namespace {

// last_norm != null: the final (black) half-sweep also accumulates the residual max-norm of
// the cells it updates there (the caller adds the red cells).  store_last: the final (black)
// half-sweep also stores the residuals of the cells it updates (level 0: H.store0), for the
// residual + restriction that follows.
void smooth(Ctx& c, Hierarchy& H, LevelData& D, int sweeps, cudaStream_t s,
            unsigned long long* last_norm = nullptr, bool time_first = false,
            bool skip_first_red = false, bool store_last = false) {
  int k = 0;
  if (D.fused) {
    // pairs of fused sweeps: phi -> phi2 -> phi
    for (; k + 1 < sweeps; k += 2) {
      launch_fill(c, *D.phi, &H.bc, s, 2);  // the fused sweep reads two layers
      launch_fused(c, D.f_ab, H.dt, s);
      launch_fill(c, *D.phi2, &H.bc, s, 2);
      launch_fused(c, D.f_ba, H.dt, s);
    }
  }
  for (; k < sweeps; ++k)
    for (int color = 0; color < 2; ++color) {
      if (skip_first_red && k == 0 && color == 0) continue;  // done by the previous step
      if (!D.direct) launch_fill(c, *D.phi, &H.bc, s, 1);  // the half-sweep reads one layer
      const bool last = k + 1 == sweeps && color == 1;
      const bool timed = time_first && k == 0 && color == 1;
      // (external records: captured into the step graph as event-record nodes)
      if (timed) MG_CK(cudaEventRecordWithFlags(H.sweep_ev[0], s, cudaEventRecordExternal));
      if (last && store_last)
        MG_CK(launch_rbgs_half_store(H.store0.rows(), H.store0.nbox, H.store0.nrows, color, s,
                                     H.store0.width));
      else
        MG_CK(launch_rbgs_half(H.dt, D.smooth.rows(), D.smooth.nbox, D.smooth.nrows, color, s,
                               D.direct, last ? last_norm : nullptr, D.smooth.width));
      if (timed) MG_CK(cudaEventRecordWithFlags(H.sweep_ev[1], s, cudaEventRecordExternal));
    }
}

void enqueue_vcycle(Ctx& c, Hierarchy& H, cudaStream_t s, unsigned long long* norm0 = nullptr,
                    bool skip_first_red = false) {
  const int nl = (int)H.L.size();
  const int top = H.lc < nl ? H.lc : nl - 1;  // levels below `top` run stage by stage
  for (int l = 0; l < top; ++l) {
    LevelData& D = H.L[l];
    if (D.fused) launch_fill(c, *D.rhs, &H.bc, s, 1);  // rhs ghosts for the redundant ring
    // the finest level with res0 (FP64, direct reads, half-sweeps): the black children's
    // residuals come from the last pre-smoothing half-sweep
    const bool stored = l == 0 && H.stored0;
    smooth(c, H, D, H.p.nu1, s, nullptr, l == 0 && H.graph_timed, l == 0 && skip_first_red,
           stored);
    if (!D.direct) launch_fill(c, *D.phi, &H.bc, s, 1);
    MG_CK(launch_residual_restrict(H.dt, D.rr.rows(), D.rr.nbox, D.rr.nrows, s, D.direct,
                                   D.rr.width, stored));
  }
  if (H.lc < nl) MG_CK(launch_coarse_cycle(H.dt, (const CoarseJob*)H.cjob->p, 1, H.csmem, s));
  else MG_CK(launch_bottom(H.dt, (const BottomJob*)H.job->p, 1, H.N, s));
  for (int l = top - 1; l >= 0; --l) {
    LevelData& D = H.L[l];
    if (H.p.prolong == MG_PROLONG_TRILINEAR) {
      launch_fill(c, *H.L[l + 1].phi, &H.bc, s, 1);  // the coarse neighbours it reads
      MG_CK(launch_prolong_trilinear(H.dt, D.prolong.rows(), D.prolong.nbox, D.prolong.nrows, s,
                                     D.prolong.width));
    } else {
      MG_CK(launch_prolong_add(H.dt, D.prolong.rows(), D.prolong.nbox, D.prolong.nrows, s,
                               D.prolong.width));
    }
    smooth(c, H, D, H.p.nu2, s, l == 0 ? norm0 : nullptr);
  }
}

// One outer iteration: the cycle (with the mixed-precision scale / correction around it),
// then the norm check of the new iterate.  variant 1 / 2 (speculating solves): the cycle
// (variant 2: without its first finest-level red half-sweep, which the previous step ran),
// whose last black half-sweep takes the black cells' residual norm, then the next cycle's
// first red half-sweep, which takes the red cells' residual norm of the same iterate and
// saves the red values it replaces.
void enqueue_step(Ctx& c, Hierarchy& H, cudaStream_t s, int variant) {
  unsigned long long* dn = (unsigned long long*)H.dnorm->p;
  if (variant > 0) {
    LevelData& D0 = H.L[0];
    MG_CK(cudaMemsetAsync(dn, 0, 8, s));
    enqueue_vcycle(c, H, s, dn, variant == 2);
    MG_CK(launch_rbgs_half(DT_F64, D0.smooth.rows(), D0.smooth.nbox, D0.smooth.nrows, 0, s, true,
                           dn, D0.smooth.width, true));
    MG_CK(cudaMemcpyAsync(H.hnorm, dn, 16, cudaMemcpyDeviceToHost, s));
    return;
  }
  if (H.mixed)  // the FP32 right-hand side from the residual of the last norm check; e = 0
    MG_CK(launch_scale_residual_f32(H.scale0.rows(), H.scale0.nbox, H.scale0.nrows, dn, s,
                                    H.scale0.width));
  // FP64 with half-sweeps on the finest level: the cycle's last (black) half-sweep there
  // takes the residual norm of the cells it updates, and only the red cells need a residual
  // pass; the values are those of a full residual pass
  bool split_norm = !H.mixed && H.lc > 0 && H.p.nu2 >= 1 && !H.L[0].fused && H.direct0 &&
                    H.L[0].direct;
  {
    int per[3];
    bc_code(&H.bc, per);
    for (int d = 0; d < 3; ++d)  // an odd periodic extent maps a ghost onto its own colour
      if (per[d] && (H.L[0].bao->ba.dom.len(d) & 1)) split_norm = false;
  }
  if (split_norm) MG_CK(cudaMemsetAsync(dn, 0, 8, s));
  enqueue_vcycle(c, H, s, split_norm ? dn : nullptr);
  if (H.mixed)  // the further FP32 cycles of the outer iteration, from the correction so far
    for (int k = 1; k < H.p.inner; ++k) enqueue_vcycle(c, H, s, nullptr);
  if (H.mixed)
    MG_CK(launch_correct_add(H.correct0.rows(), H.correct0.nbox, H.correct0.nrows, dn, s,
                             H.correct0.width));
  if (!split_norm) MG_CK(cudaMemsetAsync(dn, 0, 8, s));
  if (!H.direct0) launch_fill(c, *H.phi0, &H.bc, s, 1);
  MG_CK(launch_residual(DT_F64, H.resid0.rows(), H.resid0.nbox, H.resid0.nrows, dn, s, H.direct0,
                        split_norm ? 0 : -1));
  MG_CK(cudaMemcpyAsync(H.hnorm, dn, 16, cudaMemcpyDeviceToHost, s));
}

void drop_graphs(Hierarchy& H) {
  for (cudaGraphExec_t& g : H.step_graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

void run_step(Ctx& c, Hierarchy& H, cudaStream_t s, int variant) {
  bool graph = H.p.use_graph && s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
  if (c.sweep_timing && !H.sweep_ev[0])
    for (cudaEvent_t& e : H.sweep_ev) MG_CK(cudaEventCreate(&e));
  if (H.graph_timed != c.sweep_timing) drop_graphs(H);  // timing switched: capture again
  H.graph_timed = c.sweep_timing;
  if (graph && H.graph_stream != s) drop_graphs(H);
  cudaGraphExec_t& G = H.step_graph[variant];
  if (graph && !G) {
    cudaGraph_t g = nullptr;
    const long long before = launches_so_far();
    MG_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    try {
      enqueue_step(c, H, s, variant);
    } catch (...) {
      cudaStreamEndCapture(s, &g);
      if (g) cudaGraphDestroy(g);
      count_launches(before - launches_so_far());
      throw;
    }
    MG_CK(cudaStreamEndCapture(s, &g));
    H.graph_kernels[variant] = launches_so_far() - before;  // captured, not executed
    count_launches(-H.graph_kernels[variant]);
    cudaError_t e = cudaGraphInstantiate(&G, g, 0);
    cudaGraphDestroy(g);
    MG_CK(e);
    H.graph_stream = s;
  }
  if (graph) {
    MG_CK(cudaGraphLaunch(G, s));
    count_launches(H.graph_kernels[variant]);
  } else {
    enqueue_step(c, H, s, variant);
  }
}

double bits_to_double(unsigned long long b) {
  double d;
  std::memcpy(&d, &b, 8);
  return d;
}

}  // namespace

void enqueue_correction_cycle(Ctx& c, Hierarchy& H, cudaStream_t s) {
  MG_CK(cudaMemsetAsync(H.phi0->base, 0, H.phi0->bytes, s));
  enqueue_vcycle(c, H, s);
}

void drop_hierarchies_of(Ctx& c, int64_t fab_id) {
  std::lock_guard<std::recursive_mutex> lk(c.hier_mu);
  bool any = false;
  for (auto& h : c.hier)
    if (h->rhs_id == fab_id || h->phi_id == fab_id) any = true;
  if (!any) return;
  cudaStreamSynchronize(c.stream);
  std::vector<std::shared_ptr<Hierarchy>> keep;
  for (auto& h : c.hier)
    if (h->rhs_id != fab_id && h->phi_id != fab_id) keep.push_back(std::move(h));
  c.hier.swap(keep);
}

void destroy_hierarchies(Ctx& c) {
  std::lock_guard<std::recursive_mutex> lk(c.hier_mu);
  c.hier.clear();
}

int solve(Ctx& c, int64_t rhs_id, int64_t phi_id, const mg_bc* bc, double tol,
          const SolveParams& p, mg_result* res) {
  c.require_device();
  if (!(tol >= 0)) fail(MG_EINVAL, "tol must be >= 0");
  auto rhs = c.get_fab(rhs_id);
  auto phi = c.get_fab(phi_id);
  double t_start = c.now();
  Hierarchy& H = get_hierarchy(c, *rhs, *phi, bc, p);
  cudaStream_t s = c.stream;
  if (!H.hnorm) MG_CK(cudaMallocHost(&H.hnorm, 16));
  unsigned long long* dn = (unsigned long long*)H.dnorm->p;
  // ||rhs||_inf and the first residual norm
  MG_CK(cudaMemsetAsync(dn, 0, 16, s));
  MG_CK(launch_maxabs(DT_F64, H.rhsabs0.rows(), H.rhsabs0.nbox, H.rhsabs0.nrows, dn, s));
  if (!H.direct0) launch_fill(c, *H.phi0, bc, s, 1);
  MG_CK(launch_residual(DT_F64, H.resid0.rows(), H.resid0.nbox, H.resid0.nrows, dn, s, H.direct0));
  MG_CK(cudaMemcpyAsync(H.hnorm, dn, 16, cudaMemcpyDeviceToHost, s));
  MG_CK(cudaStreamSynchronize(s));
  const double rhsnorm = bits_to_double(H.hnorm[1]);
  mg_result r{};
  r.t_start = t_start;
  int status = MG_OK;
  int it = 0;
  double rn = bits_to_double(H.hnorm[0]);
  if (std::isnan(rhsnorm) || std::isinf(rhsnorm)) {
    status = MG_ENAN;
  } else if (rhsnorm == 0.0) {
    MG_CK(launch_set_valid(DT_F64, H.zero0_64.rows(), H.zero0_64.nbox, H.zero0_64.nrows, 0.0, s));
    MG_CK(cudaStreamSynchronize(s));
    rn = 0.0;
  } else {
    bool pending = false;  // the next cycle's first red half-sweep has run (speculatively)
    for (;;) {
      bool stop = false;
      if (std::isnan(rn) || std::isinf(rn)) { status = MG_ENAN; stop = true; }
      else if (p.fixed_vcycles >= 0) {
        stop = it == p.fixed_vcycles;
      } else {
        if (rn <= tol * rhsnorm) stop = true;
        else if (it == p.max_iter) { status = MG_NOT_CONVERGED; stop = true; }
      }
      if (stop) {
        if (pending) {  // undo the speculative red half-sweep
          const OpTable& t = H.L[0].smooth;
          MG_CK(launch_restore_colour(DT_F64, t.rows(), t.nbox, t.nrows, 0, s));
          MG_CK(cudaStreamSynchronize(s));
        }
        break;
      }
      run_step(c, H, s, H.save0 ? (pending ? 2 : 1) : 0);
      MG_CK(cudaStreamSynchronize(s));
      pending = (bool)H.save0;
      rn = bits_to_double(H.hnorm[0]);
      if (H.graph_timed && H.lc > 0 && !H.L[0].fused) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, H.sweep_ev[0], H.sweep_ev[1]) == cudaSuccess) {
          c.sweep_ms += ms;
          c.sweep_n += 1;
        }
      }
      ++it;
    }
  }
  check_device_error(c);
  r.status = status;
  r.vcycles = it;
  r.rel_resid = rhsnorm > 0 ? rn / rhsnorm : 0.0;
  r.t_end = c.now();
  r.seconds = r.t_end - t_start;
  if (res) *res = r;
  return status;
}

}  // namespace gbmg

using namespace gbmg;

extern "C" {

int mg_sweep_timing(mg_ctx_t h, int enable, double* total_ms, int64_t* launches) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    if (total_ms) *total_ms = c->sweep_ms;
    if (launches) *launches = c->sweep_n;
    c->sweep_ms = 0.0;
    c->sweep_n = 0;
    c->sweep_timing = enable != 0;
    return MG_OK;
  });
}

int mg_solve(mg_ctx_t h, mg_fab_t rhs, mg_fab_t phi, const mg_bc* bc, double tol,
             const mg_options* opt, mg_result* res) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    auto f = c->get_fab(phi);
    SolveParams p = params_from(opt, f->ba->ba);
    return solve(*c, rhs, phi, bc, tol, p, res);
  });
}

int mg_solve_batch(mg_ctx_t h, int n, const mg_fab_t* rhs, const mg_fab_t* phi, const mg_bc* bcs,
                   double tol, const mg_options* opt, mg_result* res) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c || n <= 0 || !rhs || !phi || !bcs) fail(MG_EINVAL, "bad argument");
    auto f = c->get_fab(phi[0]);
    SolveParams p = params_from(opt, f->ba->ba);
    if (!(opt && opt->h > 0)) p.h = 0.0;  // resolved per solve from its own domain
    return solve_batch(*c, n, rhs, phi, bcs, tol, p, res);
  });
}

int mg_submit(mg_ctx_t h, mg_fab_t rhs, mg_fab_t phi, const mg_bc* bc, double tol,
              const mg_options* opt, mg_ticket_t* out) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c || !out) fail(MG_EINVAL, "bad argument");
    auto f = c->get_fab(phi);
    SolveParams p = params_from(opt, f->ba->ba);
    return server_submit(*c, rhs, phi, bc, tol, p, out);
  });
}

int mg_submit_host(mg_ctx_t h, const int dom_lo[3], const int dom_hi[3], const int max_box[3],
                   const mg_bc* bc, const double* rhs, double* phi, int phi_is_guess, double tol,
                   const mg_options* opt, mg_ticket_t* out) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c || !dom_lo || !dom_hi || !max_box || !out) fail(MG_EINVAL, "NULL argument");
    auto b = std::make_shared<BoxArrayObj>();
    Box dom;
    for (int d = 0; d < 3; ++d) {
      dom.lo[d] = dom_lo[d];
      dom.hi[d] = dom_hi[d];
    }
    std::string err;
    if (!chop(dom, max_box, &b->ba, &err)) fail(MG_EINVAL, err);
    SolveParams p = params_from(opt, b->ba);
    return server_submit_host(*c, std::move(b), rhs, phi, phi_is_guess, bc, tol, p, out);
  });
}

int mg_server_trim(mg_ctx_t h) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    server_trim(*c);
    return MG_OK;
  });
}

int mg_server_stats_get(mg_ctx_t h, mg_server_stats* out) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c || !out) fail(MG_EINVAL, "NULL argument");
    server_stats(*c, out);
    return MG_OK;
  });
}

int mg_poll(mg_ctx_t h, mg_ticket_t ticket, int timeout_ms, mg_result* res) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    return server_poll(*c, ticket, timeout_ms, res);
  });
}

}  // extern "C"
