// Batched and served solves.
//
// Many independent solves advance together: each stage of the V-cycle is ONE launch whose row
// space is the concatenation of the participating solves' cached box tables (segment lists,
// the multi-solve analogue of the fused launch over all boxes of Sec. 3.2).  A solve's
// arithmetic does not depend on its company, so each result is bit-identical to the same
// solve run alone.  Solves converge and retire independently.
//
// Serving (mg_submit / mg_poll) runs the same step on a scheduler thread with continuous
// batching: requests are admitted while the pool can hold their coarse levels and a slot is
// free, their V-cycles share launches with the solves already running, and each solve's
// hierarchy is released in stream order when it retires (Sec. 3.7 async-safe arena).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "mg_runtime.hpp"
#include "mg_solver.hpp"

namespace gbmg {

namespace {

double secs_since(std::chrono::steady_clock::time_point t) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t).count();
}

double bits2d(unsigned long long b) {
  double d;
  std::memcpy(&d, &b, 8);
  return d;
}

// One solve inside a batched step.
struct Member {
  std::shared_ptr<Hierarchy> H;
  int slot = 0;            // norms[slot]: residual norm, norms[slot + 1]: rhs norm
  double tol = 1e-10;
  double rhsnorm = 0, rn = 0;
  int vcycles = 0;
  int status = MG_OK;
  bool started = false;    // first norm check taken
  bool done = false;
  bool zero_rhs = false;
  mg_result res{};
  int64_t ticket = 0;
  double t_submit = -1.0;  // served solves: submission time
  // host-memory requests: the workspace (box array, fine-level fabs, hierarchy) the
  // scheduler lent this solve, and where its answer goes
  int64_t own_ba = 0, own_rhs = 0, own_phi = 0;
  std::string ws_key;
  double* phi_host = nullptr;
  cudaEvent_t copied = nullptr;  // host-memory requests: the copy in (or out) has finished
  ~Member() {
    if (copied) cudaEventDestroy(copied);
  }
};

// Segment-list builders (host side); offsets into the step's packed upload.
struct SegB {
  std::vector<Seg> v;
  long long total = 0;
  size_t off = 0;
  bool direct = false;  // some member's rows carry box-face reads
  int width = 0;
  void add(const OpTable& t, int slot) {
    if (!t.nrows) return;
    direct = direct || t.direct;
    width = std::max(width, t.width);
    Seg s{};
    s.rows = t.rows();
    s.row_begin = total;
    s.row_count = t.nrows;
    s.nbox = t.nbox;
    s.slot = slot;
    v.push_back(s);
    total += t.nrows;
  }
};
struct TagB {
  std::vector<TagSeg> v;
  long long total = 0;
  size_t off = 0;
  void add(const FillPlan& P, void* base) {
    if (!P.nchunks()) return;
    TagSeg s{};
    s.tags = P.tags();
    s.chunks = P.chunks();
    s.base = base;
    s.chunk_begin = total;
    s.nchunks = P.nchunks();
    v.push_back(s);
    total += P.nchunks();
  }
};
struct UnitB {
  std::vector<UnitSeg> v;
  long long total = 0;
  size_t off = 0;
  int ty = 1, depth = 4, mp = 0, mpr = 0;
  bool rhs_smem = true;
  void add(const FusedTable& t) {
    UnitSeg s{};
    s.rows = t.rows.rows();
    s.units = (const int4*)t.units->p;
    s.unit_begin = total;
    s.nunits = t.nunits;
    v.push_back(s);
    total += t.nunits;
    ty = std::max(ty, t.ty);
    depth = std::min(depth, t.depth);
    mp = std::max(mp, t.max_pitch);
    mpr = std::max(mpr, t.max_pitch_r);
    rhs_smem = rhs_smem && t.rhs_smem;
  }
};
struct JobB {
  std::vector<BottomJob> v;
  int maxN = 0;
  size_t off = 0;
  void add(const Hierarchy& H) {
    v.push_back(H.job_host);
    maxN = std::max(maxN, H.N);
  }
};

struct CoarseB {
  std::vector<CoarseJob> v;
  size_t smem = 0;
  size_t off = 0;
  void add(const Hierarchy& H) {
    v.push_back(H.cjob_host);
    smem = std::max(smem, H.csmem);
  }
};

struct LevelLists {
  SegB half, half_all, rr, prolong;
  SegB prolong3;  // trilinear prolongation (members solving with that form)
  TagB fill1_half, fill1_all, fill2_phi, fill2_phi2, fill_rhs;
  TagB fill_c;    // the coarse level's phi, one layer, before the trilinear prolongation
  UnitB fab, fba;
  JobB bottom_next;      // bottoms at level l + 1
  CoarseB coarse_next;   // coarse cycles from level l + 1
};

struct StepLists {
  std::vector<LevelLists> L;
  JobB bottom0;
  CoarseB coarse0;
  SegB resid0, rhsabs0, scale0, correct0;
  TagB fill_phi0;
  int dt = DT_F64;
  bool mixed = false;
  int nu1 = 2, nu2 = 2, inner = 1;  // (the members of one step share them)
};

struct Staging {
  std::vector<unsigned char> host;
  DevBufP dev;
  template <class T>
  size_t push(const std::vector<T>& v) {
    size_t off = (host.size() + 15) / 16 * 16;
    host.resize(off + v.size() * sizeof(T));
    if (!v.empty()) std::memcpy(host.data() + off, v.data(), v.size() * sizeof(T));
    return off;
  }
};

SegList mk(const SegB& b, const unsigned char* dev) {
  SegList L{};
  L.n = (int)b.v.size();
  L.width = b.width;
  if (L.n == 1) L.one = b.v[0];
  else L.segs = (const Seg*)(dev + b.off);
  return L;
}
TagList mk(const TagB& b, const unsigned char* dev) {
  TagList L{};
  L.n = (int)b.v.size();
  if (L.n == 1) L.one = b.v[0];
  else L.segs = (const TagSeg*)(dev + b.off);
  return L;
}
UnitList mk(const UnitB& b, const unsigned char* dev) {
  UnitList L{};
  L.n = (int)b.v.size();
  if (L.n == 1) L.one = b.v[0];
  else L.segs = (const UnitSeg*)(dev + b.off);
  return L;
}

// Lists for one step.  `run`: members doing a V-cycle this step; `check`: members whose norm
// is taken at the end of the step (run plus newly admitted ones); `fresh`: members whose
// rhs norm is still unknown.
void build_lists(Ctx& c, StepLists& S, const std::vector<Member*>& run,
                 const std::vector<Member*>& check, const std::vector<Member*>& fresh) {
  size_t Lmax = 0;
  for (Member* m : run) Lmax = std::max(Lmax, m->H->L.size());
  S.L.assign(Lmax > 0 ? Lmax : 1, LevelLists{});
  for (Member* m : run) {
    Hierarchy& H = *m->H;
    S.dt = H.dt;
    S.mixed = H.mixed;
    S.nu1 = H.p.nu1;
    S.nu2 = H.p.nu2;
    S.inner = H.mixed ? H.p.inner : 1;
    const int nl = (int)H.L.size();
    if (nl == 1) S.bottom0.add(H);
    if (H.lc == 0 && nl > 1) S.coarse0.add(H);
    for (int l = 0; l + 1 < nl && l < H.lc; ++l) {
      LevelData& D = H.L[l];
      LevelLists& LL = S.L[l];
      if (D.fused) {
        LL.fab.add(D.f_ab);
        LL.fba.add(D.f_ba);
        LL.fill2_phi.add(fill_plan(c, *D.phi, &H.bc, 2), D.phi->base);
        LL.fill2_phi2.add(fill_plan(c, *D.phi2, &H.bc, 2), D.phi2->base);
        LL.fill_rhs.add(fill_plan(c, *D.rhs, &H.bc, 1), D.rhs->base);
      } else {
        LL.half.add(D.smooth, m->slot);
        if (!D.direct) LL.fill1_half.add(fill_plan(c, *D.phi, &H.bc, 1), D.phi->base);
      }
      if (!D.direct) LL.fill1_all.add(fill_plan(c, *D.phi, &H.bc, 1), D.phi->base);
      LL.half_all.add(D.smooth, m->slot);
      LL.rr.add(D.rr, m->slot);
      if (H.p.prolong == MG_PROLONG_TRILINEAR) {
        LL.prolong3.add(D.prolong, m->slot);
        FabObj& cphi = *H.L[l + 1].phi;
        LL.fill_c.add(fill_plan(c, cphi, &H.bc, 1), cphi.base);
      } else {
        LL.prolong.add(D.prolong, m->slot);
      }
      if (l + 1 == H.lc) LL.coarse_next.add(H);
      else if (l + 2 == nl) LL.bottom_next.add(H);
    }
    if (H.mixed) {
      S.scale0.add(H.scale0, m->slot);
      S.correct0.add(H.correct0, m->slot);
    }
  }
  for (Member* m : check) {
    S.resid0.add(m->H->resid0, m->slot);
    if (!m->H->direct0) S.fill_phi0.add(fill_plan(c, *m->H->phi0, &m->H->bc, 1), m->H->phi0->base);
  }
  for (Member* m : fresh) S.rhsabs0.add(m->H->rhsabs0, m->slot);
}

void upload_lists(Ctx& c, StepLists& S, Staging& st, cudaStream_t s) {
  st.host.clear();
  auto seg = [&](SegB& b) { b.off = st.push(b.v); };
  auto tag = [&](TagB& b) { b.off = st.push(b.v); };
  auto unit = [&](UnitB& b) { b.off = st.push(b.v); };
  auto job = [&](JobB& b) { b.off = st.push(b.v); };
  auto cjob = [&](CoarseB& b) { b.off = st.push(b.v); };
  for (LevelLists& LL : S.L) {
    seg(LL.half); seg(LL.half_all); seg(LL.rr); seg(LL.prolong); seg(LL.prolong3);
    tag(LL.fill1_half); tag(LL.fill1_all); tag(LL.fill2_phi); tag(LL.fill2_phi2); tag(LL.fill_rhs);
    tag(LL.fill_c);
    unit(LL.fab); unit(LL.fba);
    job(LL.bottom_next);
    cjob(LL.coarse_next);
  }
  job(S.bottom0);
  cjob(S.coarse0);
  seg(S.resid0); seg(S.rhsabs0); seg(S.scale0); seg(S.correct0);
  tag(S.fill_phi0);
  size_t need = std::max<size_t>(st.host.size(), 256);
  if (!st.dev || st.dev->bytes < need) {
    MG_CK(cudaStreamSynchronize(s));
    if (st.dev) st.dev->reset(s);
    st.dev = c.alloc(need * 2, s);
  }
  MG_CK(cudaMemcpyAsync(st.dev->p, st.host.data(), st.host.size(), cudaMemcpyHostToDevice, s));
}

void fill_l(Ctx& c, int dt, const TagB& b, const unsigned char* dev, cudaStream_t s) {
  (void)c;
  if (b.total) MG_CK(launch_copy_tags_l(dt, mk(b, dev), b.total, 1, s));
}

void smooth_l(Ctx& c, StepLists& S, LevelLists& LL, int sweeps, const unsigned char* dev,
              int* err, cudaStream_t s) {
  int k = 0;
  for (; k + 1 < sweeps; k += 2) {
    if (LL.fab.total) {
      fill_l(c, S.dt, LL.fill2_phi, dev, s);
      MG_CK(launch_rbgs_fused_l(S.dt, mk(LL.fab, dev), LL.fab.total, LL.fab.ty, LL.fab.depth,
                                LL.fab.mp, LL.fab.mpr, LL.fab.rhs_smem, err, s));
      fill_l(c, S.dt, LL.fill2_phi2, dev, s);
      MG_CK(launch_rbgs_fused_l(S.dt, mk(LL.fba, dev), LL.fba.total, LL.fba.ty, LL.fba.depth,
                                LL.fba.mp, LL.fba.mpr, LL.fba.rhs_smem, err, s));
    }
    if (LL.half.total)
      for (int j = 0; j < 2; ++j)
        for (int color = 0; color < 2; ++color) {
          fill_l(c, S.dt, LL.fill1_half, dev, s);
          MG_CK(launch_rbgs_half_l(S.dt, mk(LL.half, dev), LL.half.total, color, s, LL.half.direct));
        }
  }
  for (; k < sweeps; ++k)
    for (int color = 0; color < 2; ++color) {
      // an odd sweep: every member with half-sweeps (fused members too, in place)
      fill_l(c, S.dt, LL.fill1_all, dev, s);
      MG_CK(launch_rbgs_half_l(S.dt, mk(LL.half_all, dev), LL.half_all.total, color, s,
                               LL.half_all.direct));
    }
}

// The step: V-cycle for the `run` members, then the norm check of the `check` members.
void enqueue_step(Ctx& c, StepLists& S, const unsigned char* dev, unsigned long long* norms,
                  size_t norm_bytes, bool any_fresh, cudaStream_t s) {
  int* err = (int*)c.d_err->p;
  const int nlev = (int)S.L.size();
  if (S.mixed && S.scale0.total) {
    MG_CK(launch_scale_residual_f32_l(mk(S.scale0, dev), S.scale0.total, norms, s));
  }
  // the V-cycle (mixed form: S.inner FP32 cycles, the later ones from the correction so far)
  for (int rep = 0; rep < S.inner; ++rep) {
    if (!S.bottom0.v.empty())
      MG_CK(launch_bottom(S.dt, (const BottomJob*)(dev + S.bottom0.off), (int)S.bottom0.v.size(),
                          S.bottom0.maxN, s));
    if (!S.coarse0.v.empty())
      MG_CK(launch_coarse_cycle(S.dt, (const CoarseJob*)(dev + S.coarse0.off),
                                (int)S.coarse0.v.size(), S.coarse0.smem, s));
    for (int l = 0; l < nlev; ++l) {
      LevelLists& LL = S.L[l];
      if (!LL.rr.total) continue;
      if (LL.fill_rhs.total) fill_l(c, S.dt, LL.fill_rhs, dev, s);
      smooth_l(c, S, LL, S.nu1, dev, err, s);
      fill_l(c, S.dt, LL.fill1_all, dev, s);
      MG_CK(launch_residual_restrict_l(S.dt, mk(LL.rr, dev), LL.rr.total, s, LL.rr.direct));
      if (!LL.bottom_next.v.empty())
        MG_CK(launch_bottom(S.dt, (const BottomJob*)(dev + LL.bottom_next.off),
                            (int)LL.bottom_next.v.size(), LL.bottom_next.maxN, s));
      if (!LL.coarse_next.v.empty())
        MG_CK(launch_coarse_cycle(S.dt, (const CoarseJob*)(dev + LL.coarse_next.off),
                                  (int)LL.coarse_next.v.size(), LL.coarse_next.smem, s));
    }
    for (int l = nlev - 1; l >= 0; --l) {
      LevelLists& LL = S.L[l];
      if (!LL.prolong.total && !LL.prolong3.total) continue;
      if (LL.prolong.total) MG_CK(launch_prolong_add_l(S.dt, mk(LL.prolong, dev), LL.prolong.total, s));
      if (LL.prolong3.total) {
        fill_l(c, S.dt, LL.fill_c, dev, s);
        MG_CK(launch_prolong_trilinear_l(S.dt, mk(LL.prolong3, dev), LL.prolong3.total, s));
      }
      smooth_l(c, S, LL, S.nu2, dev, err, s);
    }
  }
  if (S.mixed && S.correct0.total)
    MG_CK(launch_correct_add_l(mk(S.correct0, dev), S.correct0.total, norms, s));
  // norm check
  MG_CK(cudaMemsetAsync(norms, 0, norm_bytes, s));
  if (any_fresh && S.rhsabs0.total)
    MG_CK(launch_maxabs_l(DT_F64, mk(S.rhsabs0, dev), S.rhsabs0.total, norms, s));
  fill_l(c, DT_F64, S.fill_phi0, dev, s);
  if (S.resid0.total) MG_CK(launch_residual_l(DT_F64, mk(S.resid0, dev), S.resid0.total, norms, s, S.resid0.direct));
}

// Applies the stop rule of a single solve to a member after its norm check.
void decide(Ctx& c, Member& m, cudaStream_t s) {
  const SolveParams& p = m.H->p;
  if (std::isnan(m.rhsnorm) || std::isinf(m.rhsnorm)) { m.status = MG_ENAN; m.done = true; return; }
  if (m.rhsnorm == 0.0) {
    const OpTable& z = m.H->zero0_64;
    MG_CK(launch_set_valid(DT_F64, z.rows(), z.nbox, z.nrows, 0.0, s));
    m.rn = 0.0;
    m.done = true;
    return;
  }
  if (std::isnan(m.rn) || std::isinf(m.rn)) { m.status = MG_ENAN; m.done = true; return; }
  if (p.fixed_vcycles >= 0) {
    if (m.vcycles == p.fixed_vcycles) m.done = true;
    return;
  }
  if (m.rn <= m.tol * m.rhsnorm) { m.done = true; return; }
  if (m.vcycles == p.max_iter) { m.status = MG_NOT_CONVERGED; m.done = true; }
  (void)c;
}

void finish(Ctx& c, Member& m) {
  m.res.status = m.status;
  m.res.vcycles = m.vcycles;
  m.res.rel_resid = m.rhsnorm > 0 ? m.rn / m.rhsnorm : 0.0;
  m.res.t_end = c.now();
  m.res.seconds = m.res.t_end - m.res.t_start;
}

// Runs one step for `run` (V-cycle) and `check` (norm check) members of one precision, reads
// the norms back and applies the stop rule.
struct StepTimes {
  double plan = 0, step = 0;
  long long steps = 0;
};

void step_and_decide(Ctx& c, Staging& st, NormBuf& nb, std::vector<Member*>& run,
                     std::vector<Member*>& check, int nslots, cudaStream_t s,
                     StepTimes* tm = nullptr) {
  auto t0 = std::chrono::steady_clock::now();
  std::vector<Member*> fresh;
  for (Member* m : check)
    if (!m->started) fresh.push_back(m);
  StepLists S;
  build_lists(c, S, run, check, fresh);
  if (!check.empty()) {
    S.dt = check[0]->H->dt;
    S.mixed = check[0]->H->mixed;
  }
  upload_lists(c, S, st, s);
  auto t1 = std::chrono::steady_clock::now();
  unsigned long long* norms = (unsigned long long*)nb.d->p;
  const size_t nbytes = (size_t)nslots * 8;
  enqueue_step(c, S, (const unsigned char*)st.dev->p, norms, nbytes, !fresh.empty(), s);
  MG_CK(cudaMemcpyAsync(nb.h, norms, nbytes, cudaMemcpyDeviceToHost, s));
  MG_CK(cudaStreamSynchronize(s));
  if (tm) {
    tm->plan += std::chrono::duration<double>(t1 - t0).count();
    tm->step += secs_since(t1);
    tm->steps += 1;
  }
  check_device_error(c);
  for (Member* m : run) m->vcycles += 1;
  for (Member* m : check) {
    if (!m->started) {
      m->rhsnorm = bits2d(nb.h[m->slot + 1]);
      m->started = true;
    }
    m->rn = bits2d(nb.h[m->slot]);
    decide(c, *m, s);
  }
  MG_CK(cudaStreamSynchronize(s));  // a zero-rhs member's phi reset completes before it retires
}

}  // namespace

int solve_batch(Ctx& c, int n, const int64_t* rhs, const int64_t* phi, const mg_bc* bcs, double tol,
                const SolveParams& p, mg_result* res) {
  c.require_device();
  if (!(tol >= 0)) fail(MG_EINVAL, "tol must be >= 0");
  cudaStream_t s = c.stream;
  std::vector<Member> M(n);
  const double t0 = c.now();
  for (int i = 0; i < n; ++i) {
    auto fr = c.get_fab(rhs[i]);
    auto fp = c.get_fab(phi[i]);
    for (int j = 0; j < i; ++j)
      if (phi[j] == phi[i]) fail(MG_EINVAL, "a phi fab appears twice in the batch");
    SolveParams pi = p;  // the default cell size belongs to each solve's own domain
    if (!(pi.h > 0)) pi.h = 1.0 / fp->ba->ba.dom.len(0);
    std::lock_guard<std::recursive_mutex> hl(c.hier_mu);
    Hierarchy& H = get_hierarchy(c, *fr, *fp, &bcs[i], pi);
    for (auto& h : c.hier)
      if (h.get() == &H) M[i].H = h;
    if (!M[i].H) fail(MG_EINVAL, "internal: hierarchy not found");
    M[i].slot = 2 * i;
    M[i].tol = tol;
    M[i].res.t_start = t0;
  }
  NormBuf& nb = c.batch_norms;
  nb.ensure(c, 2 * n, s);
  Staging st;
  std::vector<Member*> run, check;
  for (auto& m : M) check.push_back(&m);
  step_and_decide(c, st, nb, run, check, 2 * n, s);
  for (;;) {
    run.clear();
    for (auto& m : M)
      if (!m.done) run.push_back(&m);
    if (run.empty()) break;
    check = run;
    step_and_decide(c, st, nb, run, check, 2 * n, s);
  }
  int rc = MG_OK;
  for (int i = 0; i < n; ++i) {
    finish(c, M[i]);
    if (res) res[i] = M[i].res;
    if (M[i].status != MG_OK && rc == MG_OK) rc = M[i].status;
  }
  if (st.dev) st.dev->reset(s);
  MG_CK(cudaStreamSynchronize(s));
  return rc;
}

// ---- serving ---------------------------------------------------------------------------

struct Ctx::Server {
  struct Req {
    int64_t ticket, rhs, phi;
    mg_bc bc;
    double tol;
    SolveParams p;
    double t_submit;
    // host-memory requests (mg_submit_host): rhs == phi == 0, the box array chopped at
    // submission, the fabs allocated from the pool at admission
    std::shared_ptr<BoxArrayObj> hba;
    std::string ws_key;  // requests with equal keys can share a workspace, one at a time
    const double* rhs_host = nullptr;
    double* phi_host = nullptr;
    int phi_is_guess = 0;
  };
  // Workspaces of retired host-memory requests, kept for the next request of the same shape
  // (box array, faces, options) -- its hierarchy stays resident, so admitting it costs two
  // copies and no planning.  Oldest first; released, oldest first, when the pool needs room,
  // and all at once by mg_server_trim.
  struct Workspace {
    std::string key;
    int64_t ba = 0, rhs = 0, phi = 0;
  };
  std::deque<Workspace> idle;
  bool trim = false;  // mg_server_trim waiting
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req> queue;
  std::map<int64_t, mg_result> done;
  std::map<int64_t, bool> known;
  int64_t next_ticket = 1;
  bool stop = false;
  std::thread th;
  size_t max_queue = 1 << 20;
  int max_active = 4096;
  mg_server_stats stats{};
  // norm slots per step group -- members of one precision, smoothing counts and inner
  // cycles, which share their steps (separate arrays: each group's check clears its whole
  // array, and a mixed member's next step reads its last norm)
  std::map<std::array<int, 4>, NormBuf> norms;
};



namespace {

// Releases, in stream order, a host-memory workspace: its hierarchy, fabs and box array.
void release_ws(Ctx& c, int64_t ba, int64_t rhs, int64_t phi, cudaStream_t s) {
  if (rhs || phi) {
    std::lock_guard<std::recursive_mutex> hl(c.hier_mu);
    std::vector<std::shared_ptr<Hierarchy>> rest;
    for (auto& h : c.hier)
      if (!(h->rhs_id == rhs && h->phi_id == phi)) rest.push_back(h);
    c.hier.swap(rest);
  }
  if (phi) release_fab(c, phi, s);
  if (rhs) release_fab(c, rhs, s);
  if (ba) {
    std::lock_guard<std::mutex> lk(c.mu);
    c.bas.erase(ba);
  }
}
void release_own(Ctx& c, Member& m, cudaStream_t s) {
  release_ws(c, m.own_ba, m.own_rhs, m.own_phi, s);
  m.own_ba = m.own_rhs = m.own_phi = 0;
}
// Releases the oldest idle workspace; false if there is none.
bool evict_idle(Ctx& c, Ctx::Server& S, cudaStream_t s) {
  if (S.idle.empty()) return false;
  const auto w = S.idle.front();
  S.idle.pop_front();
  release_ws(c, w.ba, w.rhs, w.phi, s);
  return true;
}
// Takes the most recently idle workspace with this key into m; false if there is none.
bool take_idle(Ctx::Server& S, const std::string& key, Member& m) {
  for (size_t i = S.idle.size(); i-- > 0;)
    if (S.idle[i].key == key) {
      m.own_ba = S.idle[i].ba;
      m.own_rhs = S.idle[i].rhs;
      m.own_phi = S.idle[i].phi;
      m.ws_key = key;
      S.idle.erase(S.idle.begin() + (long)i);
      return true;
    }
  return false;
}

// Publishes a finished member's result.
void publish(Ctx::Server& S, Member& m) {
  // counted with the publication, so a caller that has polled every ticket sees them all
  std::lock_guard<std::mutex> lk(S.mu);
  S.done[m.ticket] = m.res;
  S.stats.completed += 1;
  S.cv_done.notify_all();
}

void server_loop(Ctx* c) {
  Ctx::Server& S = *c->server;
  cudaSetDevice(c->device);
  cudaStream_t s = c->stream;
  // Host-memory requests copy in and out on their own stream, so that the copies of some
  // requests overlap the shared steps of the others: a request joins the steps once its copy
  // in has finished, and completes once its copy out has.
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) cs = s;
  Staging st;
  std::vector<std::unique_ptr<Member>> active, loading, unloading;
  std::vector<int> free_slots;
  int nslots = 0;
  for (;;) {
    std::vector<Ctx::Server::Req> admit;
    {
      std::unique_lock<std::mutex> lk(S.mu);
      auto ready = [&] { return S.stop || S.trim || !S.queue.empty(); };
      if (active.empty()) {
        if (loading.empty() && unloading.empty()) S.cv_work.wait(lk, ready);
        else S.cv_work.wait_for(lk, std::chrono::microseconds(100), ready);
      }
      if (S.trim) {
        while (evict_idle(*c, S, s)) {
        }
        cudaStreamSynchronize(s);
        S.trim = false;
        S.cv_done.notify_all();
      }
      if (S.stop && S.queue.empty() && active.empty() && loading.empty() && unloading.empty())
        break;
      // admission: while a slot is free (pool room is checked when the hierarchy is built)
      while (!S.queue.empty() &&
             (int)(active.size() + loading.size() + admit.size()) < S.max_active) {
        admit.push_back(S.queue.front());
        S.queue.pop_front();
      }
    }
    std::vector<Member*> fresh_members;
    auto t_admit0 = std::chrono::steady_clock::now();
    for (size_t k = 0; k < admit.size(); ++k) {
      const auto& r = admit[k];
      std::unique_ptr<Member> m(new Member);
      m->ticket = r.ticket;
      m->tol = r.tol;
      m->t_submit = r.t_submit;
      m->res.t_admit = c->now();
      m->res.t_start = r.t_submit;
      try {
        int64_t rid = r.rhs, pid = r.phi;
        if (r.hba) {
          // the request's fine level comes from the pool too: rhs (1 ghost layer) and phi
          // (2, so that the fused smoother may run on it), filled from host memory -- in an
          // idle workspace of the same shape if there is one, else in a new one (made room
          // for by releasing idle workspaces of other shapes, oldest first)
          m->phi_host = r.phi_host;
          if (!take_idle(S, r.ws_key, *m)) {
            for (;;) {
              try {
                m->ws_key = r.ws_key;
                m->own_ba = c->add_ba(r.hba);
                m->own_rhs = add_pool_fab(*c, r.hba, m->own_ba, 1, 1, DT_F64, s);
                m->own_phi = add_pool_fab(*c, r.hba, m->own_ba, 1, 2, DT_F64, s);
                auto fr = c->get_fab(m->own_rhs);
                auto fp = c->get_fab(m->own_phi);
                std::lock_guard<std::recursive_mutex> hl(c->hier_mu);
                get_hierarchy(*c, *fr, *fp, &r.bc, r.p);
                break;
              } catch (const MgError& e) {
                release_own(*c, *m, s);
                if (e.code != MG_ENOMEM || !evict_idle(*c, S, s)) throw;
              }
            }
          }
          rid = m->own_rhs;
          pid = m->own_phi;
          dense_upload(*c, *c->get_fab(rid), r.rhs_host, cs);
          auto fp = c->get_fab(pid);
          if (r.phi_is_guess) dense_upload(*c, *fp, r.phi_host, cs);
          else MG_CK(cudaMemsetAsync(fp->base, 0, fp->bytes, cs));
          MG_CK(cudaEventCreateWithFlags(&m->copied, cudaEventDisableTiming));
          MG_CK(cudaEventRecord(m->copied, cs));
        }
        auto fr = c->get_fab(rid);
        auto fp = c->get_fab(pid);
        std::lock_guard<std::recursive_mutex> hl(c->hier_mu);
        Hierarchy& H = get_hierarchy(*c, *fr, *fp, &r.bc, r.p);
        for (auto& h : c->hier)
          if (h.get() == &H) m->H = h;
      } catch (const MgError& e) {
        cudaStreamSynchronize(cs);  // a copy in may have started
        release_own(*c, *m, s);
        if (e.code == MG_ENOMEM && !active.empty()) {
          // no room: back to the head of the queue until a running solve retires
          std::lock_guard<std::mutex> lk(S.mu);
          for (size_t j = admit.size(); j-- > k;) S.queue.push_front(admit[j]);
          break;
        }
        m->status = e.code;
        m->done = true;
        finish(*c, *m);
        publish(S, *m);
        continue;
      }
      if (m->copied) loading.push_back(std::move(m));  // joins once its data is in
      else {
        if (free_slots.empty()) {
          free_slots.push_back(nslots);
          nslots += 2;
        }
        m->slot = free_slots.back();
        free_slots.pop_back();
        fresh_members.push_back(m.get());
        active.push_back(std::move(m));
      }
    }
    // members whose copy in has finished join this step
    {
      std::vector<std::unique_ptr<Member>> still;
      for (auto& m : loading) {
        const cudaError_t q = cudaEventQuery(m->copied);
        if (q == cudaErrorNotReady) {
          still.push_back(std::move(m));
          continue;
        }
        if (q != cudaSuccess) {
          cudaGetLastError();
          cudaStreamSynchronize(cs);
          m->status = MG_ECUDA;
          m->done = true;
          finish(*c, *m);
          release_own(*c, *m, s);
          publish(S, *m);
          continue;
        }
        if (free_slots.empty()) {
          free_slots.push_back(nslots);
          nslots += 2;
        }
        m->slot = free_slots.back();
        free_slots.pop_back();
        fresh_members.push_back(m.get());
        active.push_back(std::move(m));
      }
      loading.swap(still);
    }
    {
      std::lock_guard<std::mutex> lk(S.mu);
      S.stats.admitted += (int64_t)fresh_members.size();
      S.stats.admit_seconds += secs_since(t_admit0);
      S.stats.max_active = std::max<int64_t>(S.stats.max_active, (int64_t)active.size());
    }
    try {
      // one step per group (precision, smoothing counts, inner cycles): running members
      // cycle, every member's norm is checked
      auto key_of = [](const Member& m) {
        const SolveParams& p = m.H->p;
        return std::array<int, 4>{m.H->dt, p.nu1, p.nu2, m.H->mixed ? p.inner : 1};
      };
      std::vector<std::array<int, 4>> keys;
      for (auto& m : active)
        if (!m->done && std::find(keys.begin(), keys.end(), key_of(*m)) == keys.end())
          keys.push_back(key_of(*m));
      for (const auto& key : keys) {
        NormBuf& nb = S.norms[key];
        std::vector<Member*> run, check;
        for (auto& m : active) {
          if (m->done || key_of(*m) != key) continue;
          check.push_back(m.get());
          if (m->started) run.push_back(m.get());
        }
        if (!check.empty()) {
          StepTimes tm;
          nb.ensure(*c, nslots, s);
          step_and_decide(*c, st, nb, run, check, nslots, s, &tm);
          std::lock_guard<std::mutex> lk(S.mu);
          S.stats.plan_seconds += tm.plan;
          S.stats.step_seconds += tm.step;
          S.stats.steps += tm.steps;
        }
      }
    } catch (const MgError& e) {
      for (auto& m : active) {
        m->status = e.code;
        m->done = true;
      }
    }
    // retire
    auto t_ret0 = std::chrono::steady_clock::now();
    std::vector<std::unique_ptr<Member>> keep, leaving;
    for (auto& m : active) {
      if (!m->done) {
        keep.push_back(std::move(m));
        continue;
      }
      finish(*c, *m);
      free_slots.push_back(m->slot);
      const int64_t rid = m->H ? m->H->rhs_id : 0, pid = m->H ? m->H->phi_id : 0;
      m->H.reset();
      // release the solve's hierarchy (coarse levels, tables) in stream order; a
      // host-memory request's workspace is kept whole for the next request of its shape
      if (!m->own_phi) {
        std::lock_guard<std::recursive_mutex> hl(c->hier_mu);
        std::vector<std::shared_ptr<Hierarchy>> rest;
        for (auto& h : c->hier)
          if (!(h->rhs_id == rid && h->phi_id == pid)) rest.push_back(h);
        c->hier.swap(rest);
      }
      leaving.push_back(std::move(m));
    }
    active.swap(keep);
    // host-memory requests: the answer goes back to the caller's array (on the copy stream,
    // after the steps that produced it) before completion; the others complete now
    if (!leaving.empty() && cs != s) {
      cudaEvent_t stepped;
      MG_CK(cudaEventCreateWithFlags(&stepped, cudaEventDisableTiming));
      MG_CK(cudaEventRecord(stepped, s));
      MG_CK(cudaStreamWaitEvent(cs, stepped, 0));
      cudaEventDestroy(stepped);
    }
    for (auto& m : leaving) {
      if (!m->own_phi) {
        publish(S, *m);
        continue;
      }
      try {
        if (m->phi_host) dense_download(*c, *c->get_fab(m->own_phi), m->phi_host, cs);
        if (!m->copied) MG_CK(cudaEventCreateWithFlags(&m->copied, cudaEventDisableTiming));
        MG_CK(cudaEventRecord(m->copied, cs));
        unloading.push_back(std::move(m));
      } catch (const MgError& e) {
        if (m->res.status == MG_OK) m->res.status = e.code;
        cudaStreamSynchronize(cs);
        release_own(*c, *m, s);
        publish(S, *m);
      }
    }
    // copies out that have finished: the request completes, its workspace turns idle
    {
      std::vector<std::unique_ptr<Member>> still;
      for (auto& m : unloading) {
        const cudaError_t q = cudaEventQuery(m->copied);
        if (q == cudaErrorNotReady) {
          still.push_back(std::move(m));
          continue;
        }
        if (q != cudaSuccess) {
          cudaGetLastError();
          if (m->res.status == MG_OK) m->res.status = MG_ECUDA;
        }
        m->res.t_end = c->now();
        m->res.seconds = m->res.t_end - m->res.t_start;
        if (m->res.status == MG_OK || m->res.status == MG_NOT_CONVERGED) {
          S.idle.push_back({m->ws_key, m->own_ba, m->own_rhs, m->own_phi});
          m->own_ba = m->own_rhs = m->own_phi = 0;
        } else {
          release_own(*c, *m, s);
        }
        publish(S, *m);
      }
      unloading.swap(still);
    }
    {
      std::lock_guard<std::mutex> lk(S.mu);
      S.stats.retire_seconds += secs_since(t_ret0);
    }
  }
  cudaStreamSynchronize(cs);
  while (evict_idle(*c, S, s)) {
  }
  if (st.dev) st.dev->reset(s);
  for (auto& kv : S.norms) kv.second.release(s);
  cudaStreamSynchronize(s);
  if (cs != s) cudaStreamDestroy(cs);
}

}  // namespace

int server_submit(Ctx& c, int64_t rhs, int64_t phi, const mg_bc* bc, double tol,
                  const SolveParams& p, int64_t* ticket) {
  c.require_device();
  if (!(tol >= 0)) fail(MG_EINVAL, "tol must be >= 0");
  int per[3];
  bc_code(bc, per);
  c.get_fab(rhs);
  c.get_fab(phi);
  if (!c.server) {
    c.server = std::make_shared<Ctx::Server>();
    c.server->th = std::thread(server_loop, &c);
  }
  Ctx::Server& S = *c.server;
  std::lock_guard<std::mutex> lk(S.mu);
  if (S.queue.size() >= S.max_queue) fail(MG_EAGAIN, "serving queue full");
  Ctx::Server::Req r{S.next_ticket++, rhs, phi, *bc, tol, p, c.now()};
  S.stats.submitted += 1;
  S.known[r.ticket] = true;
  S.queue.push_back(r);
  *ticket = r.ticket;
  S.cv_work.notify_one();
  return MG_OK;
}

int server_submit_host(Ctx& c, std::shared_ptr<BoxArrayObj> ba, const double* rhs, double* phi,
                       int phi_is_guess, const mg_bc* bc, double tol, const SolveParams& p,
                       int64_t* ticket) {
  c.require_device();
  if (!(tol >= 0)) fail(MG_EINVAL, "tol must be >= 0");
  if (!rhs || !phi) fail(MG_EINVAL, "NULL host array");
  int per[3];
  bc_code(bc, per);
  ba->hierarchy();  // MG_EINVAL now rather than at admission
  if (!c.server) {
    c.server = std::make_shared<Ctx::Server>();
    c.server->th = std::thread(server_loop, &c);
  }
  Ctx::Server& S = *c.server;
  std::lock_guard<std::mutex> lk(S.mu);
  if (S.queue.size() >= S.max_queue) fail(MG_EAGAIN, "serving queue full");
  Ctx::Server::Req r{S.next_ticket++, 0, 0, *bc, tol, p, c.now()};
  {
    // workspace key: the boxes, the faces and every option the hierarchy depends on
    std::string& k = r.ws_key;
    auto put = [&](const void* d, size_t n) { k.append((const char*)d, n); };
    put(&ba->ba.dom, sizeof(Box));
    for (const Box& b : ba->ba.boxes) put(&b, sizeof(Box));
    put(bc, sizeof(mg_bc));
    const int ip[8] = {p.nu1, p.nu2, p.precision, p.smoother, p.coarse_cells, p.direct_reads,
                       p.prolong, p.inner};
    put(ip, sizeof ip);
    put(&p.h, sizeof p.h);
  }
  r.hba = std::move(ba);
  r.rhs_host = rhs;
  r.phi_host = phi;
  r.phi_is_guess = phi_is_guess ? 1 : 0;
  S.stats.submitted += 1;
  S.known[r.ticket] = true;
  S.queue.push_back(r);
  *ticket = r.ticket;
  S.cv_work.notify_one();
  return MG_OK;
}

int server_poll(Ctx& c, int64_t ticket, int timeout_ms, mg_result* res) {
  if (!c.server) fail(MG_EINVAL, "unknown ticket");
  Ctx::Server& S = *c.server;
  std::unique_lock<std::mutex> lk(S.mu);
  if (!S.known.count(ticket)) fail(MG_EINVAL, "unknown ticket");
  auto ready = [&] { return S.done.count(ticket) > 0; };
  if (timeout_ms < 0) S.cv_done.wait(lk, ready);
  else if (timeout_ms > 0) S.cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
  if (!ready()) return MG_PENDING;
  if (res) *res = S.done[ticket];
  S.done.erase(ticket);
  S.known.erase(ticket);
  return MG_OK;
}

void server_stats(Ctx& c, mg_server_stats* out) {
  if (!c.server) {
    *out = mg_server_stats{};
    return;
  }
  std::lock_guard<std::mutex> lk(c.server->mu);
  *out = c.server->stats;
}

void server_trim(Ctx& c) {
  if (!c.server) return;
  Ctx::Server& S = *c.server;
  std::unique_lock<std::mutex> lk(S.mu);
  S.trim = true;
  S.cv_work.notify_all();
  S.cv_done.wait(lk, [&] { return !S.trim; });
}

void server_stop(Ctx& c) {
  if (!c.server) return;
  {
    std::lock_guard<std::mutex> lk(c.server->mu);
    c.server->stop = true;
    c.server->cv_work.notify_all();
  }
  if (c.server->th.joinable()) c.server->th.join();
  c.server.reset();
}

}  // namespace gbmg
