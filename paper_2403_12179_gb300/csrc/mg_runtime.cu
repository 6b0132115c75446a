// Context, memory pool, box arrays, fabs, ghost-fill plans and the level-operation entry
// points of the C ABI.
//
// Memory: one CUDA stream-ordered pool per context (Sec. 3.7: pre-allocated arena; the
// async-safe arena frees in stream order).  Fabs store all boxes of a level in one
// allocation (Sec. 2 FArrayBox / MultiFab) and expose per-box views (Sec. 4.1 zero-copy).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <cstdlib>
#include <sstream>

#include <cmath>

#include "mg_runtime.hpp"

namespace gbmg {

static thread_local std::string g_err;

void fail(int code, const std::string& msg) { throw MgError{code, msg}; }

void set_last_error(const std::string& msg) { g_err = msg; }

void check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();  // clear a non-sticky error
    throw MgError{MG_ECUDA, m};
  }
}

DevBuf::~DevBuf() {
  if (p && ctx) {
    cudaFreeAsync(p, ctx->stream);
    ctx->in_use -= bytes;
  }
}

void DevBuf::reset(cudaStream_t s) {
  if (p && ctx) {
    cudaFreeAsync(p, s);
    ctx->in_use -= bytes;
  }
  p = nullptr;
  bytes = 0;
}

DevBufP Ctx::alloc(size_t n, cudaStream_t s) {
  require_device();
  if (n == 0) n = 16;
  n = (n + 255) / 256 * 256;
  size_t cur = in_use.load();
  if (cur + n > pool_cap) {
    std::ostringstream o;
    o << "memory pool exhausted: " << n << " bytes requested, " << cur << " of " << pool_cap
      << " in use";
    fail(MG_ENOMEM, o.str());
  }
  void* p = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&p, n, pool, s);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    fail(MG_ENOMEM, "device out of memory");
  }
  MG_CK(e);
  in_use += n;
  DevBufP b(new DevBuf);
  b->ctx = this;
  b->p = p;
  b->bytes = n;
  return b;
}

DevBufP Ctx::upload(const void* host, size_t n, cudaStream_t s) {
  DevBufP b = alloc(n, s);
  if (n) MG_CK(cudaMemcpyAsync(b->p, host, n, cudaMemcpyHostToDevice, s));
  return b;
}

std::shared_ptr<BoxArrayObj> Ctx::get_ba(int64_t id) {
  std::lock_guard<std::mutex> lk(mu);
  auto it = bas.find(id);
  if (it == bas.end()) fail(MG_EINVAL, "unknown box array handle");
  return it->second;
}

std::shared_ptr<FabObj> Ctx::get_fab(int64_t id) {
  std::lock_guard<std::mutex> lk(mu);
  auto it = fabs.find(id);
  if (it == fabs.end()) fail(MG_EINVAL, "unknown fab handle");
  return it->second;
}

int64_t Ctx::add_ba(std::shared_ptr<BoxArrayObj> b) {
  std::lock_guard<std::mutex> lk(mu);
  int64_t id = next_id++;
  bas[id] = std::move(b);
  return id;
}

void NormBuf::ensure(Ctx& c, int n, cudaStream_t s) {
  if (n <= slots) return;
  const int m = std::max(std::max(n, 64), 2 * slots);
  DevBufP nd = c.alloc((size_t)m * 8, s);
  MG_CK(cudaMemsetAsync(nd->p, 0, (size_t)m * 8, s));
  if (d) MG_CK(cudaMemcpyAsync(nd->p, d->p, (size_t)slots * 8, cudaMemcpyDeviceToDevice, s));
  unsigned long long* nh = nullptr;
  MG_CK(cudaMallocHost(&nh, (size_t)m * 8));
  MG_CK(cudaStreamSynchronize(s));
  d = std::move(nd);
  if (h) cudaFreeHost(h);
  h = nh;
  slots = m;
}

void NormBuf::release(cudaStream_t s) {
  if (d) {
    cudaStreamSynchronize(s);
    d.reset();
  }
  if (h) cudaFreeHost(h);
  h = nullptr;
  slots = 0;
}

void Ctx::load_tune_file() {
  if (tune_loaded) return;
  tune_loaded = true;
  const char* path = std::getenv("GBMG_TUNE_FILE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[400], key[200];
  while (std::fgets(line, sizeof line, f)) {
    FusedCfg cfg;
    if (std::sscanf(line, "%199s %d %d %d %d", key, &cfg.ty, &cfg.zc, &cfg.depth, &cfg.rhs_smem) == 5 &&
        cfg.ty > 0 && cfg.zc > 0 && cfg.depth >= 1 && cfg.depth <= 4)
      tune[key] = cfg;
  }
  std::fclose(f);
}

void Ctx::save_tune_entry(const std::string& key, const FusedCfg& cfg) {
  const char* path = std::getenv("GBMG_TUNE_FILE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d %d %d %d\n", key.c_str(), cfg.ty, cfg.zc, cfg.depth, cfg.rhs_smem);
  std::fclose(f);
}

const std::vector<BoxArray>& BoxArrayObj::hierarchy() {
  if (!levels_built) {
    levels_ok = build_levels(ba, &levels, &levels_err);
    levels_built = true;
  }
  if (!levels_ok) fail(MG_EINVAL, levels_err);
  return levels;
}

int bc_code(const mg_bc* bc, int periodic[3]) {
  if (!bc) fail(MG_EINVAL, "bc is NULL");
  int code = 0;
  for (int d = 0; d < 3; ++d) {
    int a = bc->kind[d][0], b = bc->kind[d][1];
    bool ok = (a == MG_BC_PERIODIC || a == MG_BC_DIRICHLET0) &&
              (b == MG_BC_PERIODIC || b == MG_BC_DIRICHLET0);
    if (!ok) fail(MG_EINVAL, "unknown boundary kind");
    if ((a == MG_BC_PERIODIC) != (b == MG_BC_PERIODIC))
      fail(MG_EINVAL, "a periodic dimension must be periodic on both faces");
    periodic[d] = a == MG_BC_PERIODIC ? 1 : 0;
    code |= (periodic[d] ? 0 : 1) << d;
  }
  return code;
}

DView FabObj::view(int b) const {
  DView v;
  int g = lay.g;
  long long o = lay.off[b] + g * lay.plane[b] + (long long)g * lay.pitch[b] + g;
  v.p = (char*)base + o * esize();
  v.plane = lay.plane[b];
  v.cstride = lay.cstride[b];
  v.pitch = lay.pitch[b];
  v.g = g;
  return v;
}

std::vector<DTag> device_tags(const BoxArray& ba, const FabLayout& lay,
                              const std::vector<CopyTag>& tags, int base_index) {
  std::vector<DTag> out;
  out.reserve(tags.size());
  for (const CopyTag& t : tags) {
    DTag d{};
    int db = t.dst_box;
    d.dst = lay.at(ba, db, t.dst_lo[0], t.dst_lo[1], t.dst_lo[2]);
    d.dsy = lay.pitch[db];
    d.dsz = (int)lay.plane[db];
    d.dcs = lay.cstride[db];
    if (t.sign != 0) {
      int sb = t.src_box;
      d.src = lay.at(ba, sb, t.src_first[0], t.src_first[1], t.src_first[2]);
      d.ssx = t.dir[0];
      d.ssy = t.dir[1] * lay.pitch[sb];
      d.ssz = t.dir[2] * (int)lay.plane[sb];
      d.scs = lay.cstride[sb];
    }
    d.ex = t.ext[0];
    d.ey = t.ext[1];
    d.ez = t.ext[2];
    d.sign = t.sign;
    (void)base_index;
    out.push_back(d);
  }
  return out;
}

FillPlan& fill_plan(Ctx& c, FabObj& f, const mg_bc* bc, int layers) {
  int per[3];
  const int ng = (layers < 0 || layers > f.lay.g) ? f.lay.g : layers;
  const int code = bc_code(bc, per);
  const int key = code + 8 * ng;
  auto it = f.fills.find(key);
  if (it != f.fills.end()) return *it->second;
  // the pattern depends on the box array, BCs, layers filled and the fab layout only
  const BoxArray& ba = f.ba->ba;
  std::string tkey;
  int hdr[6] = {code, ng, f.lay.g, f.lay.ncomp, f.esize(), (int)ba.boxes.size()};
  tkey.append((const char*)hdr, sizeof hdr);
  tkey.append((const char*)&ba.dom, sizeof(Box));
  tkey.append((const char*)ba.boxes.data(), ba.boxes.size() * sizeof(Box));
  std::shared_ptr<TagSet> set;
  {
    std::lock_guard<std::mutex> lk(c.tag_mu);
    auto ct = c.tag_cache.find(tkey);
    if (ct != c.tag_cache.end()) set = ct->second;
  }
  if (!set) {
    std::vector<CopyTag> tags;
    std::string err;
    if (!make_copy_tags(ba, per, ng, &tags, &err)) fail(MG_EINVAL, err);
    std::vector<DTag> dt = device_tags(ba, f.lay, tags, 0);
    std::vector<int2> chunks;
    std::vector<int> first;
    for (size_t t = 0; t < dt.size(); ++t) {
      first.push_back((int)chunks.size());
      const int rows = dt[t].ey * dt[t].ez, per = tag_chunk_rows(dt[t].ex, f.lay.ncomp, f.esize());
      for (int r0 = 0; r0 < rows; r0 += per) chunks.push_back(make_int2((int)t, r0));
    }
    first.push_back((int)chunks.size());
    set = std::make_shared<TagSet>();
    set->first_chunk = std::move(first);
    set->nchunks = (int)chunks.size();
    if (set->nchunks) {
      set->tags_buf = c.upload(dt.data(), dt.size() * sizeof(DTag), c.stream);
      set->chunks_buf = c.upload(chunks.data(), chunks.size() * sizeof(int2), c.stream);
    }
    // the pattern may be used on any stream from now on
    MG_CK(cudaStreamSynchronize(c.stream));
    std::lock_guard<std::mutex> lk(c.tag_mu);
    c.tag_cache[tkey] = set;
  }
  std::unique_ptr<FillPlan> P(new FillPlan);
  P->set = set;
  FillPlan& ref = *P;
  f.fills[key] = std::move(P);
  return ref;
}

void launch_fill(Ctx& c, FabObj& f, const mg_bc* bc, cudaStream_t s, int layers) {
  FillPlan& P = fill_plan(c, f, bc, layers);
  if (!P.nchunks()) return;
  MG_CK(launch_copy_tags(f.dtype, P.tags(), P.chunks(), P.nchunks(), f.base, f.lay.ncomp, s));
}

FaceReads direct_neighbours(const FabObj& f, const int periodic[3], bool outside_ghosts) {
  FaceReads out;
  const BoxArray& ba = f.ba->ba;
  const FabLayout& lay = f.lay;
  const size_t nb = ba.boxes.size();
  if (nb == 0 || lay.g < 1) return out;
  // an odd periodic extent makes a boundary cell's periodic neighbour a cell of its own
  // colour, which a half-sweep may be updating at the same time: read filled ghosts there
  for (int d = 0; d < 3; ++d)
    if (periodic[d] && (ba.dom.len(d) & 1)) return out;
  int E[3];
  for (int d = 0; d < 3; ++d) E[d] = ba.boxes[0].len(d);
  std::map<std::array<int, 3>, int> at_lo;
  for (size_t b = 0; b < nb; ++b) {
    const Box& B = ba.boxes[b];
    for (int d = 0; d < 3; ++d)
      if (B.len(d) != E[d] || (B.lo[d] - ba.dom.lo[d]) % E[d] != 0) return out;
    if (lay.pitch[b] != lay.pitch[0] || lay.plane[b] != lay.plane[0]) return out;
    at_lo[{B.lo[0], B.lo[1], B.lo[2]}] = (int)b;
  }
  std::vector<std::array<long long, 6>> dl(nb);
  std::vector<int> fl(nb, 0);
  for (size_t b = 0; b < nb; ++b) {
    const Box& B = ba.boxes[b];
    const long long stride[3] = {1, lay.pitch[b], lay.plane[b]};
    for (int d = 0; d < 3; ++d)
      for (int side = 0; side < 2; ++side) {
        const int face = 2 * d + side;
        int g[3] = {B.lo[0], B.lo[1], B.lo[2]};  // low corner of the first ghost layer
        g[d] = side ? B.hi[d] + 1 : B.lo[d] - 1;
        const long long ghost = lay.at(ba, (int)b, g[0], g[1], g[2]);
        const int L = ba.dom.len(d);
        if (g[d] < ba.dom.lo[d] || g[d] > ba.dom.hi[d]) {
          if (!periodic[d] && outside_ghosts) {  // the ghost cell itself
            dl[b][face] = 0;
            continue;
          }
          if (!periodic[d]) {  // -(the box's own boundary layer)
            dl[b][face] = side ? -stride[d] : stride[d];
            fl[b] |= 1 << face;
            continue;
          }
          g[d] += g[d] < ba.dom.lo[d] ? L : -L;
        }
        std::array<int, 3> lo;
        for (int k = 0; k < 3; ++k)
          lo[k] = ba.dom.lo[k] + (int)std::floor((double)(g[k] - ba.dom.lo[k]) / E[k]) * E[k];
        auto it = at_lo.find(lo);
        if (it == at_lo.end()) return FaceReads{};
        dl[b][face] = lay.at(ba, it->second, g[0], g[1], g[2]) - ghost;
      }
  }
  out.d = std::move(dl);
  out.flags = std::move(fl);
  return out;
}

OpTable upload_table(Ctx& c, const std::vector<DRow>& rows, long long nrows, cudaStream_t s) {
  OpTable t;
  t.nbox = (int)rows.size();
  t.nrows = nrows;
  for (const DRow& R : rows) t.width = std::max(t.width, R.n[0]);
  if (!rows.empty()) t.d = c.upload(rows.data(), rows.size() * sizeof(DRow), s);
  return t;
}

void ensure_valid_rows(Ctx& c, FabObj& f) {
  if (f.valid_rows) return;
  std::vector<DRow> rows;
  long long n = 0;
  append_rows(&rows, &n, f.ba->ba, 0, 1.0, 0, [&](int b, DRow& R) { R.v[0] = f.view(b); });
  f.valid_rows = c.upload(rows.data(), rows.size() * sizeof(DRow), c.stream);
  f.nrows = n;
  MG_CK(cudaStreamSynchronize(c.stream));
}

int64_t add_pool_fab(Ctx& c, std::shared_ptr<BoxArrayObj> ba, int64_t ba_id, int ncomp, int g,
                     int dt, cudaStream_t s) {
  auto f = std::make_shared<FabObj>();
  f->ba_id = ba_id;
  f->ba = std::move(ba);
  f->dtype = dt;
  f->lay = make_layout(f->ba->ba, ncomp, g, f->esize());
  f->bytes = (size_t)f->lay.total * f->esize();
  f->own = c.alloc(f->bytes, s);
  f->base = f->own->p;
  MG_CK(cudaMemsetAsync(f->base, 0, f->bytes, s));
  std::lock_guard<std::mutex> lk(c.mu);
  f->id = c.next_id++;
  c.fabs[f->id] = f;
  return f->id;
}

void release_fab(Ctx& c, int64_t id, cudaStream_t s) {
  std::shared_ptr<FabObj> f;
  {
    std::lock_guard<std::mutex> lk(c.mu);
    auto it = c.fabs.find(id);
    if (it == c.fabs.end()) return;
    f = it->second;
    c.fabs.erase(it);
  }
  if (f->valid_rows) f->valid_rows->reset(s);
  if (f->own) f->own->reset(s);
}

void dense_upload(Ctx& c, FabObj& f, const void* host, cudaStream_t s) {
  ensure_valid_rows(c, f);
  const Box& D = f.ba->ba.dom;
  int n[3] = {D.len(0), D.len(1), D.len(2)};
  const size_t bytes = (size_t)D.npts() * f.lay.ncomp * f.esize();
  DevBufP stage = c.alloc(bytes, s);
  MG_CK(cudaMemcpyAsync(stage->p, host, bytes, cudaMemcpyHostToDevice, s));
  MG_CK(launch_dense_copy(f.dtype, (const DRow*)f.valid_rows->p, (int)f.ba->ba.boxes.size(),
                          f.nrows, stage->p, D.lo, n, f.lay.ncomp, 0, s));
  stage->reset(s);
}

void dense_download(Ctx& c, FabObj& f, void* host, cudaStream_t s) {
  ensure_valid_rows(c, f);
  const Box& D = f.ba->ba.dom;
  int n[3] = {D.len(0), D.len(1), D.len(2)};
  const size_t bytes = (size_t)D.npts() * f.lay.ncomp * f.esize();
  DevBufP stage = c.alloc(bytes, s);
  MG_CK(launch_dense_copy(f.dtype, (const DRow*)f.valid_rows->p, (int)f.ba->ba.boxes.size(),
                          f.nrows, stage->p, D.lo, n, f.lay.ncomp, 1, s));
  MG_CK(cudaMemcpyAsync(host, stage->p, bytes, cudaMemcpyDeviceToHost, s));
  stage->reset(s);
}

const std::vector<double>& bottom_matrix_t(Ctx& c, const int n[3], const int periodic[3],
                                           double h) {
  std::lock_guard<std::mutex> lk(c.bottom_mu);
  char key[160];
  std::snprintf(key, sizeof key, "%d,%d,%d,%d,%d,%d,%.17g", n[0], n[1], n[2], periodic[0],
                periodic[1], periodic[2], h);
  auto it = c.bottom_cache.find(key);
  if (it != c.bottom_cache.end()) return it->second;
  std::vector<double> M;
  std::string err;
  if (!bottom_matrix(n, periodic, h, &M, &err)) fail(MG_EINVAL, err);
  long long N = (long long)n[0] * n[1] * n[2];
  std::vector<double> Mt((size_t)N * N);
  for (long long i = 0; i < N; ++i)
    for (long long j = 0; j < N; ++j) Mt[(size_t)j * N + i] = M[(size_t)i * N + j];
  return c.bottom_cache[key] = std::move(Mt);
}

void drop_cached_ops_of(Ctx& c, int64_t fab_id) {
  bool synced = false;
  for (auto it = c.fused_cache.begin(); it != c.fused_cache.end();) {
    bool uses = false;
    for (int64_t id : it->second->owner_fabs) uses |= id == fab_id;
    if (uses) {
      if (!synced) { cudaDeviceSynchronize(); synced = true; }
      it = c.fused_cache.erase(it);
    } else {
      ++it;
    }
  }
  for (auto it = c.op_cache.begin(); it != c.op_cache.end();) {
    bool uses = false;
    for (int64_t id : it->second.fabs) uses |= id == fab_id;
    if (uses) {
      if (!synced) { cudaDeviceSynchronize(); synced = true; }
      it = c.op_cache.erase(it);
    } else {
      ++it;
    }
  }
}

bool fused_eligible(const FabObj& phi, const FabObj& rhs) {
  return phi.lay.g >= 2 && rhs.lay.g >= 1 && phi.dtype == rhs.dtype && phi.lay.ncomp == 1;
}

// Table of the fused sweep for one configuration: tiles of cfg.ty rows x cfg.zc planes
// (chunk ends are recomputed by both neighbours), prefetch depth cfg.depth.
static FusedTable build_fused(Ctx& c, const BoxArray& ba, double h, const FabObj& src,
                              const FabObj& rhs, const FabObj& dst, const int periodic[3],
                              FusedCfg cfg, cudaStream_t s) {
  FusedTable t;
  int maxn1 = 1, maxn2 = 1;
  for (size_t b = 0; b < ba.boxes.size(); ++b) {
    t.max_pitch = std::max(t.max_pitch, src.lay.pitch[b]);
    t.max_pitch_r = std::max(t.max_pitch_r, rhs.lay.pitch[b]);
    maxn1 = std::max(maxn1, ba.boxes[b].len(1));
    maxn2 = std::max(maxn2, ba.boxes[b].len(2));
  }
  t.ty = std::max(1, std::min(cfg.ty, maxn1));
  t.zc = std::max(1, std::min(cfg.zc, maxn2));
  t.depth = cfg.depth;
  t.rhs_smem = cfg.rhs_smem != 0;
  if (fused_smem_bytes(src.dtype, t.ty, t.max_pitch, t.max_pitch_r, t.depth, t.rhs_smem) > 200 * 1024)
    return t;
  std::vector<DRow> rows;
  long long nr = 0;
  append_rows(&rows, &nr, ba, 0, h, 0, [&](int b, DRow& R) {
    R.v[0] = src.view(b);
    R.v[1] = rhs.view(b);
    R.v[2] = dst.view(b);
    int fl = 0;
    const Box& B = ba.boxes[b];
    for (int d = 0; d < 3; ++d) {
      if (!periodic[d] && B.lo[d] == ba.dom.lo[d]) fl |= 1 << d;
      if (!periodic[d] && B.hi[d] == ba.dom.hi[d]) fl |= 8 << d;
    }
    R.pad_ = fl;
  });
  std::vector<int4> units;  // {box, y0 | ty << 16, z0, z1}
  for (size_t b = 0; b < ba.boxes.size(); ++b)
    for (int z0 = 0; z0 < ba.boxes[b].len(2); z0 += t.zc)
      for (int y0 = 0; y0 < ba.boxes[b].len(1); y0 += t.ty)
        units.push_back(make_int4((int)b, y0 | (t.ty << 16), z0,
                                  std::min(z0 + t.zc, ba.boxes[b].len(2))));
  t.rows = upload_table(c, rows, nr, s);
  t.units = c.upload(units.data(), units.size() * sizeof(int4), s);
  t.nunits = (int)units.size();
  t.ok = true;
  return t;
}

// Autotuned fused table: the first time a (type, box shape, box count, pitches) is seen,
// every candidate (tile rows, z-chunk, prefetch depth) is timed on the live fabs -- each
// writes the same result into dst -- and the fastest is kept for that shape (and appended
// to the file named by GBMG_TUNE_FILE, if set, which later contexts read back).
FusedTable make_fused(Ctx& c, const BoxArray& ba, double h, const FabObj& src, const FabObj& rhs,
                      const FabObj& dst, const int periodic[3], cudaStream_t s) {
  FusedTable none;
  if (!fused_eligible(src, rhs) || dst.lay.g != src.lay.g || dst.dtype != src.dtype) return none;
  int mx[3] = {1, 1, 1}, mp = 0, mpr = 0;
  for (size_t b = 0; b < ba.boxes.size(); ++b) {
    for (int d = 0; d < 3; ++d) mx[d] = std::max(mx[d], ba.boxes[b].len(d));
    mp = std::max(mp, src.lay.pitch[b]);
    mpr = std::max(mpr, rhs.lay.pitch[b]);
  }
  char key[160];
  std::snprintf(key, sizeof key, "v2_dt%d_b%dx%dx%d_n%zu_p%d_%d_g%d_%d", src.dtype, mx[0], mx[1], mx[2],
                ba.boxes.size(), mp, mpr, src.lay.g, rhs.lay.g);
  {
    std::lock_guard<std::mutex> lk(c.tune_mu);
    c.load_tune_file();
    auto it = c.tune.find(key);
    if (it != c.tune.end()) return build_fused(c, ba, h, src, rhs, dst, periodic, it->second, s);
  }
  FusedCfg best{16, 16, 2};
  float best_ms = 1e30f;
  FusedTable best_t;
  cudaEvent_t e0, e1;
  MG_CK(cudaEventCreate(&e0));
  MG_CK(cudaEventCreate(&e1));
  for (int rs : {1, 0})
  for (int depth : {2, 3, 4})
    // tile rows: powers of two, and ty + 2 (the rows of a red pass with its ring) a
    // multiple of 8 or 16 (the rows the consumers cover in one pass for wide boxes)
    for (int ty : {4, 6, 8, 14, 16, 22, 30, 32}) {
      if (ty > 2 * mx[1] && ty != 4) continue;
      for (int zc : {8, 16, 32, 64}) {
        if (zc > 2 * mx[2] && zc != 8) continue;
        FusedTable t = build_fused(c, ba, h, src, rhs, dst, periodic, FusedCfg{ty, zc, depth, rs}, s);
        if (!t.ok) continue;
        launch_fused(c, t, src.dtype, s);  // warm
        MG_CK(cudaEventRecord(e0, s));
        for (int r = 0; r < 3; ++r) launch_fused(c, t, src.dtype, s);
        MG_CK(cudaEventRecord(e1, s));
        MG_CK(cudaEventSynchronize(e1));
        float ms = 0;
        MG_CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms) {
          best_ms = ms;
          best = FusedCfg{t.ty, t.zc, t.depth, t.rhs_smem ? 1 : 0};
          best_t = std::move(t);
        }
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  check_device_error(c);
  if (!best_t.ok) return none;
  {
    std::lock_guard<std::mutex> lk(c.tune_mu);
    c.tune[key] = best;
    c.save_tune_entry(key, best);
  }
  return best_t;
}

void launch_fused(Ctx& c, const FusedTable& t, int dt, cudaStream_t s) {
  MG_CK(launch_rbgs_fused(dt, t.rows.rows(), (const int4*)t.units->p, t.nunits, t.ty, t.depth,
                          t.max_pitch, t.max_pitch_r, t.rhs_smem, (int*)c.d_err->p, s));
}

const FusedTable& fused_table(Ctx& c, int64_t src_id, FabObj& src, int64_t rhs_id, FabObj& rhs,
                              int64_t dst_id, FabObj& dst, const mg_bc* bc, double h) {
  int per[3];
  int code = bc_code(bc, per);
  char key[200];
  std::snprintf(key, sizeof key, "%lld:%lld:%lld:%d:%.17g", (long long)src_id, (long long)rhs_id,
                (long long)dst_id, code, h);
  auto it = c.fused_cache.find(key);
  if (it != c.fused_cache.end()) return *it->second;
  auto t = std::make_shared<FusedTable>(make_fused(c, src.ba->ba, h, src, rhs, dst, per, c.stream));
  MG_CK(cudaStreamSynchronize(c.stream));
  t->owner_fabs = {src_id, rhs_id, dst_id < 0 ? -dst_id : dst_id};
  c.fused_cache[key] = t;
  return *t;
}

std::shared_ptr<FabObj> partner_of(Ctx& c, FabObj& f) {
  if (f.partner) return f.partner;
  auto p = std::make_shared<FabObj>();
  p->ba = f.ba;
  p->ba_id = f.ba_id;
  p->dtype = f.dtype;
  p->lay = f.lay;
  p->bytes = f.bytes;
  p->own = c.alloc(p->bytes, c.stream);
  p->base = p->own->p;
  MG_CK(cudaMemsetAsync(p->base, 0, p->bytes, c.stream));
  MG_CK(cudaStreamSynchronize(c.stream));
  f.partner = p;
  return p;
}

void check_device_error(Ctx& c) {
  int e = 0;
  MG_CK(cudaMemcpy(&e, c.d_err->p, sizeof e, cudaMemcpyDeviceToHost));
  if (e) {
    MG_CK(cudaMemset(c.d_err->p, 0, sizeof e));
    fail(MG_ETIMEDOUT, "a kernel's bounded wait for its shared-memory copies expired");
  }
}

SolveParams params_from(const mg_options* o, const BoxArray& ba) {
  SolveParams p;
  if (o) {
    p.nu1 = o->nu1;
    p.nu2 = o->nu2;
    p.max_iter = o->max_iter;
    p.precision = o->precision;
    p.smoother = o->smoother;
    p.use_graph = o->use_graph;
    p.fixed_vcycles = o->fixed_vcycles;
    p.h = o->h;
    p.coarse_cells = o->coarse_cells;
    p.direct_reads = o->direct_reads;
    p.prolong = o->prolong;
    p.inner = o->inner_cycles == 0 ? kDefaultInnerCycles : o->inner_cycles;
  }
  if (p.h <= 0.0) p.h = 1.0 / ba.dom.len(0);
  if (p.nu1 < 0 || p.nu2 < 0 || p.max_iter < 0 || p.nu1 + p.nu2 == 0)
    fail(MG_EINVAL, "invalid smoothing counts or max_iter");
  if (p.precision != MG_PREC_F64 && p.precision != MG_PREC_MIXED)
    fail(MG_EINVAL, "unknown precision mode");
  if (p.smoother < MG_SMOOTH_AUTO || p.smoother > MG_SMOOTH_FUSED)
    fail(MG_EINVAL, "unknown smoother");
  if (p.prolong != MG_PROLONG_CONSTANT && p.prolong != MG_PROLONG_TRILINEAR)
    fail(MG_EINVAL, "unknown prolongation");
  if (p.inner < 1 || p.inner > kMaxInnerCycles) fail(MG_EINVAL, "inner_cycles out of range");
  return p;
}

}  // namespace gbmg

using namespace gbmg;

namespace {

Box box_of(const int lo[3], const int hi[3]) {
  Box b;
  for (int d = 0; d < 3; ++d) { b.lo[d] = lo[d]; b.hi[d] = hi[d]; }
  return b;
}

cudaStream_t S(void* s) { return (cudaStream_t)s; }

void same_shape(const FabObj& a, const FabObj& b, const char* what) {
  if (a.ba->ba.boxes.size() != b.ba->ba.boxes.size() ||
      std::memcmp(a.ba->ba.boxes.data(), b.ba->ba.boxes.data(),
                  a.ba->ba.boxes.size() * sizeof(Box)) != 0 ||
      std::memcmp(&a.ba->ba.dom, &b.ba->ba.dom, sizeof(Box)) != 0)
    fail(MG_EINVAL, std::string(what) + ": fabs are on different box arrays");
  if (a.dtype != b.dtype) fail(MG_EINVAL, std::string(what) + ": fabs differ in type");
}

double default_h(const FabObj& f, double h) { return h > 0 ? h : 1.0 / f.ba->ba.dom.len(0); }

// The coarse fab must be on level 1 of the fine fab's hierarchy (domain halved, boxes the
// coarsened fine boxes or one box covering the coarse domain).  Returns, for every fine
// box, the coarse box holding its parent cells.
std::vector<int> coarse_map(const FabObj& fine, const FabObj& coarse) {
  const BoxArray& F = fine.ba->ba;
  const BoxArray& C = coarse.ba->ba;
  for (int d = 0; d < 3; ++d)
    if (C.dom.lo[d] != fdiv2(F.dom.lo[d]) || C.dom.hi[d] != fdiv2(F.dom.hi[d] + 1) - 1)
      fail(MG_EINVAL, "coarse domain is not the fine domain coarsened by 2");
  std::vector<int> map(F.boxes.size(), -1);
  for (size_t b = 0; b < F.boxes.size(); ++b) {
    Box p;
    for (int d = 0; d < 3; ++d) {
      p.lo[d] = fdiv2(F.boxes[b].lo[d]);
      p.hi[d] = fdiv2(F.boxes[b].hi[d]);
    }
    for (size_t cb = 0; cb < C.boxes.size(); ++cb)
      if (intersect(p, C.boxes[cb]).npts() == p.npts()) { map[b] = (int)cb; break; }
    if (map[b] < 0) fail(MG_EINVAL, "a fine box's parent cells span several coarse boxes");
  }
  return map;
}

// View of the coarse fab addressing coarse cell floor(lo_fine / 2) of the mapped box.
DView coarse_view(const FabObj& coarse, int cb, const Box& fine_box) {
  DView v = coarse.view(cb);
  const Box& C = coarse.ba->ba.boxes[cb];
  long long o = (long long)(fdiv2(fine_box.lo[2]) - C.lo[2]) * v.plane +
                (long long)(fdiv2(fine_box.lo[1]) - C.lo[1]) * v.pitch +
                (fdiv2(fine_box.lo[0]) - C.lo[0]);
  v.p = (char*)v.p + o * coarse.esize();
  return v;
}

}  // namespace

extern "C" {

int mg_version(void) { return 1; }

int mg_pool_info(mg_ctx_t h, size_t* cap, size_t* in_use) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    if (cap) *cap = c->pool_cap;
    if (in_use) *in_use = c->in_use.load();
    return MG_OK;
  });
}

int mg_kernel_launches(int64_t* n) {
  if (!n) return MG_EINVAL;
  *n = launches_so_far();
  return MG_OK;
}

const char* mg_last_error(void) { return g_err.c_str(); }

int mg_init(int device, size_t pool_bytes, mg_ctx_t* out) {
  return guard([&] {
    if (!out) fail(MG_EINVAL, "out is NULL");
    std::unique_ptr<Ctx> c(new Ctx);
    c->t0 = std::chrono::steady_clock::now();
    c->device = device;
    if (device >= 0) {
      int n = 0;
      MG_CK(cudaGetDeviceCount(&n));
      if (device >= n) fail(MG_EINVAL, "no such device");
      MG_CK(cudaSetDevice(device));
      MG_CK(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking));
      c->stream = c->own_stream;
      cudaMemPoolProps props{};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = device;
      MG_CK(cudaMemPoolCreate(&c->pool, &props));
      uint64_t thr = UINT64_MAX;
      MG_CK(cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &thr));
      size_t fr = 0, tot = 0;
      MG_CK(cudaMemGetInfo(&fr, &tot));
      c->pool_cap = pool_bytes ? pool_bytes : (size_t)(0.9 * (double)fr);
      c->batch_norms.ensure(*c, 64, c->stream);
      c->op_norm.ensure(*c, 1, c->stream);
      c->d_err = c->alloc(256, c->stream);
      MG_CK(cudaMemsetAsync(c->d_err->p, 0, 256, c->stream));
      MG_CK(cudaStreamSynchronize(c->stream));
    }
    *out = (mg_ctx_t)c.release();
    return MG_OK;
  });
}

int mg_finalize(mg_ctx_t h) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    if (c->device >= 0) {
      cudaSetDevice(c->device);
      server_stop(*c);
      cudaDeviceSynchronize();
    }
    amr_drop_plans(*c, 0);
    destroy_hierarchies(*c);
    c->op_cache.clear();
    c->fused_cache.clear();
    c->fabs.clear();
    c->tag_cache.clear();
    c->bas.clear();
    c->batch_norms.release(c->stream);
    c->op_norm.release(c->stream);
    c->d_err.reset();
    if (c->device >= 0) {
      cudaStreamSynchronize(c->stream);
      cudaDeviceSynchronize();
      if (c->pool) cudaMemPoolDestroy(c->pool);
      if (c->own_stream) cudaStreamDestroy(c->own_stream);
    }
    delete c;
    return MG_OK;
  });
}

int mg_set_stream(mg_ctx_t h, void* stream) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    c->require_device();
    MG_CK(cudaStreamSynchronize(c->stream));
    c->stream = stream ? S(stream) : c->own_stream;
    return MG_OK;
  });
}

int mg_box_array_create(mg_ctx_t h, const int dom_lo[3], const int dom_hi[3],
                        const int max_box[3], mg_ba_t* out) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c || !dom_lo || !dom_hi || !max_box || !out) fail(MG_EINVAL, "NULL argument");
    auto b = std::make_shared<BoxArrayObj>();
    std::string err;
    if (!chop(box_of(dom_lo, dom_hi), max_box, &b->ba, &err)) fail(MG_EINVAL, err);
    *out = c->add_ba(b);
    return MG_OK;
  });
}

int mg_box_array_from_list(mg_ctx_t h, const int dom_lo[3], const int dom_hi[3], int nbox,
                           const int* lo_hi, mg_ba_t* out) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c || !dom_lo || !dom_hi || !lo_hi || !out || nbox <= 0) fail(MG_EINVAL, "bad argument");
    auto b = std::make_shared<BoxArrayObj>();
    b->ba.dom = box_of(dom_lo, dom_hi);
    for (int i = 0; i < nbox; ++i) b->ba.boxes.push_back(box_of(lo_hi + 6 * i, lo_hi + 6 * i + 3));
    std::string err;
    if (!validate(b->ba, &err)) fail(MG_EINVAL, err);
    *out = c->add_ba(b);
    return MG_OK;
  });
}

int mg_box_array_info(mg_ctx_t h, mg_ba_t ba, int* nbox, int* dom_lohi, int* lo_hi) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    auto b = c->get_ba(ba);
    if (nbox) *nbox = (int)b->ba.boxes.size();
    if (dom_lohi)
      for (int d = 0; d < 3; ++d) { dom_lohi[d] = b->ba.dom.lo[d]; dom_lohi[3 + d] = b->ba.dom.hi[d]; }
    if (lo_hi)
      for (size_t i = 0; i < b->ba.boxes.size(); ++i)
        for (int d = 0; d < 3; ++d) {
          lo_hi[6 * i + d] = b->ba.boxes[i].lo[d];
          lo_hi[6 * i + 3 + d] = b->ba.boxes[i].hi[d];
        }
    return MG_OK;
  });
}

int mg_box_array_free(mg_ctx_t h, mg_ba_t ba) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    if (!c->bas.erase(ba)) fail(MG_EINVAL, "unknown box array handle");
    return MG_OK;
  });
}

int mg_hierarchy_levels(mg_ctx_t h, mg_ba_t ba, int* nlevels) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c || !nlevels) fail(MG_EINVAL, "NULL argument");
    *nlevels = (int)c->get_ba(ba)->hierarchy().size();
    return MG_OK;
  });
}

int mg_hierarchy_level(mg_ctx_t h, mg_ba_t ba, int level, mg_ba_t* out) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c || !out) fail(MG_EINVAL, "NULL argument");
    const auto& L = c->get_ba(ba)->hierarchy();
    if (level < 0 || level >= (int)L.size()) fail(MG_EINVAL, "level out of range");
    auto b = std::make_shared<BoxArrayObj>();
    b->ba = L[level];
    *out = c->add_ba(b);
    return MG_OK;
  });
}

int mg_copy_tags(mg_ctx_t h, mg_ba_t ba, const mg_bc* bc, int nghost, int64_t cap, int* tags,
                 int64_t* ntags) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c || !ntags) fail(MG_EINVAL, "NULL argument");
    int per[3];
    bc_code(bc, per);
    std::vector<CopyTag> t;
    std::string err;
    if (!make_copy_tags(c->get_ba(ba)->ba, per, nghost, &t, &err)) fail(MG_EINVAL, err);
    *ntags = (int64_t)t.size();
    if ((int64_t)t.size() > cap || !tags) fail(MG_EINVAL, "tag buffer too small");
    for (size_t i = 0; i < t.size(); ++i) {
      int* o = tags + 16 * i;
      o[0] = t[i].src_box;
      o[1] = t[i].dst_box;
      for (int d = 0; d < 3; ++d) {
        o[2 + d] = t[i].src_first[d];
        o[5 + d] = t[i].dst_lo[d];
        o[8 + d] = t[i].dir[d];
        o[11 + d] = t[i].ext[d];
      }
      o[14] = t[i].sign;
      o[15] = 0;
    }
    return MG_OK;
  });
}

int mg_bottom_matrix(const int n[3], const int periodic[3], double hh, double* M) {
  return guard([&] {
    if (!n || !periodic || !M || !(hh > 0)) fail(MG_EINVAL, "bad argument");
    std::vector<double> m;
    std::string err;
    if (!bottom_matrix(n, periodic, hh, &m, &err)) fail(MG_EINVAL, err);
    std::memcpy(M, m.data(), m.size() * sizeof(double));
    return MG_OK;
  });
}

int mg_fab_layout(mg_ctx_t h, mg_ba_t ba, int ncomp, int nghost, int dtype, size_t* bytes) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c || !bytes || ncomp < 1 || nghost < 0 || (dtype != MG_F64 && dtype != MG_F32))
      fail(MG_EINVAL, "bad argument");
    FabLayout L = make_layout(c->get_ba(ba)->ba, ncomp, nghost, dtype == MG_F64 ? 8 : 4);
    *bytes = (size_t)L.total * (dtype == MG_F64 ? 8 : 4);
    return MG_OK;
  });
}

static int64_t new_fab(Ctx* c, mg_ba_t ba, int ncomp, int nghost, int dtype, void* mem,
                       size_t bytes) {
  if (ncomp < 1 || nghost < 0 || (dtype != MG_F64 && dtype != MG_F32))
    fail(MG_EINVAL, "bad fab shape");
  c->require_device();
  auto f = std::make_shared<FabObj>();
  f->ba_id = ba;
  f->ba = c->get_ba(ba);
  f->dtype = dtype == MG_F64 ? DT_F64 : DT_F32;
  f->lay = make_layout(f->ba->ba, ncomp, nghost, f->esize());
  f->bytes = (size_t)f->lay.total * f->esize();
  if (mem) {
    if (bytes < f->bytes) fail(MG_EINVAL, "wrapped buffer smaller than mg_fab_layout bytes");
    if (((uintptr_t)mem & 255) != 0) fail(MG_EINVAL, "wrapped buffer must be 256-byte aligned");
    f->base = mem;
  } else {
    f->own = c->alloc(f->bytes, c->stream);
    f->base = f->own->p;
    MG_CK(cudaMemsetAsync(f->base, 0, f->bytes, c->stream));
    MG_CK(cudaStreamSynchronize(c->stream));
  }
  std::lock_guard<std::mutex> lk(c->mu);
  f->id = c->next_id++;
  c->fabs[f->id] = f;
  return f->id;
}

int mg_fab_alloc(mg_ctx_t h, mg_ba_t ba, int ncomp, int nghost, int dtype, mg_fab_t* out) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c || !out) fail(MG_EINVAL, "NULL argument");
    *out = new_fab(c, ba, ncomp, nghost, dtype, nullptr, 0);
    return MG_OK;
  });
}

int mg_fab_wrap(mg_ctx_t h, mg_ba_t ba, int ncomp, int nghost, int dtype, void* dptr,
                size_t bytes, mg_fab_t* out) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c || !out || !dptr) fail(MG_EINVAL, "NULL argument");
    *out = new_fab(c, ba, ncomp, nghost, dtype, dptr, bytes);
    return MG_OK;
  });
}

int mg_fab_ptr(mg_ctx_t h, mg_fab_t fab, int box, void** dptr, int64_t strides[4]) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c || !dptr) fail(MG_EINVAL, "NULL argument");
    auto f = c->get_fab(fab);
    if (box < 0 || box >= (int)f->ba->ba.boxes.size()) fail(MG_EINVAL, "box out of range");
    *dptr = (char*)f->base + f->lay.off[box] * f->esize();
    if (strides) {
      strides[0] = 1;
      strides[1] = f->lay.pitch[box];
      strides[2] = f->lay.plane[box];
      strides[3] = f->lay.cstride[box];
    }
    return MG_OK;
  });
}

int mg_fab_info(mg_ctx_t h, mg_fab_t fab, mg_ba_t* ba, int* ncomp, int* nghost, int* dtype) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    auto f = c->get_fab(fab);
    if (ba) *ba = f->ba_id;
    if (ncomp) *ncomp = f->lay.ncomp;
    if (nghost) *nghost = f->lay.g;
    if (dtype) *dtype = f->dtype == DT_F64 ? MG_F64 : MG_F32;
    return MG_OK;
  });
}

int mg_fab_free(mg_ctx_t h, mg_fab_t fab, void* stream) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    std::shared_ptr<FabObj> f;
    {
      std::lock_guard<std::mutex> lk(c->mu);
      auto it = c->fabs.find(fab);
      if (it == c->fabs.end()) fail(MG_EINVAL, "unknown fab handle");
      f = it->second;
      c->fabs.erase(it);
    }
    amr_drop_plans(*c, fab);
    drop_hierarchies_of(*c, fab);
    drop_cached_ops_of(*c, fab);
    // Order the release after the caller's stream and the context stream.
    cudaStream_t s = stream ? S(stream) : c->stream;
    if (s != c->stream) {
      cudaEvent_t ev;
      MG_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      MG_CK(cudaEventRecord(ev, c->stream));
      MG_CK(cudaStreamWaitEvent(s, ev, 0));
      cudaEventDestroy(ev);
    }
    if (f->valid_rows) f->valid_rows->reset(s);
    if (f->own) f->own->reset(s);
    return MG_OK;
  });
}

int mg_fab_copy_from_dense(mg_ctx_t h, mg_fab_t fab, const void* src, int src_on_host,
                           void* stream) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c || !src) fail(MG_EINVAL, "NULL argument");
    auto f = c->get_fab(fab);
    ensure_valid_rows(*c, *f);
    cudaStream_t s = S(stream);
    const Box& D = f->ba->ba.dom;
    int n[3] = {D.len(0), D.len(1), D.len(2)};
    size_t bytes = (size_t)D.npts() * f->lay.ncomp * f->esize();
    DevBufP stage;
    const void* dsrc = src;
    if (src_on_host) {
      stage = c->alloc(bytes, s);
      MG_CK(cudaMemcpyAsync(stage->p, src, bytes, cudaMemcpyHostToDevice, s));
      dsrc = stage->p;
    }
    MG_CK(launch_dense_copy(f->dtype, (const DRow*)f->valid_rows->p, (int)f->ba->ba.boxes.size(),
                            f->nrows, const_cast<void*>(dsrc), D.lo, n, f->lay.ncomp, 0, s));
    if (stage) stage->reset(s);
    return MG_OK;
  });
}

int mg_fab_copy_to_dense(mg_ctx_t h, mg_fab_t fab, void* dst, int dst_on_host, void* stream) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c || !dst) fail(MG_EINVAL, "NULL argument");
    auto f = c->get_fab(fab);
    ensure_valid_rows(*c, *f);
    cudaStream_t s = S(stream);
    const Box& D = f->ba->ba.dom;
    int n[3] = {D.len(0), D.len(1), D.len(2)};
    size_t bytes = (size_t)D.npts() * f->lay.ncomp * f->esize();
    DevBufP stage;
    void* ddst = dst;
    if (dst_on_host) {
      stage = c->alloc(bytes, s);
      ddst = stage->p;
    }
    MG_CK(launch_dense_copy(f->dtype, (const DRow*)f->valid_rows->p, (int)f->ba->ba.boxes.size(),
                            f->nrows, ddst, D.lo, n, f->lay.ncomp, 1, s));
    if (dst_on_host) {
      MG_CK(cudaMemcpyAsync(dst, stage->p, bytes, cudaMemcpyDeviceToHost, s));
      stage->reset(s);
    }
    return MG_OK;
  });
}

int mg_fab_set_val(mg_ctx_t h, mg_fab_t fab, double v, int include_ghosts, void* stream) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    auto f = c->get_fab(fab);
    cudaStream_t s = S(stream);
    if (include_ghosts) {
      MG_CK(launch_set_flat(f->dtype, f->base, f->lay.total, v, s));
    } else {
      ensure_valid_rows(*c, *f);
      // every component: one launch per component over the valid rows
      for (int comp = 0; comp < f->lay.ncomp; ++comp) {
        std::vector<DRow> rows;
        long long n = 0;
        append_rows(&rows, &n, f->ba->ba, 0, 1.0, 0, [&](int b, DRow& R) {
          R.v[0] = f->view(b);
          R.v[0].p = (char*)R.v[0].p + comp * R.v[0].cstride * f->esize();
        });
        OpTable t = upload_table(*c, rows, n, s);
        MG_CK(launch_set_valid(f->dtype, t.rows(), t.nbox, t.nrows, v, s));
        t.d->reset(s);
      }
    }
    return MG_OK;
  });
}

int mg_fill_boundary(mg_ctx_t h, mg_fab_t fab, const mg_bc* bc, void* stream) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    auto f = c->get_fab(fab);
    launch_fill(*c, *f, bc, S(stream));
    return MG_OK;
  });
}

int mg_fill_boundary_unfused(mg_ctx_t h, mg_fab_t fab, const mg_bc* bc, void* stream) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    auto f = c->get_fab(fab);
    FillPlan& P = fill_plan(*c, *f, bc, -1);
    cudaStream_t s = S(stream);
    for (int t = 0; t < P.ntags(); ++t) {
      const int a = P.set->first_chunk[t], b = P.set->first_chunk[t + 1];
      if (b > a)
        MG_CK(launch_copy_tags(f->dtype, P.tags(), P.chunks() + a, b - a, f->base, f->lay.ncomp, s));
    }
    return MG_OK;
  });
}

int mg_smooth(mg_ctx_t h, mg_fab_t phi, mg_fab_t rhs, const mg_bc* bc, double hh, int color,
              void* stream) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    auto fp = c->get_fab(phi);
    auto fr = c->get_fab(rhs);
    same_shape(*fp, *fr, "mg_smooth");
    if (fp->lay.g < 1) fail(MG_EINVAL, "phi needs at least one ghost cell");
    if ((color & ~MG_SMOOTH_DIRECT_READS) == 0 || (color & ~MG_SMOOTH_DIRECT_READS) == 1) {
      if (color & MG_SMOOTH_DIRECT_READS) {  // one half-sweep reading neighbouring boxes
        int per[3];
        const int code = bc_code(bc, per);
        cudaStream_t s = S(stream);
        double hv = default_h(*fp, hh);
        const std::string op = "smooth_direct" + std::to_string(code);
        const OpTable& t = op_table(*c, op.c_str(), {phi, rhs}, hv, [&] {
          FaceReads faces = direct_neighbours(*fp, per);
          if (!faces.ok())
            fail(MG_EINVAL, "direct reads need boxes on a regular grid and even periodic extents");
          OpTable tt = make_table(*c, fp->ba->ba, 0, hv, 0, [&](int b, DRow& R) {
            R.v[0] = fp->view(b);
            R.v[1] = fr->view(b);
            faces.apply(b, R);
          }, c->stream);
          tt.direct = true;
          return tt;
        });
        MG_CK(launch_rbgs_half(fp->dtype, t.rows(), t.nbox, t.nrows, color & 1, s, true, nullptr, t.width));
        return MG_OK;
      }
    }
    if (color < 0 || color > 2) fail(MG_EINVAL, "color must be 0, 1 or 2 (0 / 1 may add MG_SMOOTH_DIRECT_READS)");
    cudaStream_t s = S(stream);
    double hv = default_h(*fp, hh);
    const OpTable& t = op_table(*c, "smooth", {phi, rhs}, hv, [&] {
      return make_table(*c, fp->ba->ba, 0, hv, 0, [&](int b, DRow& R) {
        R.v[0] = fp->view(b);
        R.v[1] = fr->view(b);
      }, c->stream);
    });
    if (color == 2 && fused_eligible(*fp, *fr)) {
      // one fused sweep into the scratch partner, then copied back (ghosts included; they
      // are refilled before the next read)
      auto tmp = partner_of(*c, *fp);
      int per[3];
      bc_code(bc, per);
      const FusedTable* ft = &fused_table(*c, phi, *fp, rhs, *fr, -phi, *tmp, bc, hv);
      if (ft->ok) {
        launch_fill(*c, *fp, bc, s);
        launch_fill(*c, *fr, bc, s);
        launch_fused(*c, *ft, fp->dtype, s);
        MG_CK(cudaMemcpyAsync(fp->base, tmp->base, fp->bytes, cudaMemcpyDeviceToDevice, s));
        return MG_OK;
      }
    }
    if (color < 2) {
      MG_CK(launch_rbgs_half(fp->dtype, t.rows(), t.nbox, t.nrows, color, s, false, nullptr, t.width));
    } else {
      for (int col = 0; col < 2; ++col) {
        launch_fill(*c, *fp, bc, s);
        MG_CK(launch_rbgs_half(fp->dtype, t.rows(), t.nbox, t.nrows, col, s, false, nullptr, t.width));
      }
    }
    return MG_OK;
  });
}

int mg_smooth_fused(mg_ctx_t h, mg_fab_t phi_src, mg_fab_t rhs, mg_fab_t phi_dst,
                    const mg_bc* bc, double hh, void* stream) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    auto fa = c->get_fab(phi_src);
    auto fr = c->get_fab(rhs);
    auto fb = c->get_fab(phi_dst);
    same_shape(*fa, *fr, "mg_smooth_fused");
    same_shape(*fa, *fb, "mg_smooth_fused");
    if (!fused_eligible(*fa, *fr)) fail(MG_EINVAL, "fused sweep needs phi nghost >= 2, rhs >= 1");
    if (fb->lay.g != fa->lay.g || fb->lay.ncomp != 1)
      fail(MG_EINVAL, "phi_dst must have the layout of phi_src");
    if (phi_src == phi_dst) fail(MG_EINVAL, "the fused sweep is out of place");
    double hv = default_h(*fa, hh);
    const FusedTable& t = fused_table(*c, phi_src, *fa, rhs, *fr, phi_dst, *fb, bc, hv);
    if (!t.ok) fail(MG_EINVAL, "boxes too large for the fused sweep's shared-memory tiles");
    launch_fused(*c, t, fa->dtype, S(stream));
    return MG_OK;
  });
}

int mg_residual(mg_ctx_t h, mg_fab_t phi, mg_fab_t rhs, mg_fab_t r, double hh, double* norm,
                void* stream) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    auto fp = c->get_fab(phi);
    auto fr = c->get_fab(rhs);
    same_shape(*fp, *fr, "mg_residual");
    std::shared_ptr<FabObj> fo;
    if (r) {
      fo = c->get_fab(r);
      same_shape(*fp, *fo, "mg_residual");
    }
    if (fp->lay.g < 1) fail(MG_EINVAL, "phi needs at least one ghost cell");
    cudaStream_t s = S(stream);
    double hv = default_h(*fp, hh);
    const OpTable& t = op_table(*c, "residual", {phi, rhs, r}, hv, [&] {
      return make_table(*c, fp->ba->ba, 0, hv, 0, [&](int b, DRow& R) {
        R.v[0] = fp->view(b);
        R.v[1] = fr->view(b);
        if (fo) R.v[2] = fo->view(b);
      }, c->stream);
    });
    std::lock_guard<std::mutex> nl(c->op_norm_mu);
    unsigned long long* dn = (unsigned long long*)c->op_norm.d->p;
    MG_CK(cudaMemsetAsync(dn, 0, 8, s));
    MG_CK(launch_residual(fp->dtype, t.rows(), t.nbox, t.nrows, dn, s));
    if (norm) {
      MG_CK(cudaMemcpyAsync(c->op_norm.h, dn, 8, cudaMemcpyDeviceToHost, s));
      MG_CK(cudaStreamSynchronize(s));
      std::memcpy(norm, c->op_norm.h, 8);
    }
    return MG_OK;
  });
}

int mg_residual_restrict(mg_ctx_t h, mg_fab_t phi, mg_fab_t rhs, mg_fab_t crhs, mg_fab_t cphi,
                         double hh, void* stream) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    auto fp = c->get_fab(phi);
    auto fr = c->get_fab(rhs);
    auto fc = c->get_fab(crhs);
    std::shared_ptr<FabObj> fz;
    if (cphi) {
      fz = c->get_fab(cphi);
      same_shape(*fc, *fz, "mg_residual_restrict");
    }
    same_shape(*fp, *fr, "mg_residual_restrict");
    if (fc->dtype != fp->dtype) fail(MG_EINVAL, "coarse and fine types differ");
    if (!aligned(fp->ba->ba)) fail(MG_EINVAL, "fine boxes must have even bounds");
    if (fp->lay.g < 1) fail(MG_EINVAL, "phi needs at least one ghost cell");
    std::vector<int> map = coarse_map(*fp, *fc);
    cudaStream_t s = S(stream);
    double hv = default_h(*fp, hh);
    const BoxArray& F = fp->ba->ba;
    const OpTable& t = op_table(*c, "resrestrict", {phi, rhs, crhs, cphi}, hv, [&] {
      return make_table(*c, F, 1, hv, 0, [&](int b, DRow& R) {
        R.v[0] = fp->view(b);
        R.v[1] = fr->view(b);
        R.c[0] = coarse_view(*fc, map[b], F.boxes[b]);
        if (fz) R.c[1] = coarse_view(*fz, map[b], F.boxes[b]);
      }, c->stream);
    });
    MG_CK(launch_residual_restrict(fp->dtype, t.rows(), t.nbox, t.nrows, s, false, t.width));
    return MG_OK;
  });
}

int mg_restrict(mg_ctx_t h, mg_fab_t fine, mg_fab_t coarse, void* stream) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    auto ff = c->get_fab(fine);
    auto fc = c->get_fab(coarse);
    if (fc->dtype != ff->dtype) fail(MG_EINVAL, "coarse and fine types differ");
    if (!aligned(ff->ba->ba)) fail(MG_EINVAL, "fine boxes must have even bounds");
    std::vector<int> map = coarse_map(*ff, *fc);
    cudaStream_t s = S(stream);
    const BoxArray& F = ff->ba->ba;
    const OpTable& t = op_table(*c, "restrict", {fine, coarse}, 1.0, [&] {
      return make_table(*c, F, 1, 1.0, 0, [&](int b, DRow& R) {
        R.v[0] = ff->view(b);
        R.c[0] = coarse_view(*fc, map[b], F.boxes[b]);
      }, c->stream);
    });
    MG_CK(launch_restrict(ff->dtype, t.rows(), t.nbox, t.nrows, s));
    return MG_OK;
  });
}

int mg_prolong_add(mg_ctx_t h, mg_fab_t coarse, mg_fab_t fine, void* stream) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    auto ff = c->get_fab(fine);
    auto fc = c->get_fab(coarse);
    if (fc->dtype != ff->dtype) fail(MG_EINVAL, "coarse and fine types differ");
    std::vector<int> map = coarse_map(*ff, *fc);
    cudaStream_t s = S(stream);
    const BoxArray& F = ff->ba->ba;
    const OpTable& t = op_table(*c, "prolong", {coarse, fine}, 1.0, [&] {
      return make_table(*c, F, 0, 1.0, 0, [&](int b, DRow& R) {
        R.v[0] = ff->view(b);
        R.c[0] = coarse_view(*fc, map[b], F.boxes[b]);
      }, c->stream);
    });
    MG_CK(launch_prolong_add(ff->dtype, t.rows(), t.nbox, t.nrows, s, t.width));
    return MG_OK;
  });
}

int mg_prolong_add_trilinear(mg_ctx_t h, mg_fab_t coarse, mg_fab_t fine, void* stream) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    auto ff = c->get_fab(fine);
    auto fc = c->get_fab(coarse);
    if (fc->dtype != ff->dtype) fail(MG_EINVAL, "coarse and fine types differ");
    if (fc->lay.g < 1) fail(MG_EINVAL, "trilinear prolongation reads one coarse ghost layer");
    std::vector<int> map = coarse_map(*ff, *fc);
    cudaStream_t s = S(stream);
    const BoxArray& F = ff->ba->ba;
    const OpTable& t = op_table(*c, "prolong", {coarse, fine}, 1.0, [&] {
      return make_table(*c, F, 0, 1.0, 0, [&](int b, DRow& R) {
        R.v[0] = ff->view(b);
        R.c[0] = coarse_view(*fc, map[b], F.boxes[b]);
      }, c->stream);
    });
    MG_CK(launch_prolong_trilinear(ff->dtype, t.rows(), t.nbox, t.nrows, s, t.width));
    return MG_OK;
  });
}

int mg_bottom_solve(mg_ctx_t h, mg_fab_t rhs, mg_fab_t phi, const mg_bc* bc, double hh,
                    void* stream) {
  return guard([&] {
    Ctx* c = (Ctx*)h;
    if (!c) fail(MG_EINVAL, "ctx is NULL");
    auto fr = c->get_fab(rhs);
    auto fp = c->get_fab(phi);
    same_shape(*fr, *fp, "mg_bottom_solve");
    int per[3];
    bc_code(bc, per);
    const BoxArray& B = fp->ba->ba;
    int n[3] = {B.dom.len(0), B.dom.len(1), B.dom.len(2)};
    double hv = default_h(*fp, hh);
    const std::vector<double>& Mt = bottom_matrix_t(*c, n, per, hv);
    long long N = B.dom.npts();
    std::vector<long long> orhs(N), ophi(N);
    for (size_t b = 0; b < B.boxes.size(); ++b) {
      const Box& X = B.boxes[b];
      for (int z = X.lo[2]; z <= X.hi[2]; ++z)
        for (int y = X.lo[1]; y <= X.hi[1]; ++y)
          for (int x = X.lo[0]; x <= X.hi[0]; ++x) {
            long long i = ((long long)(z - B.dom.lo[2]) * n[1] + (y - B.dom.lo[1])) * n[0] +
                          (x - B.dom.lo[0]);
            orhs[i] = fr->lay.at(B, (int)b, x, y, z);
            ophi[i] = fp->lay.at(B, (int)b, x, y, z);
          }
    }
    cudaStream_t s = S(stream);
    DevBufP dM = c->upload(Mt.data(), Mt.size() * 8, s);
    DevBufP dr = c->upload(orhs.data(), N * 8, s);
    DevBufP dp = c->upload(ophi.data(), N * 8, s);
    BottomJob J{};
    J.Mt = (const double*)dM->p;
    J.off_rhs = (const long long*)dr->p;
    J.off_phi = (const long long*)dp->p;
    J.rhs = fr->base;
    J.phi = fp->base;
    J.N = (int)N;
    DevBufP dj = c->upload(&J, sizeof J, s);
    MG_CK(launch_bottom(fp->dtype, (const BottomJob*)dj->p, 1, (int)N, s));
    dj->reset(s);
    dp->reset(s);
    dr->reset(s);
    dM->reset(s);
    return MG_OK;
  });
}

}  // extern "C"
