// Runtime objects behind the C ABI: context, stream-ordered memory pool, box arrays, fabs,
// cached ghost-fill plans and stencil tables, multigrid hierarchies.
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/gbmg.h"
#include "mg_host.hpp"
#include "mg_kernels.hpp"

namespace gbmg {

struct MgError {
  int code;
  std::string msg;
};

[[noreturn]] void fail(int code, const std::string& msg);
void check_cuda(cudaError_t e, const char* what);
void set_last_error(const std::string& msg);

// Runs f() and converts exceptions into MG_E* codes plus the thread's last-error message.
template <class F>
int guard(F&& f) {
  try {
    set_last_error("");
    return f();
  } catch (const MgError& e) {
    set_last_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error("host out of memory");
    return MG_ENOMEM;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return MG_EINVAL;
  }
}
#define MG_CK(call) ::gbmg::check_cuda((call), #call)

struct Ctx;

// Device memory from the context pool, released in stream order.
struct DevBuf {
  Ctx* ctx = nullptr;
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf();
  void reset(cudaStream_t s);
};
using DevBufP = std::unique_ptr<DevBuf>;

struct Ctx;

// Norm slots of batched steps: a device array of max-norm bit patterns and its pinned host
// mirror.  Growing keeps the device values: a mixed-precision member's next step scales its
// residual by the norm its last check left there.
struct NormBuf {
  DevBufP d;
  unsigned long long* h = nullptr;
  int slots = 0;
  void ensure(Ctx& c, int n, cudaStream_t s);  // at least n slots (new slots zero)
  void release(cudaStream_t s);
};

struct BoxArrayObj {
  BoxArray ba;
  bool levels_built = false;
  bool levels_ok = false;
  std::string levels_err;
  std::vector<BoxArray> levels;
  const std::vector<BoxArray>& hierarchy();  // throws MG_EINVAL if no valid hierarchy
};

// Device copy tags + chunk list of one ghost-fill pattern.  Offsets are relative to a fab's
// base, so every fab with the same box array, ghost width, type and component count shares
// one set (the cached communication pattern of Sec. 2).
struct TagSet {
  DevBufP tags_buf, chunks_buf;
  int nchunks = 0;
  std::vector<int> first_chunk;  // chunks of tag t: [first_chunk[t], first_chunk[t+1])
};

// A fab's ghost-fill plan for one set of BCs and number of layers.
struct FillPlan {
  std::shared_ptr<TagSet> set;
  const DTag* tags() const { return set && set->tags_buf ? (const DTag*)set->tags_buf->p : nullptr; }
  const int2* chunks() const { return set && set->chunks_buf ? (const int2*)set->chunks_buf->p : nullptr; }
  int nchunks() const { return set ? set->nchunks : 0; }
  int ntags() const { return set ? (int)set->first_chunk.size() - 1 : 0; }
};

struct FabObj {
  int64_t id = 0;
  int64_t ba_id = 0;
  std::shared_ptr<BoxArrayObj> ba;
  FabLayout lay;
  int dtype = DT_F64;
  void* base = nullptr;
  size_t bytes = 0;
  DevBufP own;  // null for wrapped memory
  std::map<int, std::unique_ptr<FillPlan>> fills;  // key: bc code
  DevBufP valid_rows;  // DRow table, v[0] = this fab (fine x-lines)
  long long nrows = 0;
  std::shared_ptr<FabObj> partner;  // same-layout scratch for out-of-place sweeps
  DView view(int b) const;
  int esize() const { return dtype == DT_F64 ? 8 : 4; }
};

// Face reads of the stencil kernels (DRow::nbd / nbf) for the boxes of fab f under the given
// BCs.  Returns false, leaving `out` empty, unless the boxes form a regular grid (equal
// extents on a lattice anchored at the domain's low corner) with one layout and every
// periodic extent is even (an odd one would make a cell's periodic image one of its own
// colour, updated by the same half-sweep), so that each
// face's first ghost layer is exactly one face layer of one box (or its periodic image), or
// lies across a Dirichlet face; the kernels must then read filled ghost cells.
struct FaceReads {
  std::vector<std::array<long long, 6>> d;
  std::vector<int> flags;
  bool ok() const { return !d.empty(); }
  void apply(int b, DRow& R) const {
    if (!ok()) return;
    for (int f = 0; f < 6; ++f) R.nbd[f] = d[b][f];
    R.nbf = flags[b];
  }
};
// outside_ghosts: faces on the domain boundary that are not periodic read their own ghost
// cells (filled by the caller, e.g. coarse/fine ghosts of a refined region) instead of the
// negated boundary cell.
FaceReads direct_neighbours(const FabObj& f, const int periodic[3], bool outside_ghosts = false);

struct OpTable {
  DevBufP d;
  int nbox = 0;
  long long nrows = 0;
  bool direct = false;  // rows carry box-face reads (DRow::nbd / nbf)
  int width = 0;        // widest box x-extent of the rows
  const DRow* rows() const { return d ? (const DRow*)d->p : nullptr; }
};

struct Hierarchy;

// Launch configuration of the fused sweep: tile rows, z-planes per CTA, prefetch depth, rhs
// staged through shared memory (1) or read from global memory (0).
struct FusedCfg {
  int ty = 16, zc = 16, depth = 2, rhs_smem = 1;
};

struct Ctx {
  // Timing of the finest-level half-sweep inside solves (one CUDA event pair around the
  // first such launch of every V-cycle, recorded on the solve stream; captured into the
  // step graph when enabled).
  bool sweep_timing = false;
  double sweep_ms = 0.0;
  long long sweep_n = 0;
  int device = -1;
  cudaStream_t stream = nullptr;   // context stream (solves)
  cudaStream_t own_stream = nullptr;
  cudaMemPool_t pool = nullptr;
  size_t pool_cap = 0;
  std::atomic<size_t> in_use{0};
  std::mutex mu;  // guards the handle maps and the pool accounting
  std::map<int64_t, std::shared_ptr<BoxArrayObj>> bas;
  std::map<int64_t, std::shared_ptr<FabObj>> fabs;
  int64_t next_id = 1;
  std::chrono::steady_clock::time_point t0;
  std::vector<std::shared_ptr<Hierarchy>> hier;   // cached solver hierarchies
  std::recursive_mutex hier_mu;                    // guards hier (scheduler thread + callers)
  std::map<std::string, std::vector<double>> bottom_cache;  // key -> transposed M
  // device error word written by kernels whose bounded waits expire (0 = fine)
  DevBufP d_err;
  // norm slots of mg_solve_batch, and the one norm of the level-operation entry points
  // (the serving scheduler keeps its own, one set per precision)
  NormBuf batch_norms, op_norm;
  std::mutex op_norm_mu;
  // cached stencil tables of the level-operation entry points, keyed by op, fabs and h
  struct CachedOp {
    std::vector<int64_t> fabs;
    OpTable t;
  };
  std::map<std::string, CachedOp> op_cache;
  std::map<std::string, std::shared_ptr<struct FusedTable>> fused_cache;
  // ghost-fill patterns shared by all fabs of one layout
  std::mutex tag_mu;
  std::map<std::string, std::shared_ptr<TagSet>> tag_cache;
  std::mutex bottom_mu;  // guards bottom_cache
  // fused-sweep autotuning results per box shape
  std::mutex tune_mu;
  std::map<std::string, FusedCfg> tune;
  bool tune_loaded = false;
  void load_tune_file();
  void save_tune_entry(const std::string& key, const FusedCfg& cfg);
  // serving
  struct Server;
  std::shared_ptr<Server> server;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  void require_device() const {
    if (device < 0) fail(MG_EINVAL, "host-only context: no device memory or kernels");
  }
  DevBufP alloc(size_t bytes, cudaStream_t s);
  DevBufP upload(const void* host, size_t bytes, cudaStream_t s);
  std::shared_ptr<BoxArrayObj> get_ba(int64_t id);
  std::shared_ptr<FabObj> get_fab(int64_t id);
  int64_t add_ba(std::shared_ptr<BoxArrayObj> b);
};

int bc_code(const mg_bc* bc, int periodic[3]);  // validates; returns a small cache key

// Plans and tables ----------------------------------------------------------------------
// Ghost fill of the first `layers` ghost layers (-1: all of the fab's layers).
FillPlan& fill_plan(Ctx& c, FabObj& f, const mg_bc* bc, int layers = -1);
void launch_fill(Ctx& c, FabObj& f, const mg_bc* bc, cudaStream_t s, int layers = -1);
void ensure_valid_rows(Ctx& c, FabObj& f);

// Fabs owned by the library on behalf of a request (host-memory serving): allocated from the
// pool and zero-filled on stream s (no synchronisation), registered under a new handle;
// released in stream order on s.  Dense (nz, ny, nx) host arrays move in and out through a
// pool staging buffer on s (the host memory must stay valid until s has passed the copy).
int64_t add_pool_fab(Ctx& c, std::shared_ptr<BoxArrayObj> ba, int64_t ba_id, int ncomp, int g,
                     int dt, cudaStream_t s);
void release_fab(Ctx& c, int64_t id, cudaStream_t s);
void dense_upload(Ctx& c, FabObj& f, const void* host, cudaStream_t s);
void dense_download(Ctx& c, FabObj& f, void* host, cudaStream_t s);

// Appends one row per box of `ba` to a host table; views(b, row) fills the views of box b.
// kind 0: rows are fine x-lines; kind 1: rows are coarse x-lines (n/2 of each dimension).
template <class F>
void append_rows(std::vector<DRow>* rows, long long* nrows, const BoxArray& ba, int kind,
                 double h, int solve, F&& views) {
  for (size_t b = 0; b < ba.boxes.size(); ++b) {
    DRow R{};
    const Box& B = ba.boxes[b];
    for (int d = 0; d < 3; ++d) { R.lo[d] = B.lo[d]; R.n[d] = B.len(d); }
    R.solve = solve;
    R.row0 = *nrows;
    R.h2 = h * h;
    R.ih2 = 1.0 / (h * h);
    views((int)b, R);
    *nrows += kind == 0 ? (long long)R.n[1] * R.n[2] : (long long)(R.n[1] / 2) * (R.n[2] / 2);
    rows->push_back(R);
  }
}
OpTable upload_table(Ctx& c, const std::vector<DRow>& rows, long long nrows, cudaStream_t s);

template <class F>
OpTable make_table(Ctx& c, const BoxArray& ba, int kind, double h, int solve, F&& views,
                   cudaStream_t s) {
  std::vector<DRow> rows;
  long long n = 0;
  append_rows(&rows, &n, ba, kind, h, solve, views);
  return upload_table(c, rows, n, s);
}

// Cached table for a level operation on the given fabs (built on the context stream).
template <class B>
const OpTable& op_table(Ctx& c, const char* op, std::vector<int64_t> ids, double h, B&& build) {
  std::string key = op;
  for (int64_t id : ids) key += ":" + std::to_string(id);
  unsigned long long hb;
  static_assert(sizeof hb == sizeof h, "");
  std::memcpy(&hb, &h, sizeof h);
  key += ":" + std::to_string(hb);
  auto it = c.op_cache.find(key);
  if (it != c.op_cache.end()) return it->second.t;
  OpTable t = build();
  check_cuda(cudaStreamSynchronize(c.stream), "cudaStreamSynchronize");
  auto& e = c.op_cache[key];
  e.fabs = std::move(ids);
  e.t = std::move(t);
  return e.t;
}
void drop_cached_ops_of(Ctx& c, int64_t fab_id);

// Fused red + black sweep table: rows (src, rhs, dst views + Dirichlet-face flags) and
// (box, y0) tiles.  ok == false when the layout cannot use the fused kernel.
struct FusedTable {
  bool ok = false;
  OpTable rows;
  DevBufP units;
  int nunits = 0, ty = 16, zc = 16, depth = 2, max_pitch = 0, max_pitch_r = 0;
  bool rhs_smem = true;
  std::vector<int64_t> owner_fabs;  // for cache invalidation
};
bool fused_eligible(const FabObj& phi, const FabObj& rhs);
FusedTable make_fused(Ctx& c, const BoxArray& ba, double h, const FabObj& src, const FabObj& rhs,
                      const FabObj& dst, const int periodic[3], cudaStream_t s);
void launch_fused(Ctx& c, const FusedTable& t, int dt, cudaStream_t s);
// Cached fused table for (src, rhs, dst, bc, h); src/rhs/dst ids are the fab handles (0 for
// internal fabs, which must then be cached by their owner instead).
const FusedTable& fused_table(Ctx& c, int64_t src_id, FabObj& src, int64_t rhs_id, FabObj& rhs,
                              int64_t dst_id, FabObj& dst, const mg_bc* bc, double h);
std::shared_ptr<FabObj> partner_of(Ctx& c, FabObj& f);
void check_device_error(Ctx& c);

// Copy-tag conversion to device layout (offsets relative to the fab base).
std::vector<DTag> device_tags(const BoxArray& ba, const FabLayout& lay,
                              const std::vector<CopyTag>& tags, int base_index);

// Hierarchy / solve -----------------------------------------------------------------------
// FP32 V-cycles per outer FP64 iteration of the mixed form by default (measured on GB300:
// the 512^3 mixed solve 69.6 ms with one, 59.6 ms with two).
constexpr int kDefaultInnerCycles = 2, kMaxInnerCycles = 8;
struct SolveParams {
  int nu1 = 2, nu2 = 2, max_iter = 50, precision = MG_PREC_F64, smoother = MG_SMOOTH_AUTO;
  int use_graph = 1, fixed_vcycles = -1, coarse_cells = 0, direct_reads = 1;
  int prolong = MG_PROLONG_CONSTANT;
  int inner = kDefaultInnerCycles;  // FP32 V-cycles per outer iteration (mixed form)
  double h = 0.0;
};
SolveParams params_from(const mg_options* o, const BoxArray& ba);

int solve(Ctx& c, int64_t rhs, int64_t phi, const mg_bc* bc, double tol, const SolveParams& p,
          mg_result* res);
int solve_batch(Ctx& c, int n, const int64_t* rhs, const int64_t* phi, const mg_bc* bcs,
                double tol, const SolveParams& p, mg_result* res);
void drop_hierarchies_of(Ctx& c, int64_t fab_id);
void destroy_hierarchies(Ctx& c);

// Serving
int server_submit(Ctx& c, int64_t rhs, int64_t phi, const mg_bc* bc, double tol,
                  const SolveParams& p, int64_t* ticket);
int server_submit_host(Ctx& c, std::shared_ptr<BoxArrayObj> ba, const double* rhs, double* phi,
                       int phi_is_guess, const mg_bc* bc, double tol, const SolveParams& p,
                       int64_t* ticket);
int server_poll(Ctx& c, int64_t ticket, int timeout_ms, mg_result* res);
void server_stop(Ctx& c);
// Two-level AMR plans (mg_amr.cu): drop those using fab `fab` (0: all of the context).
void amr_drop_plans(Ctx& c, int64_t fab);
void server_trim(Ctx& c);
void server_stats(Ctx& c, mg_server_stats* out);

// Bottom matrix (transposed), cached per (n, periodic, h).
const std::vector<double>& bottom_matrix_t(Ctx& c, const int n[3], const int periodic[3],
                                           double h);

}  // namespace gbmg
