// Device-side tables and kernel launchers of the multigrid path (sm_103a).
//
// Every stencil operation is one launch over all boxes of a level (or of several levels of
// several solves): the launch walks a device "box table" of DRow entries, the analogue of
// the array of Array4 views behind the fused ParallelFor of Sec. 3.2 of the AMReX/pyAMReX
// review.  The ghost fill walks a device copy-tag table (Sec. 2 cached communication
// patterns, Sec. 3.5 fused pack/unpack).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gbmg {

enum { DT_F64 = 0, DT_F32 = 1 };

// View of one box of a fab: p addresses the first valid cell (local (0,0,0), component 0);
// cell (x,y,z) is p[z*plane + y*pitch + x], ghosts at negative / >= n local indices.
struct DView {
  void* p;
  long long plane;
  long long cstride;  // elements per component
  int pitch;
  int g;
};

// One box of a level in a stencil launch.  row0 is the first "row" (an x-line, or a coarse
// x-line for restriction) of this box in the launch's row space; rows of a box are ordered
// y fastest, then z.
struct DRow {
  int lo[3];
  int n[3];
  int solve;     // slot in per-solve arrays (norms, scales)
  int pad_;
  long long row0;
  double h2;     // h*h of this level
  double ih2;    // 1/(h*h)
  DView v[3];    // op-specific fine views (see each launcher)
  DView c[2];    // op-specific coarse views, addressing coarse cell floor(lo/2)
  // Neighbour reads of the FP64 smoother / residual / residual+restriction kernels, per face
  // x-, x+, y-, y+, z-, z+ of the box: a stencil value in the face's first ghost layer is read
  // at (ghost cell + nbd[f]) elements of v[0], negated if bit f of nbf is set.  All zero: the
  // ghost cells themselves (filled beforehand).  Set from the box array (direct_neighbours):
  // the cell of the neighbouring box or periodic image that the fill would copy, or the box's
  // own boundary cell (negated) across a Dirichlet face.
  long long nbd[6];
  int nbf;
  int pad2_;
};

// Ghost-fill tag: destination cells dst + x + y*dsy + z*dsz (0 <= x < ex ...) take
// sign * base[src + x*ssx + y*ssy + z*ssz]; components at +c*dcs / +c*scs.  Offsets are in
// elements from the fab's base address.  sign 0 writes 0.
struct DTag {
  long long src, dst;
  long long scs, dcs;
  int ssx, ssy, ssz;
  int dsy, dsz;
  int ex, ey, ez;
  int sign;
  int pad_[3];
};

// Exact bottom solve of one level: phi[off_phi[i]] = sum_j Mt[j*N + i] * rhs[off_rhs[j]].
struct BottomJob {
  const double* Mt;        // transposed (pseudo-)inverse, N x N
  const long long* off_rhs;
  const long long* off_phi;
  const void* rhs;
  void* phi;
  int N;
  int pad_;
};

// The coarse end of a V-cycle (levels lc .. bottom) in one CTA: every level held densely in
// shared memory (phi with one ghost layer, then rhs, x fastest), offsets in elements of the
// level's type.  Level lc's cell i (dense, x fastest) lives at phi[off_phi[i]] and
// rhs[off_rhs[i]] in its fabs: phi and rhs are gathered from there and phi scattered back.
constexpr int kMaxCoarseLevels = 8;
struct CoarseLevel {
  int n[3];   // level domain extents
  int lo[3];  // level domain low corner (colour parity, gather offsets)
  int off_phi, off_rhs;
  double h2, ih2;
};
struct CoarseJob {
  const long long* off_phi;
  const long long* off_rhs;
  void* phi;
  const void* rhs;
  const double* Mt;  // bottom (pseudo-)inverse, transposed, over the last level's cells
  int nlev, nu1, nu2, N;
  int periodic[3];
  CoarseLevel lev[kMaxCoarseLevels];
};

// The copy-tag kernel gives each warp a chunk of whole x-rows of one tag: about kTagChunk1
// destination cells for one-component FP64 fabs, kTagChunk1F for one-component FP32 fabs
// (the mixed form's fused levels: 512^3 mixed solve 59.8 -> 59.2 ms against 64), kTagChunkN
// for more components (measured best on GB300),
// at least one row.  Chunks are int2 {tag, first row}; host and device derive a chunk's row
// count from the tag's x-extent, the fab's components and element size with tag_chunk_rows.
constexpr int kTagChunk1 = 64, kTagChunk1F = 256, kTagChunkN = 128;
__host__ __device__ inline int tag_chunk_rows(int ex, int ncomp, int esize = 8) {
  const int cells = ncomp == 1 ? (esize == 4 ? kTagChunk1F : kTagChunk1) : kTagChunkN;
  return ex >= cells ? 1 : cells / ex;
}

// A launch may cover the box tables of several independent solves (batched and served
// solves): each solve's table is one segment of the launch's row space.  norms and scales
// of a row live at index slot + DRow::solve.
struct Seg {
  const DRow* rows;
  long long row_begin;  // first launch row of this segment
  long long row_count;  // rows of this segment (0: the launch's row count)
  int nbox;
  int slot;
};
struct SegList {
  const Seg* segs;  // device array, used when n > 1
  Seg one;          // the segment when n == 1
  int n;
  int width;        // host hint: widest box x-extent (cells) in the launch, 0 = unknown; the
                    // launchers size the lane groups of narrow rows from it
};
inline SegList one_seg(const DRow* rows, int nbox, int slot = 0, int width = 0) {
  SegList L{};
  L.one.rows = rows;
  L.one.row_begin = 0;
  L.one.nbox = nbox;
  L.one.slot = slot;
  L.n = 1;
  L.width = width;
  return L;
}

// Copy tags of one fab (offsets relative to base) in a fill launch covering several fabs.
struct TagSeg {
  const DTag* tags;
  const int2* chunks;
  void* base;
  long long chunk_begin;
  int nchunks;
  int pad_;
};
struct TagList {
  const TagSeg* segs;
  TagSeg one;
  int n;
};

// Tiles of one solve's level in a fused-sweep launch covering several solves.
struct UnitSeg {
  const DRow* rows;
  const int4* units;  // {box, y0, z0, z1}
  long long unit_begin;
  int nunits;
  int pad_;
};
struct UnitList {
  const UnitSeg* segs;
  UnitSeg one;
  int n;
};

int num_sms();

// Raise a kernel's dynamic shared memory limit to at least smem on the current device (once
// per kernel, device and size; thread-safe).
cudaError_t opt_in_smem(const void* kernel, size_t smem);

// Process-wide count of kernels enqueued by the launchers below (plus graph kernel nodes
// per replay, added by the graph owner).
void count_launches(long long n);
long long launches_so_far();

// Programmatic dependent launch.  Every kernel of this library is launched through launch_k,
// which lets the GPU start launching it as the blocks of the kernel before it in the stream
// exit, and begins with pdl_begin(): wait until that kernel has completed and its writes are
// visible.  The stencil chains of a V-cycle are hundreds of dependent launches, many of them
// a few microseconds long on the coarse levels, so the launch latency would otherwise sit
// between every two of them.  No kernel triggers its dependents early: a trigger at kernel
// start (so that the next kernel's blocks wait on the SMs) made every measured solve slower
// (256^3 FP64 1.1%, 512^3 mixed 4%), while the implicit trigger at block exit gives the 64^3
// solve 5% and the 256^3 one 0.2% (GB300).  Results do not depend on it (the wait comes
// before any memory access); GBMG_NO_PDL=1 in the environment launches without the
// attribute.
bool pdl_enabled();
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
template <class... P, class... A>
inline void launch_k(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     A&&... a) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k, static_cast<A&&>(a)...);  // errors: cudaGetLastError()
}
#endif

cudaError_t launch_copy_tags(int dt, const DTag* tags, const int2* chunks, int nchunks,
                             void* base, int ncomp, cudaStream_t s);

// Stencil launchers: with direct = true the kernel reads box-face neighbours through
// DRow::nbd / nbf (rows whose nbd / nbf are zero read their ghost cells); with false it reads
// the ghost cells (filled beforehand) through plain offsets.
// v[0] = phi, v[1] = rhs.  norms != null (direct, single-table launches only): also atomicMax
// of |residual| of every updated cell after its update into norms[solve] (valid when the
// box array's periodic extents are even).  width: the widest box x-extent of the table
// (0 = unknown; any value gives the same results, it only picks the lanes per row).
// pre = true (needs norms): the norm is that of each updated cell's residual just before its
// update, and the values before the update are saved to v[2] (a one-colour view: cell x of
// row (y, z) at element x / 2 of that row; row pitch and plane of its own) so that
// launch_restore_colour can undo the half-sweep.
cudaError_t launch_rbgs_half(int dt, const DRow* rows, int nbox, long long nrows, int color,
                             cudaStream_t s, bool direct = false,
                             unsigned long long* norms = nullptr, int width = 0, bool pre = false);
// v[0] = phi, v[2] = saved values (one-colour view): cells of colour `color` take their
// saved values back.
cudaError_t launch_restore_colour(int dt, const DRow* rows, int nbox, long long nrows, int color,
                                  cudaStream_t s);

// v[0] = phi, v[1] = rhs, v[2] = r (p == null: not stored).  norms[solve] receives
// atomicMax of the bit pattern of |r| (NaN propagates as the largest pattern).  color < 0:
// every cell; 0 / 1: the cells of that colour only.
cudaError_t launch_residual(int dt, const DRow* rows, int nbox, long long nrows,
                            unsigned long long* norms, cudaStream_t s, bool direct = false,
                            int color = -1);

// Rows are coarse x-lines.  v[0] = phi, v[1] = rhs (fine); c[0] = coarse rhs,
// c[1] = coarse phi (p == null: not zeroed).  stored (FP64, direct): the fine cells of colour
// 1 take the residual in v[2] (one-colour view) that launch_rbgs_half_store left there.
cudaError_t launch_residual_restrict(int dt, const DRow* rows, int nbox, long long nrows,
                                     cudaStream_t s, bool direct = false, int width = 0,
                                     bool stored = false);
// FP64 half-sweep (direct reads, one table) that also stores, in v[2] (one-colour view), the
// residual of every cell it updates just after its update (the values a residual pass would
// compute next).
cudaError_t launch_rbgs_half_store(const DRow* rows, int nbox, long long nrows, int color,
                                   cudaStream_t s, int width);

// Rows are coarse x-lines.  v[0] = fine field; c[0] = coarse field.
cudaError_t launch_restrict(int dt, const DRow* rows, int nbox, long long nrows, cudaStream_t s);

// Rows are fine x-lines.  v[0] = fine field (+=); c[0] = coarse field.
cudaError_t launch_prolong_add(int dt, const DRow* rows, int nbox, long long nrows,
                               cudaStream_t s, int width = 0);
// The trilinear form (same rows); reads the coarse field's first ghost layer (filled).
cudaError_t launch_prolong_trilinear(int dt, const DRow* rows, int nbox, long long nrows,
                                     cudaStream_t s, int width = 0);

// Fused red + black sweep (see mg_fused.cu).  Rows: v[0] = source phi (2 ghost layers,
// filled), v[1] = rhs (1 ghost layer, filled), v[2] = destination phi with the source's
// layout; pad_ = Dirichlet-face flags (bit d: low face of dim d, bit 3+d: high face).
// units[i] = {box, y0, z0, z1}: rows [y0, y0+ty) x planes [z0, z1) of a box; depth = planes
// loaded ahead (1 to 3).  rhs_smem: rhs staged through shared memory too (else read from
// global memory).
size_t fused_smem_bytes(int dt, int ty, int max_pitch, int max_pitch_r, int depth, bool rhs_smem);
cudaError_t launch_rbgs_fused(int dt, const DRow* rows, const int4* units, int nunits, int ty,
                              int depth, int max_pitch, int max_pitch_r, bool rhs_smem, int* err,
                              cudaStream_t s);

cudaError_t launch_bottom(int dt, const BottomJob* jobs, int njobs, int maxN, cudaStream_t s);

// Shared memory of a coarse job whose levels have extents n[0..nlev); launch with the largest
// value over the jobs.
size_t coarse_smem_bytes(int dt, const int (*n)[3], int nlev);
constexpr size_t kCoarseSmemMax = 200 * 1024;
// Raises the kernel's shared-memory limit to smem (once; call outside stream capture).
cudaError_t coarse_opt_in(int dt, size_t smem);
cudaError_t launch_coarse_cycle(int dt, const CoarseJob* jobs, int njobs, size_t smem,
                                cudaStream_t s);

// v[0] += v[1] on valid cells.
cudaError_t launch_add_valid(int dt, const DRow* rows, int nbox, long long nrows, cudaStream_t s);

// v[0] = field: valid cells = value.
cudaError_t launch_set_valid(int dt, const DRow* rows, int nbox, long long nrows, double value,
                             cudaStream_t s);
// Whole allocation (ghosts and padding included) = value.
cudaError_t launch_set_flat(int dt, void* p, long long n, double value, cudaStream_t s);

// Dense domain array (ncomp, nz, ny, nx) <-> valid cells of a fab; v[0] = fab view (with
// cstride).  to_dense: 1 copies fab -> dense, 0 dense -> fab.
cudaError_t launch_dense_copy(int dt, const DRow* rows, int nbox, long long nrows, void* dense,
                              const int dom_lo[3], const int dom_n[3], int ncomp, int to_dense,
                              cudaStream_t s);

// max |value| over valid cells, atomicMax of bit patterns into norms[solve]; v[0] = field.
cudaError_t launch_maxabs(int dt, const DRow* rows, int nbox, long long nrows,
                          unsigned long long* norms, cudaStream_t s);

// Mixed precision.  v[0] = r (FP64 residual stored by the norm check), c[0] = r32 out,
// c[1] = e32 out (FP32 views with the same box geometry): r32 = float(r * 2^-e) with
// 2^e <= norms[solve] < 2^(e+1), e32 = 0.
cudaError_t launch_scale_residual_f32(const DRow* rows, int nbox, long long nrows,
                                      const unsigned long long* norms, cudaStream_t s,
                                      int width = 0);
// v[0] = phi (FP64), c[0] = e (FP32 view, same geometry): phi = phi + 2^e * double(e32) with
// the 2^e of the scale above.
cudaError_t launch_correct_add(const DRow* rows, int nbox, long long nrows,
                               const unsigned long long* norms, cudaStream_t s, int width = 0);

// Launchers over segment lists (several solves per launch); nrows / nchunks / nunits are
// the totals over all segments.
cudaError_t launch_copy_tags_l(int dt, const TagList& L, long long nchunks, int ncomp, cudaStream_t s);
cudaError_t launch_rbgs_half_l(int dt, const SegList& L, long long nrows, int color, cudaStream_t s,
                               bool direct = false, unsigned long long* norms = nullptr,
                               bool pre = false);
cudaError_t launch_residual_l(int dt, const SegList& L, long long nrows, unsigned long long* norms,
                              cudaStream_t s, bool direct = false, int color = -1);
cudaError_t launch_residual_restrict_l(int dt, const SegList& L, long long nrows, cudaStream_t s,
                                       bool direct = false, bool stored = false);
cudaError_t launch_prolong_add_l(int dt, const SegList& L, long long nrows, cudaStream_t s);
cudaError_t launch_prolong_trilinear_l(int dt, const SegList& L, long long nrows, cudaStream_t s);
cudaError_t launch_set_valid_l(int dt, const SegList& L, long long nrows, double value, cudaStream_t s);
// v[0] = a, v[1] = b, v[2] = c: a = fma(s, c, b) on valid cells.
cudaError_t launch_triad_l(int dt, const SegList& L, long long nrows, double s, cudaStream_t st);
// FP64 throughput probe: blocks x 256 threads, each running 8 independent chains of `iters`
// fused multiply-adds; *lane_ops = the FP64 lane operations issued.
cudaError_t launch_fp64_probe(int iters, long long* lane_ops, cudaStream_t s);
cudaError_t launch_maxabs_l(int dt, const SegList& L, long long nrows, unsigned long long* norms,
                            cudaStream_t s);
cudaError_t launch_scale_residual_f32_l(const SegList& L, long long nrows,
                                        const unsigned long long* norms, cudaStream_t s);
cudaError_t launch_correct_add_l(const SegList& L, long long nrows, const unsigned long long* norms,
                                 cudaStream_t s);
cudaError_t launch_rbgs_fused_l(int dt, const UnitList& L, long long nunits, int ty, int depth,
                                int max_pitch, int max_pitch_r, bool rhs_smem, int* err,
                                cudaStream_t s);

}  // namespace gbmg
