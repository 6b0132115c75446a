/*
 * gbmg.h -- C ABI of the GB300 (sm_103a) cell-centered geometric-multigrid Poisson library.
 *
 * The library implements, on one GPU, the data-parallel mesh path of the block-structured
 * framework reviewed in "AMReX and pyAMReX: Looking beyond the exascale computing project"
 * (arXiv 2403.12179): a single-level union of boxes (Sec. 2: Box, FArrayBox, MultiFab),
 * ghost-cell exchange between boxes and across periodic / Dirichlet faces (Sec. 2 cached
 * communication patterns; Sec. 3.5 fused pack/unpack), one kernel launch over all boxes of
 * a level (Sec. 3.2 kernel fusing), fused reductions (Sec. 3.4), a stream-ordered memory
 * pool (Sec. 3.7) and zero-copy device views (Sec. 4.1), driving a V-cycle solve of the
 * 7-point Poisson problem (Sec. 2: "linear solvers for cell-centered ... data").
 *
 * Conventions shared by every entry point:
 *  - Return value: MG_OK (0) on success, a negative MG_E* code on failure (the message is
 *    then available from mg_last_error() in the calling thread), or MG_PENDING (1) where
 *    stated.  No C++ exception crosses this boundary.
 *  - Indices are global cell indices; boxes are inclusive [lo, hi] triples (x, y, z).
 *    Arrays of boxes are int[6*nbox] laid out lo0 lo1 lo2 hi0 hi1 hi2 per box.
 *  - Dense domain arrays are (ncomp, nz, ny, nx), x fastest, covering the domain exactly.
 *  - Fab storage per box: x fastest, then y, z, component (Fortran order, Sec. 4.1), each
 *    row padded to a multiple of 16 bytes, ghosts included; see mg_fab_ptr.
 *  - `stream` arguments are cudaStream_t values passed as void* (NULL = legacy default
 *    stream).  Calls that take a stream are asynchronous on it unless stated otherwise.
 *  - A context may be used from one host thread at a time, except mg_poll / mg_submit which
 *    are safe to call from any thread.
 *  - The PDE is  lap(phi) = rhs  with the 7-point operator
 *    (A phi)_c = (sum of the 6 neighbours - 6 phi_c) / h^2.
 */
#ifndef GBMG_H
#define GBMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_ctx* mg_ctx_t;
typedef int64_t mg_ba_t;     /* box-array handle (> 0) */
typedef int64_t mg_fab_t;    /* fab handle (> 0) */
typedef int64_t mg_ticket_t; /* serving ticket (> 0) */

enum {
  MG_OK = 0,
  MG_PENDING = 1,         /* mg_poll: the solve has not finished */
  MG_EINVAL = -1,         /* bad argument or unsupported configuration */
  MG_ENOMEM = -2,         /* the context's memory pool cannot hold the request */
  MG_EAGAIN = -3,         /* serving queue full; retry later */
  MG_NOT_CONVERGED = -4,  /* max_iter V-cycles without reaching tol */
  MG_ETIMEDOUT = -5,      /* mg_poll timeout, or a device-side bounded wait gave up */
  MG_ECUDA = -6,          /* a CUDA runtime call failed */
  MG_ENAN = -7            /* the residual norm became NaN or Inf */
};

enum { MG_F64 = 0, MG_F32 = 1 };                    /* fab element types */
enum { MG_BC_PERIODIC = 0, MG_BC_DIRICHLET0 = 1 };  /* face kinds */
enum { MG_PREC_F64 = 0, MG_PREC_MIXED = 1 };        /* solver precision */
enum { MG_SMOOTH_AUTO = 0, MG_SMOOTH_HALF = 1, MG_SMOOTH_FUSED = 2 };
enum { MG_SMOOTH_DIRECT_READS = 4 };  /* flag for mg_smooth's color (see there) */
enum { MG_PROLONG_CONSTANT = 0, MG_PROLONG_TRILINEAR = 1 };  /* prolongation forms */

/* Boundary conditions: kind[d][0] / kind[d][1] for the low / high face of dimension d.
 * A periodic dimension must be periodic on both faces.  MG_BC_DIRICHLET0 is homogeneous
 * Dirichlet with the face half way between the boundary cell and its ghost:
 * ghost = -(mirror cell across the face). */
typedef struct {
  int kind[3][2];
} mg_bc;

/* Solver options; pass NULL for the defaults shown. */
typedef struct {
  int nu1;            /* pre-smoothing sweeps (red + black), default 2 */
  int nu2;            /* post-smoothing sweeps, default 2 */
  int max_iter;       /* V-cycle limit, default 50 */
  int precision;      /* MG_PREC_F64 (default) or MG_PREC_MIXED */
  int smoother;       /* MG_SMOOTH_AUTO (default): the fused red + black sweep on FP32 levels
                         of at least 256^3 cells, half-sweeps elsewhere; _HALF: half-sweeps
                         everywhere; _FUSED: the fused sweep on every level but the bottom
                         (the caller's FP64 level 0 then needs phi nghost >= 2, rhs >= 1).
                         All three give the same results. */
  int use_graph;      /* 1 (default): replay each V-cycle as a CUDA graph */
  int fixed_vcycles;  /* >= 0: run exactly this many V-cycles, no stop test; -1 default */
  double h;           /* cell size; 0 (default) means 1 / (domain x extent) */
  int coarse_cells;   /* the levels from the first one with at most this many cells down to
                         the bottom run as ONE launch per V-cycle (one CTA per solve, levels
                         held in shared memory; same arithmetic, bit-identical results).
                         0 (default): 512 for FP64 levels, 4096 for FP32 levels; -1: off */
  int direct_reads;   /* 1 (default): on levels whose boxes form a regular grid, the
                         smoother, residual and residual+restriction read the neighbouring
                         boxes (or the periodic image, or the negated boundary cell across a
                         Dirichlet face) directly instead of first filling one ghost layer:
                         the same values, without the fill launches.  0: always fill. */
  int prolong;        /* MG_PROLONG_CONSTANT (default): piecewise-constant injection;
                         MG_PROLONG_TRILINEAR: per dimension 3/4 parent + 1/4 neighbour
                         towards the fine cell (x, then y, then z), from the coarse level's
                         filled first ghost layer.  Trilinear runs every level as separate
                         launches (coarse_cells is ignored).  With the 8-cell-average
                         restriction it does not converge faster than injection. */
  int inner_cycles;   /* MG_PREC_MIXED: FP32 V-cycles on the scaled residual per outer FP64
                         iteration (1 to 8; 0 = default 2).  Each outer iteration then gains
                         about the contraction of that many V-cycles, at one FP64 residual
                         pass, one scaling and one correction; `vcycles` in mg_result counts
                         outer iterations. */
} mg_options;

typedef struct {
  int status;        /* MG_OK, MG_NOT_CONVERGED, MG_ENAN, ... */
  int vcycles;       /* V-cycles (outer iterations for MG_PREC_MIXED) performed */
  double rel_resid;  /* ||rhs - A phi||_inf / ||rhs||_inf at exit */
  double seconds;    /* t_end - t_start: for served solves the latency submit -> done */
  double t_admit;    /* serving: seconds since context creation at admission (else 0) */
  double t_start;    /* seconds since context creation when the call started (served:
                        when mg_submit queued the request) */
  double t_end;      /* seconds since context creation at completion */
} mg_result;

/* ---- context --------------------------------------------------------------------------- */

/* Create a context on CUDA device `device`, with a stream-ordered device memory pool capped
 * at pool_bytes (0: 90% of the device memory free at creation).  device = -1 creates a
 * host-only context on which box arrays, hierarchies and copy tags can be built and
 * inspected but no fab can be allocated (used for planning and host-side tests).
 * Errors: MG_EINVAL (bad device), MG_ECUDA. */
int mg_init(int device, size_t pool_bytes, mg_ctx_t* out);

/* Wait for all work of the context, free every fab, box array and cached plan, destroy the
 * pool.  The context pointer is invalid afterwards. */
int mg_finalize(mg_ctx_t ctx);

/* Message of the last failing call made by this thread ("" if none).  Owned by the library,
 * valid until the thread's next call. */
const char* mg_last_error(void);

/* Library ABI version (increases on incompatible changes). */
int mg_version(void);

/* Stream used by mg_solve / mg_solve_batch (default: a stream the context creates). */
int mg_set_stream(mg_ctx_t ctx, void* stream);

/* Memory pool of the context (Sec. 3.7 arena): its cap and the bytes currently allocated
 * from it (fabs, coarse levels, tables, scratch).  Either pointer may be NULL. */
int mg_pool_info(mg_ctx_t ctx, size_t* cap, size_t* in_use);

/* Instrumentation (no counterpart in the paper): number of kernels this process has
 * enqueued through the library so far, counting each kernel node of a replayed CUDA graph
 * once per replay.  Process-wide, monotonic. */
int mg_kernel_launches(int64_t* n);

/* ---- box arrays (Sec. 2: Box, BoxArray / MultiFab layout) --------------------------- */

/* Chop the domain [dom_lo, dom_hi] into boxes of edge <= max_box per dimension: pieces of
 * max_box starting at dom_lo, the remainder last; boxes ordered x fastest.
 * Errors: MG_EINVAL (empty domain, max_box < 1). */
int mg_box_array_create(mg_ctx_t ctx, const int dom_lo[3], const int dom_hi[3],
                        const int max_box[3], mg_ba_t* out);

/* Box array from an explicit list of boxes (int[6*nbox]) that must be disjoint and cover
 * the domain exactly.  Errors: MG_EINVAL (overlap, gap, box outside the domain). */
int mg_box_array_from_list(mg_ctx_t ctx, const int dom_lo[3], const int dom_hi[3], int nbox,
                           const int* lo_hi, mg_ba_t* out);

/* Box count, domain (int[6], nullable) and boxes (int[6*nbox], nullable). */
int mg_box_array_info(mg_ctx_t ctx, mg_ba_t ba, int* nbox, int* dom_lohi, int* lo_hi);

int mg_box_array_free(mg_ctx_t ctx, mg_ba_t ba);

/* ---- multigrid hierarchy (host planning; works on a host-only context) ---------------- */

/* Level count of the hierarchy built from `ba`: level l+1 exists while every domain edge
 * of level l is even and >= 4 (and the domain lo is even); its boxes are the level-l boxes
 * coarsened by 2, or one box covering the coarse domain when some level-l box has odd
 * bounds or would coarsen to an edge below 2.  The last level is solved exactly and must
 * hold at most 1024 cells.  Errors: MG_EINVAL (bottom too large). */
int mg_hierarchy_levels(mg_ctx_t ctx, mg_ba_t ba, int* nlevels);

/* Box array handle for level `level` of the hierarchy of `ba` (a new handle owned by the
 * context; free with mg_box_array_free). */
int mg_hierarchy_level(mg_ctx_t ctx, mg_ba_t ba, int level, mg_ba_t* out);

/* Copy tags of a ghost fill (Sec. 2 cached communication pattern), for inspection: tag t
 * occupies 16 ints = {src_box, dst_box, src_first[3], dst_lo[3], src_dir[3], extent[3],
 * sign, 0}.  Destination cells dst_lo + (i, j, k), 0 <= i,j,k < extent, take
 * sign * value(src_box, src_first + src_dir * (i, j, k)); sign 0 means "set to 0".
 * If cap is too small, *ntags is set and MG_EINVAL returned. */
int mg_copy_tags(mg_ctx_t ctx, mg_ba_t ba, const mg_bc* bc, int nghost, int64_t cap,
                 int* tags, int64_t* ntags);

/* Closed-form (pseudo-)inverse of the 7-point operator on an n[0] x n[1] x n[2] box with
 * the given per-dimension periodicity (others homogeneous Dirichlet), cell size h, ordered
 * x fastest: M[i*N + j], N = n0*n1*n2 <= 1024.  Host only.  Errors: MG_EINVAL. */
int mg_bottom_matrix(const int n[3], const int periodic[3], double h, double* M);

/* ---- fabs (Sec. 2 FArrayBox / MultiFab; Sec. 3.7 arena; Sec. 4.1 zero-copy) -------- */

/* Bytes a fab of this shape needs (for mg_fab_wrap). */
int mg_fab_layout(mg_ctx_t ctx, mg_ba_t ba, int ncomp, int nghost, int dtype, size_t* bytes);

/* Allocate a fab (all boxes of the box array in one pool allocation, 256-byte aligned per
 * box), zero-filled, on the context stream.  Errors: MG_ENOMEM, MG_EINVAL. */
int mg_fab_alloc(mg_ctx_t ctx, mg_ba_t ba, int ncomp, int nghost, int dtype, mg_fab_t* out);

/* Wrap caller-owned device memory (e.g. a torch tensor of mg_fab_layout bytes, 256-byte
 * aligned) as a fab.  The library never frees it; the caller keeps it alive until
 * mg_fab_free of the handle has been called. */
int mg_fab_wrap(mg_ctx_t ctx, mg_ba_t ba, int ncomp, int nghost, int dtype, void* dptr,
                size_t bytes, mg_fab_t* out);

/* Zero-copy view of box `box`: *dptr = address of cell (lo - g) component 0, strides in
 * elements for (x, y, z, component) -- x stride is 1. */
int mg_fab_ptr(mg_ctx_t ctx, mg_fab_t fab, int box, void** dptr, int64_t strides[4]);

/* Shape of a fab: its box array, ncomp, nghost, dtype (any pointer may be NULL). */
int mg_fab_info(mg_ctx_t ctx, mg_fab_t fab, mg_ba_t* ba, int* ncomp, int* nghost, int* dtype);

/* Release a fab in stream order (Sec. 3.7 async-safe arena): the memory returns to the
 * pool after all work already queued on `stream` (and the context stream) completes. */
int mg_fab_free(mg_ctx_t ctx, mg_fab_t fab, void* stream);

/* Copy a dense domain array (ncomp, nz, ny, nx) of the fab's type into the valid cells
 * (src_on_host: 1 = host memory, pinned or pageable; 0 = device memory), or back out. */
int mg_fab_copy_from_dense(mg_ctx_t ctx, mg_fab_t fab, const void* src, int src_on_host,
                           void* stream);
int mg_fab_copy_to_dense(mg_ctx_t ctx, mg_fab_t fab, void* dst, int dst_on_host, void* stream);

/* Set every cell (include_ghosts = 1) or every valid cell to v. */
int mg_fab_set_val(mg_ctx_t ctx, mg_fab_t fab, double v, int include_ghosts, void* stream);

/* ---- level operations (Sec. 3.2: one launch over all boxes of a level) -------------- */

/* Ghost-cell exchange (Sec. 2; Sec. 3.5 fused pack/unpack): one kernel over the cached
 * copy-tag list fills every ghost cell (all 26 directions, nghost layers, all components):
 * from the box owning its periodically wrapped position, else -(mirror cell) across a
 * Dirichlet face, else (outside the domain across two or more Dirichlet directions) 0. */
int mg_fill_boundary(mg_ctx_t ctx, mg_fab_t fab, const mg_bc* bc, void* stream);

/* The same ghost fill with one launch per copy tag (Sec. 3.2's unfused form, kept as the
 * baseline the fused launch is measured against); same results. */
int mg_fill_boundary_unfused(mg_ctx_t ctx, mg_fab_t fab, const mg_bc* bc, void* stream);

/* Red-black Gauss-Seidel on 1-component fabs of one box array with cell size h.
 * color 0 / 1: one half-sweep of that colour ((i+j+k) mod 2 on global indices), using
 *   phi's ghosts as they are (fill them first); rhs needs no ghosts.
 * color 0 / 1 | MG_SMOOTH_DIRECT_READS: the same half-sweep reading each box's neighbours
 *   (periodic images; the negated boundary cell across a Dirichlet face) directly instead of
 *   ghost cells, as the solver does; boxes must form a regular grid and periodic extents
 *   must be even (else MG_EINVAL: an odd periodic extent makes a cell's periodic image one of
 *   its own colour).
 * color 2: one full sweep, equal to fill, red, fill, black; with phi nghost >= 2 and rhs
 *   nghost >= 1 it runs as one fused kernel after one fill of each.
 * Update: phi_c = (s - h^2 rhs_c) / 6, s = x- + x+ + y- + y+ + z- + z+ (in that order). */
int mg_smooth(mg_ctx_t ctx, mg_fab_t phi, mg_fab_t rhs, const mg_bc* bc, double h, int color,
              void* stream);

/* One fused red + black sweep from phi_src into phi_dst (a second fab with the same box
 * array and layout), equal bit for bit to fill, red, fill, black on phi_src: phi_src needs
 * nghost >= 2 and rhs nghost >= 1, both with ghosts already filled (mg_fill_boundary).
 * One launch streams z-planes of every (box, y-tile) through shared memory with TMA bulk
 * copies.  phi_dst's ghost cells are left stale.  Errors: MG_EINVAL (layout). */
int mg_smooth_fused(mg_ctx_t ctx, mg_fab_t phi_src, mg_fab_t rhs, mg_fab_t phi_dst,
                    const mg_bc* bc, double h, void* stream);

/* Residual r = rhs - (s - 6 phi) / h^2 (computed as (s - 6 phi) * (1/h^2)) on valid cells,
 * into r (or not stored if r == 0), and its max-norm (Sec. 3.4 fused reduction) into
 * *norm if non-NULL (this synchronises the stream).  phi's ghosts are used as they are. */
int mg_residual(mg_ctx_t ctx, mg_fab_t phi, mg_fab_t rhs, mg_fab_t r, double h, double* norm,
                void* stream);

/* Fused residual + restriction: crhs(I) = (sum of the residuals of the 8 children, x
 * fastest) * 1/8 and cphi(I) = 0 on valid coarse cells.  cphi may be 0.  The coarse box
 * array must be level 1 of the fine box array's hierarchy. */
int mg_residual_restrict(mg_ctx_t ctx, mg_fab_t phi, mg_fab_t rhs, mg_fab_t crhs,
                         mg_fab_t cphi, double h, void* stream);

/* Plain restriction: coarse(I) = (sum of the 8 children, x fastest) * 1/8. */
int mg_restrict(mg_ctx_t ctx, mg_fab_t fine, mg_fab_t coarse, void* stream);

/* Piecewise-constant prolongation added to the fine field: fine(c) += coarse(floor(c/2)). */
int mg_prolong_add(mg_ctx_t ctx, mg_fab_t coarse, mg_fab_t fine, void* stream);

/* Trilinear prolongation added to the fine field (the MG_PROLONG_TRILINEAR form of
 * mg_options): per dimension 3/4 of the parent plus 1/4 of the parent's neighbour on the fine
 * cell's side, dimension by dimension (x, y, z), each step fma(1/4, b, 3/4 * a).  coarse needs
 * one ghost layer, filled beforehand (mg_fill_boundary); MG_EINVAL without ghosts. */
int mg_prolong_add_trilinear(mg_ctx_t ctx, mg_fab_t coarse, mg_fab_t fine, void* stream);

/* Exact bottom solve on a box array of at most 1024 cells: phi = M rhs with M from
 * mg_bottom_matrix (FP64 arithmetic for either fab type). */
int mg_bottom_solve(mg_ctx_t ctx, mg_fab_t rhs, mg_fab_t phi, const mg_bc* bc, double h,
                    void* stream);

/* Residual max-norm that allocates nothing (the paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- code running under a frozen
 * memory budget, inside a framework that owns every device allocation, or where an
 * allocation could stall other streams).  It computes the same value as mg_residual's norm,
 * max |rhs - A phi| over valid cells, without a context or fab handles: the caller passes
 * the box array (domain and int[6*nbox] boxes) and the device base addresses of two FP64,
 * 1-component buffers laid out exactly as mg_fab_layout describes for that box array with
 * phi_nghost (>= 1) and rhs_nghost ghost layers; phi's ghost cells are used as they are.
 * h <= 0 means 1 / (domain x extent).  The norm is written to the host double *norm; the
 * call synchronises `stream`.
 * Scratch: a file-scope device array of 1024 box-table rows plus an 8-byte accumulator
 * (278,784 bytes), held by every GPU that loads the library until the process exits; no
 * cudaMalloc, cudaFree or pool allocation happens in this call.  At most 1024 boxes
 * (MG_EINVAL beyond).  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and caches it for the life of the
 * process (after cudaDeviceReset the library must be loaded again); make that first call
 * before any stream capture.  `stream` must belong to the current device (MG_EINVAL
 * otherwise).  Every call shares the array and it keeps the last call's contents (the
 * accumulator is cleared at the start of each call).  Calls from one process are
 * serialised: each holds a process-wide lock until it has synchronised `stream`, so they do
 * not overlap on the GPU; work that reached the array any other way while a call runs
 * would race with it. */
int mg_residual_norm_noalloc(const int dom_lo[3], const int dom_hi[3], int nbox, const int* lo_hi,
                             const double* phi, int phi_nghost, const double* rhs, int rhs_nghost,
                             double h, double* norm, void* stream);

/* ---- solves --------------------------------------------------------------------------- */

/* Synchronous V(nu1,nu2) solve of lap(phi) = rhs (Sec. 2: the framework's linear solvers
 * for cell-centered data; the paper names them without their numerics, so the cycle is the
 * reading stated at the top of this file and in mg_options: red-black Gauss-Seidel,
 * residual restriction by 8-cell means, injection, exact bottom solve) on FP64 fabs with 1
 * component and the same box array (phi is the initial guess and the result).  Each stage
 * is one launch over all boxes of a level (Sec. 3.2); the cycle is replayed as a CUDA
 * graph.  Stops when ||rhs - A phi||_inf <=
 * tol ||rhs||_inf (checked before each V-cycle), or after max_iter V-cycles
 * (MG_NOT_CONVERGED).  rhs == 0 gives phi = 0.  With fully periodic faces rhs must have
 * zero mean (to within tol).  The coarse levels are allocated on first use and cached per
 * (box array, bc, options) until mg_finalize.  Returns res->status. */
int mg_solve(mg_ctx_t ctx, mg_fab_t rhs, mg_fab_t phi, const mg_bc* bc, double tol,
             const mg_options* opt, mg_result* res);

/* Synchronous solve of n independent problems whose boxes are packed into one box table
 * per V-cycle stage (one launch per stage for all problems: Sec. 3.2's fused launch over
 * many boxes, extended across solves; each solve is mg_solve's cycle, Sec. 2).  Each problem converges and
 * retires on its own; res[i] receives its result.  Returns MG_OK if every solve did. */
int mg_solve_batch(mg_ctx_t ctx, int n, const mg_fab_t* rhs, const mg_fab_t* phi,
                   const mg_bc* bcs, double tol, const mg_options* opt, mg_result* res);

/* ---- serving (continuous batching; no counterpart in the paper) ---------------------- */

/* Queue a solve for the context's scheduler thread (started on the first call), which
 * admits requests in arrival order while a slot is free and the context pool can hold their
 * coarse levels, runs the V-cycles of all admitted solves in shared launches (one launch per
 * stage for the whole mix), retires each solve when it converges and releases its coarse
 * levels in stream order.  A request that cannot fit even into an empty pool completes with
 * MG_ENOMEM.  rhs / phi must stay allocated, and untouched by other calls, until mg_poll
 * reports completion; while requests are in flight the context's stream belongs to the
 * scheduler (use another context for synchronous solves).  Errors: MG_EAGAIN (queue full),
 * MG_EINVAL. */
int mg_submit(mg_ctx_t ctx, mg_fab_t rhs, mg_fab_t phi, const mg_bc* bc, double tol,
              const mg_options* opt, mg_ticket_t* out);

/* Queue a solve whose data lives in host memory (no counterpart in the paper): the domain
 * [dom_lo, dom_hi] chopped into boxes of edge <= max_box (as mg_box_array_create), rhs a
 * dense FP64 array (nz, ny, nx), x fastest, and phi a dense FP64 array of the same shape that
 * receives the answer (and holds the initial guess if phi_is_guess is 1; else the guess is
 * 0).  At admission the scheduler allocates the request's fine-level fabs (rhs with one ghost
 * layer, phi with two) from the context pool together with its coarse levels -- a request
 * waits in the queue until the pool can hold all of it -- and copies rhs in; at completion
 * it copies phi out and releases everything in stream order.  The result's latency
 * (mg_result.seconds, submit -> done) therefore includes both copies.  Pinned host memory
 * (cudaHostAlloc) lets the copies run at full speed; rhs and phi must stay valid and
 * untouched until mg_poll reports completion.  With phi_is_guess = 0, phi may be the rhs
 * array itself (rhs is copied in before phi is written).  Otherwise as mg_submit: FP64 or mixed
 * precision per opt, results bit-identical to mg_solve on the same data.
 * When a host-memory request completes, its workspace (fine-level fabs and level hierarchy)
 * stays resident for the next request of the same shape (box array, faces and options),
 * which is then admitted without any planning; idle workspaces are released, oldest first,
 * when the pool needs room for another request, and all at once by mg_server_trim.
 * Errors: MG_EINVAL (bad domain, box size or options), MG_EAGAIN (queue full). */
int mg_submit_host(mg_ctx_t ctx, const int dom_lo[3], const int dom_hi[3], const int max_box[3],
                   const mg_bc* bc, const double* rhs, double* phi, int phi_is_guess, double tol,
                   const mg_options* opt, mg_ticket_t* out);

/* Release the scheduler's idle host-memory workspaces (see mg_submit_host) in stream order;
 * returns once they are gone.  Workspaces in use are not touched. */
int mg_server_trim(mg_ctx_t ctx);

/* Serving statistics since the scheduler started (no counterpart in the paper). */
typedef struct {
  int64_t submitted, admitted, completed, steps;
  int64_t max_active;        /* largest number of solves in flight at once */
  double admit_seconds;      /* host time building hierarchies of admitted requests */
  double plan_seconds;       /* host time building and uploading per-step launch lists */
  double step_seconds;       /* time from a step's first launch to its norms on the host */
  double retire_seconds;     /* host time releasing finished solves */
} mg_server_stats;
int mg_server_stats_get(mg_ctx_t ctx, mg_server_stats* out);

/* Wait up to timeout_ms (0: do not wait, -1: forever) for a ticket.  Returns MG_OK with
 * *res filled when done (the ticket is then released), MG_PENDING if not done in time,
 * MG_EINVAL for an unknown ticket. */
int mg_poll(mg_ctx_t ctx, mg_ticket_t ticket, int timeout_ms, mg_result* res);

/* ---- two-level AMR composite solve (Sec. 1, Sec. 2: AMR hierarchy, inter-level ops) ---- */

/* Composite Poisson problem on two levels (refinement ratio 2): level 0 (fabs rhs0 / phi0 on
 * a box array over the domain [0, n0), any faces from bc) and level 1 (rhs1 / phi1 on a box
 * array whose domain is a coarse box region [A, B) refined by 2, i.e. fine cells [2A, 2B),
 * with A >= 1 and B <= n0 - 1 in every dimension and even box bounds).  Unknowns are the fine
 * cells and the coarse cells outside the region; the paper gives no coarse/fine
 * discretisation, so the one here is this library's reading:
 *  - fine cells: the 7-point operator with h1 = h0 / 2; a neighbour across the coarse/fine
 *    boundary is the ghost value g = 8/15 c + 2/3 f1 - 1/5 f2, where f1, f2 are the first two
 *    fine cells inside along the normal and c is the quadratic interpolation, over the 3 x 3
 *    coarse cells of the layer just outside the region, at the ghost's tangential position
 *    (3-point Lagrange weights at offset -1/4 or +1/4 coarse cells, lower-numbered tangential
 *    dimension first);
 *  - uncovered coarse cells: the 7-point operator with h0, except that the flux through a face
 *    shared with the region is the mean of the four fine fluxes (phi_f - g_f) / h1 through it
 *    (flux matching: the composite operator is conservative);
 *  - covered coarse cells are not unknowns; on return they hold the mean of their 8 children.
 * h0 = opt->h, or 1 / n0[0].  FP64 fabs, 1 component, phi0 and phi1 with >= 1 ghost layer.
 * The iteration (stop test ||f - A phi||_inf <= tol ||f||_inf before each, over fine and
 * uncovered coarse cells): one V(nu1, nu2) cycle of the single-level solver on level 0 for the
 * composite residual (covered cells: the mean of the fine residual), added to phi0 and, by
 * injection, to phi1; then nu1 + nu2 red-black sweeps on level 1 with the coarse/fine ghosts
 * refreshed before each colour; then the covered coarse cells take their children's mean.
 * res->vcycles counts these iterations.  Tables and work fabs are built on first use and
 * cached per (fabs, bc, options) until one of the fabs is freed.  Returns res->status. */
int mg_amr2_solve(mg_ctx_t ctx, mg_fab_t rhs0, mg_fab_t phi0, mg_fab_t rhs1, mg_fab_t phi1,
                  const mg_bc* bc, double tol, const mg_options* opt, mg_result* res);

/* The composite residual of mg_amr2_solve's problem at the current phi (after the covered
 * coarse cells of phi0 take the mean of their children): r0 (a level-0 fab without ghosts,
 * covered cells: the mean of the fine residual) and r1 (level 1, no ghosts), either may be 0;
 * its max-norm over fine and uncovered coarse cells into *norm (if non-NULL).  h <= 0: 1 / n0[0].
 * Synchronous. */
int mg_amr2_residual(mg_ctx_t ctx, mg_fab_t rhs0, mg_fab_t phi0, mg_fab_t rhs1, mg_fab_t phi1,
                     const mg_bc* bc, double h, mg_fab_t r0, mg_fab_t r1, double* norm);

/* ---- calibration (Sec. 3.1-3.2 STREAM triad; FP64 rate) ------------------------------ */

/* STREAM triad a = b + s c (computed as one fma per cell) on the valid cells of three
 * one-component fabs of one box array and type: the bandwidth example of Sec. 3.1, launched
 * either as ONE kernel over all boxes (per_box = 0, the fused launch of Sec. 3.2) or as one
 * launch per box (per_box = 1, Sec. 3.2's unfused form).  Asynchronous on `stream`.
 * Algorithmic traffic: 3 element sizes per cell.  Errors: MG_EINVAL (shapes differ). */
int mg_triad(mg_ctx_t ctx, mg_fab_t a, mg_fab_t b, mg_fab_t c, double s, int per_box,
             void* stream);

/* FP64 rate probe (no counterpart in the paper): enqueues on `stream` (current device) one
 * kernel of independent FP64 fused multiply-add chains, iters steps each, and returns the
 * FP64 lane operations it issues in *lane_ops; timing it gives the device's FP64 issue rate,
 * the ceiling of the FP64 stencil kernels.  Errors: MG_EINVAL (iters < 1). */
int mg_calib_fp64(void* stream, int iters, int64_t* lane_ops);

/* ---- instrumentation (no counterpart in the paper) ---------------------------------- */

/* Device time of the finest-level red-black half-sweep inside mg_solve: while enabled, each
 * V-cycle of an FP64 solve (finest level smoothed by half-sweeps) records a CUDA event pair on
 * the solve stream around its first finest-level half-sweep (captured into the step graph).
 * Returns in *total_ms / *launches (either may be NULL) the sum and count accumulated since
 * the previous call, resets them, and sets the mode for later solves. */
int mg_sweep_timing(mg_ctx_t ctx, int enable, double* total_ms, int64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* GBMG_H */
