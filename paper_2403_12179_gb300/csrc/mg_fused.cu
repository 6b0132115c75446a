// Fused red + black Gauss-Seidel sweep for sm_103a (one launch = one full sweep of a level).
//
// Equivalent, bit for bit, to: fill ghosts, red half-sweep, fill ghosts, black half-sweep.
// The source phi has 2 ghost layers and rhs 1, both filled beforehand.  A CTA owns one
// (box, y-tile) and streams its z-planes through shared memory:
//   * TMA bulk copies (cp.async.bulk, one per plane) bring phi rows [y0-2, y0+TY+2) and rhs
//     rows [y0-1, y0+TY+1) of each plane into a ring of shared-memory buffers, completing on
//     mbarriers; a producer lane issues each load as soon as its slot is free, D planes
//     beyond the ones in use;
//   * a CTA owns planes [z0, z1) of its tile; in stages z0-1 .. z1 the consumer warps
//     red-update plane s over the tile plus a one-cell ring (the ring cells belong
//     to neighbouring tiles / boxes / periodic images and are recomputed redundantly from the
//     second ghost layer -- exactly the values their owners compute; planes z0-1 and z1 are
//     recomputed the same way under the tile only) and black-update plane s-1;
//   * the producer stores the finished plane s-1 to global memory by one bulk copy of whole
//     rows into the destination buffer (a second phi allocation: tiles read each other's
//     rows as halos, so the sweep cannot be done in place).
// Ghost cells outside the domain (Dirichlet faces) are never updated: a boundary cell's
// ghost equals -(its own value before this half-sweep), which the fill already holds for
// every cell that the half-sweep updates.
//
// Every mbarrier wait is bounded; on expiry the CTA records an error code, the producer
// drains its outstanding copies (again bounded) and every thread returns.
#include <cuda_runtime.h>

#include <cstdint>

#include "mg_kernels.hpp"

namespace gbmg {

namespace {

template <class T>
struct Ar;
template <>
struct Ar<double> {
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};
template <>
struct Ar<float> {
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};

// phi = fma(-h^2, rhs, s) * (1/6); mh2 = -h^2
template <class T>
__device__ __forceinline__ T gs_update(T s, T rhs, T mh2) {
  constexpr T inv6 = T(1) / T(6);
  return Ar<T>::mul(Ar<T>::fma(mh2, rhs, s), inv6);
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// One try_wait that may suspend the thread for up to ~2 us while the phase is pending.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(2000u)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_addr(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // a wait this long is stuck

// Bounded wait on one phase of an mbarrier.  Returns false after kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (global_ns() - t0 < kWaitLimitNs)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

template <class T>
struct Sweep {
  // per-CTA constants
  const DRow* R;
  int y0, ty;            // tile rows [y0, y0+ty)
  int nx, ny, nz;
  int pitch, pr;         // phi / rhs pitches (elements)
  int g, gr;             // ghost widths
  long long plane, planer;
  int flags;             // bit d: low face of dim d is a Dirichlet domain face; bit 3+d: high
  uint32_t pbytes, rbytes;
  T mh2;  // -h^2
  int lox, loy, loz;
};

}  // namespace

// Shared memory: NP phi buffers, NR rhs buffers, then NP + NR + kStageBars mbarriers.
__device__ __forceinline__ int find_unitseg(const UnitSeg* __restrict__ segs, int n, long long u) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (segs[mid].unit_begin <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Roles: warps 0..7 (kConsumers threads) update cells; warp 8 lane 0 is the producer, which
// queues every TMA load as soon as its ring slot is free and stores each finished plane.
// Consumers wait on the load mbarriers themselves and sync with one named barrier per stage;
// consumer thread 0 then arrives on the stage's completion mbarrier (stage s on
// stage_bar[s % kStageBars], so the producer may lag kStageBars - 1 stages without
// confusing phases).
constexpr int kConsumers = 256;
constexpr int kFusedThreads = kConsumers + 32;
constexpr int kStageBars = 8;

// Named barrier 1 over the consumers; returns the OR of every consumer's flag, the same
// value in every consumer.
__device__ __forceinline__ bool consumer_sync_or(bool flag) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)flag), "n"(kConsumers)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// RS: rhs staged through shared memory by TMA like phi; else read from global memory (each
// rhs value is read once per sweep, so staging buys no reuse -- it only costs shared memory).
template <class T, int D, bool RS>
__global__ void __launch_bounds__(kFusedThreads) k_rbgs_fused(UnitList L, int ty_max,
                                                              unsigned phi_buf_elems,
                                                              unsigned rhs_buf_elems,
                                                              int* __restrict__ err) {
  pdl_begin();
  constexpr int NP = 4 + D;  // live phi planes s-2..s+1 plus D in flight
  constexpr int NR = RS ? 2 + D : 0;  // live rhs planes s-1, s plus D in flight
  extern __shared__ __align__(128) unsigned char smem[];
  T* pbuf = (T*)smem;
  T* rbuf = pbuf + (size_t)NP * phi_buf_elems;
  uint64_t* bars = (uint64_t*)(rbuf + (size_t)NR * rhs_buf_elems);
  uint64_t* pbar = bars;
  uint64_t* rbar = bars + NP;
  uint64_t* sbar = bars + NP + NR;

  UnitSeg U = L.one;
  if (L.n > 1) U = L.segs[find_unitseg(L.segs, L.n, blockIdx.x)];
  const int4 u = U.units[blockIdx.x - U.unit_begin];  // box, y0, z0, z1
  const DRow& R = U.rows[u.x];
  Sweep<T> S;
  S.nx = R.n[0];
  S.ny = R.n[1];
  S.nz = R.n[2];
  S.y0 = u.y & 0xFFFF;
  S.ty = min(min(u.y >> 16, ty_max), S.ny - S.y0);
  S.pitch = R.v[0].pitch;
  S.plane = R.v[0].plane;
  S.g = R.v[0].g;
  S.pr = R.v[1].pitch;
  S.planer = R.v[1].plane;
  S.gr = R.v[1].g;
  S.flags = R.pad_;
  S.mh2 = -(T)R.h2;
  S.lox = R.lo[0];
  S.loy = R.lo[1];
  S.loz = R.lo[2];
  S.pbytes = (uint32_t)((S.ty + 4) * S.pitch * sizeof(T));
  S.rbytes = (uint32_t)((S.ty + 2) * S.pr * sizeof(T));

  const T* src = (const T*)R.v[0].p;  // valid cell (0,0,0) of the source phi
  const T* rhs = (const T*)R.v[1].p;
  T* dst = (T*)R.v[2].p;              // valid cell (0,0,0) of the destination phi
  const int tid = threadIdx.x;
  const int nzl = S.nz;
  const int z0 = u.z, z1 = u.w;  // this CTA finishes planes [z0, z1)

  if (tid == 0) {
    for (int i = 0; i < NP + NR; ++i) mbar_init(&bars[i], 1);
    for (int i = 0; i < kStageBars; ++i) mbar_init(&sbar[i], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // planes are loaded in order from z0-2 (phi) / z0-1 (rhs); slot and mbarrier parity
  auto pslot = [&](int p) { return (p - z0 + 2) % NP; };
  auto rslot = [&](int p) { return (p - z0 + 1) % (NR > 0 ? NR : 1); };
  auto pphase = [&](int p) { return (uint32_t)(((p - z0 + 2) / NP) & 1); };
  auto rphase = [&](int p) { return (uint32_t)(((p - z0 + 1) / (NR > 0 ? NR : 1)) & 1); };
  const int s_first = z0 - 1, s_last = z1;  // stages

  if (tid >= kConsumers) {
    // ---------------- producer ----------------
    if (tid != kConsumers) return;
    const int pmax = z1 + 1, rmax = z1;  // last planes loaded
    int p_issued = z0 - 3, r_issued = z0 - 2;
    auto issue_phi = [&](int p) {
      if (p > pmax) return;
      uint64_t* b = &pbar[pslot(p)];
      mbar_expect_tx(b, S.pbytes);
      bulk_load(pbuf + (size_t)pslot(p) * phi_buf_elems,
                src + (long long)p * S.plane + (long long)(S.y0 - 2) * S.pitch - S.g, S.pbytes, b);
      p_issued = p;
    };
    auto issue_rhs = [&](int p) {
      if (!RS || p > rmax) return;
      uint64_t* b = &rbar[rslot(p)];
      mbar_expect_tx(b, S.rbytes);
      bulk_load(rbuf + (size_t)rslot(p) * rhs_buf_elems,
                rhs + (long long)p * S.planer + (long long)(S.y0 - 1) * S.pr - S.gr, S.rbytes, b);
      r_issued = p;
    };
    // every slot starts free
    for (int p = z0 - 2; p < z0 - 2 + NP; ++p) issue_phi(p);
    if (RS)
      for (int p = z0 - 1; p < z0 - 1 + NR; ++p) issue_rhs(p);
    bool ok = true;
    for (int st = s_first; st <= s_last && ok; ++st) {
      const int k = st - s_first;
      if (!mbar_wait_bounded(&sbar[k % kStageBars], (uint32_t)((k / kStageBars) & 1))) {
        ok = false;
        break;
      }
      if (st - 1 >= z0 && st - 1 < z1) {
        // plane st-1 is final: whole rows y0..y0+ty-1 (the destination's x ghosts are
        // overwritten; they are refilled before they are read)
        T* gdst = dst + (long long)(st - 1) * S.plane + (long long)S.y0 * S.pitch - S.g;
        bulk_store(gdst, pbuf + (size_t)pslot(st - 1) * phi_buf_elems + 2 * S.pitch,
                   (uint32_t)(S.ty * S.pitch * sizeof(T)));
        bulk_commit();
      }
      // from stage z0 on, phi plane st-2 and rhs plane st-1 (loaded by the prologue or an
      // earlier stage) were last read in stage st; the store of plane st-2 (issued one
      // stage earlier) must have finished reading its slot
      if (st >= z0) {
        bulk_wait_read1();
        issue_phi(st - 2 + NP);
        if (RS) issue_rhs(st - 1 + NR);
      }
    }
    if (!ok) atomicExch(err, 1);  // the consumers time out on their own
    // drain: every issued load has landed (consumed or not) and every store has read and
    // written its data before the CTA's shared memory goes away.  A slot is reissued only
    // after its previous plane landed and was consumed, so only the latest plane of each
    // slot can still be in flight (earlier phases of a slot cannot be waited on again).
    for (int p = max(z0 - 2, p_issued - NP + 1); p <= p_issued; ++p)
      mbar_wait_bounded(&pbar[pslot(p)], pphase(p));
    if (RS)
      for (int p = max(z0 - 1, r_issued - NR + 1); p <= r_issued; ++p)
        mbar_wait_bounded(&rbar[rslot(p)], rphase(p));
    bulk_wait_all();
    return;
  }

  // ---------------- consumers ----------------
  // Lane mapping of a plane: lanes per row lpr = smallest power of two >= the row's
  // x-pairs (at most 16); a warp covers 32 / lpr rows per pass, the 8 warps interleave.
  const int npv = (S.nx + 1) >> 1;
  int lsh = 0;
  while ((1 << lsh) < npv && lsh < 4) ++lsh;  // at most 16 lanes per row: pairs of cells
  const int lpr = 1 << lsh;
  const int plane_lane = (tid & 31) & (lpr - 1);
  const int row0 = (tid >> 5) * (32 >> lsh) + ((tid & 31) >> lsh);
  const int row_step = (kConsumers >> 5) * (32 >> lsh);

  for (int s = s_first; s <= s_last; ++s) {
    // inputs of stage s: phi planes s-1..s+1 (and s-2 for the black pass), rhs s and s-1;
    // waits on landed phases return at once
    bool ok = true;
    for (int p = (s == s_first ? z0 - 2 : s + 1); p <= s + 1; ++p)
      ok = ok && mbar_wait_bounded(&pbar[pslot(p)], pphase(p));
    if (RS) ok = ok && mbar_wait_bounded(&rbar[rslot(s)], rphase(s));
    if (ok) {
    // Stage s red-updates plane s and black-updates plane s-1.  Both passes map (row, x) to
    // the same thread, and the red cell (x, y, s) sits right above the black cell
    // (x, y, s-1): the red update reads that black cell's old value, the black update reads
    // the red cell's new one, and every other input of either update was finished in an
    // earlier stage.  So the two passes need no barrier between them.
    T* P0 = pbuf + (size_t)pslot(s - 1) * phi_buf_elems;
    T* P1 = pbuf + (size_t)pslot(s) * phi_buf_elems;
    const T* P2 = pbuf + (size_t)pslot(s + 1) * phi_buf_elems;
    // rhs rows as staged: element (x, y) at [(y - y0 + 1) * pr + x + gr]
    const T* Q = RS ? rbuf + (size_t)rslot(s) * rhs_buf_elems
                    : rhs + (long long)s * S.planer + (long long)(S.y0 - 1) * S.pr - S.gr;
    // element (x, y) of a phi buffer: [(y - y0 + 2) * pitch + x + g]; rhs: [(y - y0 + 1) * pr + x + gr]
    const int gz = S.loz + s;
    // red rows [ya, yb] of plane s: planes outside [z0, z1) are needed only under the tile
    // (as z-neighbours of black cells), the others with a one-row ring
    const bool ghost_plane = (s < z0 || s >= z1);
    const bool red = !((s < 0 && (S.flags & 4)) || (s >= nzl && (S.flags & 32)));
    int ya = ghost_plane ? S.y0 : S.y0 - 1;
    int yb = ghost_plane ? S.y0 + S.ty - 1 : S.y0 + S.ty;
    if (!ghost_plane) {
      if (ya < 0 && (S.flags & 2)) ya = 0;
      if (yb >= S.ny && (S.flags & 16)) yb = S.ny - 1;
    }
    const bool black = (s - 1 >= z0 && s - 1 < z1);  // black rows [y0, y0+ty) of plane s-1
    const T* B0 = black ? pbuf + (size_t)pslot(s - 2) * phi_buf_elems : P0;
    const T* QB = !black ? Q
                  : RS   ? rbuf + (size_t)rslot(s - 1) * rhs_buf_elems
                         : rhs + (long long)(s - 1) * S.planer + (long long)(S.y0 - 1) * S.pr - S.gr;
    {
      int y = S.y0 - 1 + row0;
      int par = (S.lox + S.loy + y + gz) & 1;  // first red x >= 0 of row y in plane s
      const int pflip = row_step & 1;
      for (; y <= S.y0 + S.ty; y += row_step, par ^= pflip) {
        const bool r_on = red && y >= ya && y <= yb;
        const bool b_on = black && y >= S.y0 && y < S.y0 + S.ty;
        if (!r_on && !b_on) continue;
        const int o = (y - S.y0 + 2) * S.pitch + S.g;
        const int oq = (y - S.y0 + 1) * S.pr + S.gr;
        T* p1 = P1 + o;
        T* p0 = P0 + o;
        // cells x and x2 = x + 2 lpr together: both red (or both black), so neither reads
        // the other; all loads of a pair go before its stores (two independent chains)
        auto red_sum = [&](int x) {
          T a = p1[x - 1];
          a = Ar<T>::add(a, p1[x + 1]);
          a = Ar<T>::add(a, p1[x - S.pitch]);
          a = Ar<T>::add(a, p1[x + S.pitch]);
          a = Ar<T>::add(a, p0[x]);
          return Ar<T>::add(a, P2[o + x]);
        };
        auto black_sum = [&](int x, T zr) {
          T a = p0[x - 1];
          a = Ar<T>::add(a, p0[x + 1]);
          a = Ar<T>::add(a, p0[x - S.pitch]);
          a = Ar<T>::add(a, p0[x + S.pitch]);
          a = Ar<T>::add(a, B0[o + x]);
          return Ar<T>::add(a, zr);
        };
        for (int x = par + 2 * plane_lane; x < S.nx; x += 4 * lpr) {
          const int x2 = x + 2 * lpr;
          const bool two = x2 < S.nx;
          const int xb = two ? x2 : x;  // (a harmless repeat of x when there is no second cell)
          // red values above the black cells: new if updated now
          T zr1 = p1[x], zr2 = p1[xb];
          if (r_on) {
            const T a1 = red_sum(x), a2 = red_sum(xb);
            const T q1 = Q[oq + x], q2 = Q[oq + xb];
            zr1 = gs_update(a1, q1, S.mh2);
            zr2 = gs_update(a2, q2, S.mh2);
            p1[x] = zr1;
            if (two) p1[x2] = zr2;
          }
          if (b_on) {
            const T a1 = black_sum(x, zr1), a2 = black_sum(xb, zr2);
            const T q1 = QB[oq + x], q2 = QB[oq + xb];
            const T b1 = gs_update(a1, q1, S.mh2), b2 = gs_update(a2, q2, S.mh2);
            p0[x] = b1;
            if (two) p0[x2] = b2;
          }
        }
      }
    }
    // red ring cells x = -1 and x = nx of rows inside the box (their red value feeds the
    // black update of x = 0 / nx-1 in the next stage), one thread per row, counted from the
    // last consumer down (the first warps take the rows past a full pass above)
    if (red && !ghost_plane) {
      const bool lo_in = !(S.flags & 1), hi_in = !(S.flags & 8);
      for (int y = ya + (kConsumers - 1 - tid); y <= yb; y += kConsumers) {
        if (y < 0 || y >= S.ny) continue;
        const int gy = S.loy + y;
        const int orow = (y - S.y0 + 2) * S.pitch + S.g;
        const int qrow = (y - S.y0 + 1) * S.pr + S.gr;
        for (int side = 0; side < 2; ++side) {
          const int x = side ? S.nx : -1;
          if (!(side ? hi_in : lo_in) || ((S.lox + x + gy + gz) & 1)) continue;
          const int o = orow + x;
          T a = P1[o - 1];
          a = Ar<T>::add(a, P1[o + 1]);
          a = Ar<T>::add(a, P1[o - S.pitch]);
          a = Ar<T>::add(a, P1[o + S.pitch]);
          a = Ar<T>::add(a, P0[o]);
          a = Ar<T>::add(a, P2[o]);
          P1[o] = gs_update(a, Q[qrow + x], S.mh2);
        }
      }
    }
      fence_async_smem();  // make the generic-proxy writes visible to the bulk stores
    }
    // stage s finished by every consumer; a wait that expired anywhere ends the CTA's work
    if (consumer_sync_or(!ok)) {
      if (tid == 0) atomicExch(err, 1);
      break;
    }
    if (tid == 0) mbar_arrive(&sbar[(s - s_first) % kStageBars]);
  }
}

template <class T, int D, bool RS>
static cudaError_t launch_fused_t(const UnitList& L, long long nunits, int ty, int max_pitch,
                                  int max_pitch_r, int* err, cudaStream_t s) {
  constexpr int NP = 4 + D, NR = RS ? 2 + D : 0;
  unsigned pe = (unsigned)((ty + 4) * max_pitch);
  unsigned re = (unsigned)((ty + 2) * max_pitch_r);
  const unsigned align = 128 / sizeof(T);
  pe = (pe + align - 1) / align * align;
  re = (re + align - 1) / align * align;
  size_t smem = ((size_t)NP * pe + (size_t)NR * re) * sizeof(T) + (NP + NR + kStageBars) * 8;
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = opt_in_smem((const void*)k_rbgs_fused<T, D, RS>, smem);
  if (e != cudaSuccess) return e;
  launch_k(k_rbgs_fused<T, D, RS>, (unsigned)nunits, kFusedThreads, smem, s, L, ty, pe, re, err);
  count_launches(1);
  return cudaGetLastError();
}

size_t fused_smem_bytes(int dt, int ty, int max_pitch, int max_pitch_r, int depth, bool rhs_smem) {
  size_t es = dt == DT_F64 ? 8 : 4;
  int NP = 4 + depth, NR = rhs_smem ? 2 + depth : 0;
  size_t align = 128 / es;
  size_t pe = ((size_t)(ty + 4) * max_pitch + align - 1) / align * align;
  size_t re = ((size_t)(ty + 2) * max_pitch_r + align - 1) / align * align;
  return (NP * pe + NR * re) * es + (NP + NR + kStageBars) * 8;
}

template <class T, bool RS>
static cudaError_t launch_fused_d(const UnitList& L, long long nunits, int ty, int depth,
                                  int max_pitch, int max_pitch_r, int* err, cudaStream_t s) {
  if (depth <= 1) return launch_fused_t<T, 1, RS>(L, nunits, ty, max_pitch, max_pitch_r, err, s);
  if (depth == 2) return launch_fused_t<T, 2, RS>(L, nunits, ty, max_pitch, max_pitch_r, err, s);
  if (depth == 3) return launch_fused_t<T, 3, RS>(L, nunits, ty, max_pitch, max_pitch_r, err, s);
  return launch_fused_t<T, 4, RS>(L, nunits, ty, max_pitch, max_pitch_r, err, s);
}

cudaError_t launch_rbgs_fused_l(int dt, const UnitList& L, long long nunits, int ty, int depth,
                                int max_pitch, int max_pitch_r, bool rhs_smem, int* err,
                                cudaStream_t s) {
  if (nunits <= 0) return cudaSuccess;
  if (dt == DT_F64)
    return rhs_smem ? launch_fused_d<double, true>(L, nunits, ty, depth, max_pitch, max_pitch_r, err, s)
                    : launch_fused_d<double, false>(L, nunits, ty, depth, max_pitch, max_pitch_r, err, s);
  return rhs_smem ? launch_fused_d<float, true>(L, nunits, ty, depth, max_pitch, max_pitch_r, err, s)
                  : launch_fused_d<float, false>(L, nunits, ty, depth, max_pitch, max_pitch_r, err, s);
}

cudaError_t launch_rbgs_fused(int dt, const DRow* rows, const int4* units, int nunits, int ty,
                              int depth, int max_pitch, int max_pitch_r, bool rhs_smem, int* err,
                              cudaStream_t s) {
  UnitList L{};
  L.one.rows = rows;
  L.one.units = units;
  L.one.unit_begin = 0;
  L.one.nunits = nunits;
  L.n = 1;
  return launch_rbgs_fused_l(dt, L, nunits, ty, depth, max_pitch, max_pitch_r, rhs_smem, err, s);
}

}  // namespace gbmg
