// Kernels of the multigrid path on sm_103a: ghost fill over copy tags, red-black
// Gauss-Seidel half-sweeps, residual with fused max-norm, fused residual + restriction,
// restriction, prolongation, bottom solve and the mixed-precision scale / correction.
//
// All stencil kernels are bounded by HBM bandwidth (about 1 flop per byte), so none of them
// uses the tensor cores.  Each launch covers every box of its table (Sec. 3.2 kernel fusing).
// Arithmetic goes through __{d,f}{add,mul,fma}_rn intrinsics in a fixed order, each one IEEE
// round-to-nearest step, so results match the documented formulas bit for bit.  On GB300
// FP64 instructions are scarce (the FP64 pipe issues far fewer lanes per clock than FP32), so
// the FP64 forms use fused multiply-adds and a multiplication by the rounded 1/6, and sign
// flips and absolute values are integer operations on the bit pattern.
#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <mutex>
#include <cstdio>

#include "mg_bits.hpp"
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
  // sign flip and |.| as integer operations (no FP64 pipe instruction)
  static __device__ __forceinline__ double neg(double a) {
    return __longlong_as_double(__double_as_longlong(a) ^ (long long)0x8000000000000000ull);
  }
  // monotonic key of |a| (NaN above Inf), comparable across a warp.  The sign is cleared in
  // the high 32-bit word: written as a 64-bit mask, the compiler turned it into an FP64
  // absolute value -- one FP64-pipe instruction per cell in the norm-taking kernels (GB300:
  // FP64 residual 272 -> 238 us at 256^3, 256^3 solve 56.1 -> 57.1 solves/s).
  static __device__ __forceinline__ unsigned long long abskey(double a) {
    unsigned lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(a));
    return ((unsigned long long)(hi & 0x7FFFFFFFu) << 32) | lo;
  }
  // key -> bit pattern of the double |a|
  static __device__ __forceinline__ unsigned long long key_to_f64bits(unsigned long long k) { return k; }
};
template <>
struct Ar<float> {
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
  static __device__ __forceinline__ float neg(float a) {
    return __int_as_float(__float_as_int(a) ^ (int)0x80000000u);
  }
  static __device__ __forceinline__ unsigned long long abskey(float a) {
    return (unsigned long long)((unsigned)__float_as_int(a) & 0x7FFFFFFFu);
  }
  static __device__ __forceinline__ unsigned long long key_to_f64bits(unsigned long long k) {
    return k ? (unsigned long long)__double_as_longlong((double)__int_as_float((int)k)) : 0ull;
  }
};

// Gauss-Seidel update and residual of one cell (s = ordered neighbour sum):
//   update   phi = fma(-h^2, rhs, s) * (1/6)
//   residual r   = fma(-1/h^2, fma(-6, phi, s), rhs)
template <class T>
__device__ __forceinline__ T gs_update(T s, T rhs, T h2) {
  constexpr T inv6 = T(1) / T(6);
  return Ar<T>::mul(Ar<T>::fma(Ar<T>::neg(h2), rhs, s), inv6);
}
template <class T>
__device__ __forceinline__ T residual_of(T s, T phi, T rhs, T ih2) {
  return Ar<T>::fma(Ar<T>::neg(ih2), Ar<T>::fma(T(-6), phi, s), rhs);
}

// A level constant (h^2, 1/h^2; binary64 in the box table) in the kernel's type.  For binary32
// the rounding is done with integer operations: a conversion would occupy the FP64 pipe once per
// row and lane of an otherwise FP32 kernel.
template <class T>
__device__ __forceinline__ T level_const(double d);
template <>
__device__ __forceinline__ double level_const<double>(double d) { return d; }
template <>
__device__ __forceinline__ float level_const<float>(double d) {
  float f;
  return bits::scale_to_f32(d, 0, &f) ? f : __double2float_rn(d);
}

constexpr int kWarps = 8;  // warps per block in the row kernels
constexpr int kThreads = kWarps * 32;

// Box of segment row r (0 <= r < cnt).  Boxes of equal row counts (the usual case) are found
// by the proportional guess, checked with two independent loads; else binary search.
__device__ __forceinline__ int find_box(const DRow* __restrict__ rows, int nbox, long long r,
                                        long long cnt) {
  if (cnt > 0 && cnt * nbox < (1ll << 32)) {
    int g = (int)((unsigned)(r * nbox) / (unsigned)cnt);
    g = g < nbox - 1 ? g : nbox - 1;
    const long long a = rows[g].row0;
    const long long e = g + 1 < nbox ? rows[g + 1].row0 : cnt;
    if (a <= r && r < e) return g;
  }
  int lo = 0, hi = nbox - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (rows[mid].row0 <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int find_seg(const Seg* __restrict__ segs, int n, long long r) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (segs[mid].row_begin <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Block k owns launch rows [k*per, (k+1)*per).  A warp is split into HW lane groups of
// 32 / HW lanes, each with its own row: group q of warp w takes rows begin + HW*w + q, step
// HW*kWarps.  f(row, row-within-box, slot) is called once per row with all lanes of the
// group active.
template <int HW = 1, class F>
__device__ __forceinline__ void for_rows(const SegList& L, long long nrows, long long per, F&& f) {
  long long begin = (long long)blockIdx.x * per;
  long long end = begin + per < nrows ? begin + per : nrows;
  long long r = begin + (long long)(threadIdx.x >> 5) * HW + (int)((threadIdx.x & 31) / (32 / HW));
  if (r >= end) return;
  int si = 0;
  Seg S = L.one;
  if (L.n > 1) {
    si = find_seg(L.segs, L.n, r);
    S = L.segs[si];
  }
  int b = find_box(S.rows, S.nbox, r - S.row_begin, L.n > 1 ? S.row_count : nrows);
  for (; r < end; r += kWarps * HW) {
    if (L.n > 1) {
      bool moved = false;
      while (si + 1 < L.n && L.segs[si + 1].row_begin <= r) {
        ++si;
        moved = true;
      }
      if (moved) {
        S = L.segs[si];
        b = 0;
      }
    }
    const long long lr = r - S.row_begin;
    while (b + 1 < S.nbox && S.rows[b + 1].row0 <= lr) ++b;
    const DRow& R = S.rows[b];
    f(R, lr - R.row0, S.slot);
  }
}

__device__ __forceinline__ unsigned long long warp_max(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Sum of the six neighbours of p[0] in the order x-, x+, y-, y+, z-, z+ (ghost cells read as
// they are).
template <class T>
__device__ __forceinline__ T nbr_sum(const T* p, int pitch, long long plane) {
  T s = p[-1];
  s = Ar<T>::add(s, p[1]);
  s = Ar<T>::add(s, p[-pitch]);
  s = Ar<T>::add(s, p[pitch]);
  s = Ar<T>::add(s, p[-plane]);
  s = Ar<T>::add(s, p[plane]);
  return s;
}

template <class T>
__device__ __forceinline__ T* line(const DView& v, int y, int z) {
  return (T*)v.p + (long long)z * v.plane + (long long)y * v.pitch;
}

// Neighbour rows of row (y, z) of v[0] for the stencil kernels, with the box-face reads of
// DRow::nbd / nbf applied (ghost cells when those are zero).  Negations are applied as XORs of
// the sign bit with a runtime 0/1 flag, so they never turn into extra floating-point work.
template <class T>
struct Nbr {
  const T* ym;
  const T* yp;
  const T* zm;
  const T* zp;
  long long dxm, dxp;  // x- at x = 0, x+ at x = nx-1
  unsigned neg;        // bit f: negate face f's reads (x-, x+, y-, y+, z-, z+) in this row
};
__device__ __forceinline__ double xsign(double v, unsigned n) {
  // (on the high 32-bit word: measured 0.5% faster in the 256^3 solve than a 64-bit XOR)
  unsigned lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(v));
  double r;
  asm("mov.b64 %0, {%1, %2};" : "=d"(r) : "r"(lo), "r"(hi ^ (n << 31)));
  return r;
}
__device__ __forceinline__ float xsign(float v, unsigned n) {
  return __int_as_float(__float_as_int(v) ^ (int)(n << 31));
}

template <class T>
__device__ __forceinline__ Nbr<T> nbr_rows(const DRow& R, const T* row, int y, int z) {
  const int pitch = R.v[0].pitch;
  const long long plane = R.v[0].plane;
  const unsigned f = (unsigned)R.nbf;
  const bool y0 = y == 0, y1 = y == R.n[1] - 1, z0 = z == 0, z1 = z == R.n[2] - 1;
  Nbr<T> b;
  b.ym = row - pitch + (y0 ? R.nbd[2] : 0);
  b.yp = row + pitch + (y1 ? R.nbd[3] : 0);
  b.zm = row - plane + (z0 ? R.nbd[4] : 0);
  b.zp = row + plane + (z1 ? R.nbd[5] : 0);
  b.dxm = R.nbd[0];
  b.dxp = R.nbd[1];
  b.neg = (f & 3u) | (y0 ? f & 4u : 0u) | (y1 ? f & 8u : 0u) | (z0 ? f & 16u : 0u) |
          (z1 ? f & 32u : 0u);
  return b;
}

// The six-neighbour sum of cell x of `row` (order x-, x+, y-, y+, z-, z+) through Nbr.  The
// x-face negations (whole boxes) apply to the end cells only; NEGYZ: the row also has negated
// y / z reads (its box's face rows at a Dirichlet face -- decided per row, so a warp takes
// one branch).
template <bool NEGYZ, class T>
__device__ __forceinline__ T nbr_sum_rows(const T* row, int x, int nx, const Nbr<T>& b) {
  const bool e0 = x == 0, e1 = x == nx - 1;
  T xm = row[x - 1 + (e0 ? b.dxm : 0)];
  T xp = row[x + 1 + (e1 ? b.dxp : 0)];
  if (e0) xm = xsign(xm, b.neg & 1u);
  if (e1) xp = xsign(xp, (b.neg >> 1) & 1u);
  T ym = b.ym[x], yp = b.yp[x], zm = b.zm[x], zp = b.zp[x];
  if (NEGYZ) {
    ym = xsign(ym, (b.neg >> 2) & 1u);
    yp = xsign(yp, (b.neg >> 3) & 1u);
    zm = xsign(zm, (b.neg >> 4) & 1u);
    zp = xsign(zp, (b.neg >> 5) & 1u);
  }
  T s = Ar<T>::add(xm, xp);
  s = Ar<T>::add(s, ym);
  s = Ar<T>::add(s, yp);
  s = Ar<T>::add(s, zm);
  s = Ar<T>::add(s, zp);
  return s;
}

// ---------------------------------------------------------------------------------------
// Copy tags (ghost fill).  One warp per chunk of whole x-rows of one tag (tag_chunk_rows).
// Segments = fabs.  Sources are valid cells and destinations ghost cells, never the same
// memory within a launch, so sources are read through the read-only path.
__device__ __forceinline__ int find_tagseg(const TagSeg* __restrict__ segs, int n, long long w) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (segs[mid].chunk_begin <= w) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <class T>
__device__ __forceinline__ T tag_value(const T* p, int sign) {
  if (sign == 0) return T(0);
  const T v = __ldg(p);
  return sign > 0 ? v : Ar<T>::neg(v);
}

// A lane handles cells lane, lane + 32, ... of its warp's chunk (x fastest), U at a time
// (the chunk's cells per lane): all loads of a batch are issued before its stores, so each
// lane keeps several independent loads in flight (the fill is bound by memory latency, not
// bandwidth).  NC = 1: one component; NC = 0: ncomp components.
template <class T, int NC>
__global__ void __launch_bounds__(256) k_copy_tags(TagList L, long long nchunks, int ncomp) {
  pdl_begin();
  constexpr int U = (NC == 1 ? (sizeof(T) == 4 ? kTagChunk1F : kTagChunk1) : kTagChunkN) / 32;
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (w >= nchunks) return;
  const int lane = threadIdx.x & 31;
  TagSeg S = L.one;
  if (L.n > 1) S = L.segs[find_tagseg(L.segs, L.n, w)];
  const int2 ch = S.chunks[w - S.chunk_begin];
  const DTag t = S.tags[ch.x];
  const int r1 = min(ch.y + tag_chunk_rows(t.ex, ncomp, (int)sizeof(T)), t.ey * t.ez);
  const int ncell = (r1 - ch.y) * t.ex;
  T* __restrict__ base = (T*)S.base;
  const int nc = NC ? NC : ncomp;
  for (int i0 = lane; i0 < ncell; i0 += 32 * U) {
    long long so[U], d[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = min(i0 + 32 * u, ncell - 1);  // tail lanes repeat the last cell
      const int x = i % t.ex, r = ch.y + i / t.ex;
      const int y = r % t.ey, z = r / t.ey;
      so[u] = t.src + (long long)x * t.ssx + (long long)y * t.ssy + (long long)z * t.ssz;
      d[u] = t.dst + x + (long long)y * t.dsy + (long long)z * t.dsz;
    }
    for (int c = 0; c < nc; ++c) {
      T v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = tag_value(base + so[u] + c * t.scs, t.sign);
#pragma unroll
      for (int u = 0; u < U; ++u) base[d[u] + c * t.dcs] = v[u];
    }
  }
}

// The same fill for fabs of 2 to 4 components (NC = 4): every component's loads of a lane's
// U cells are issued before any store, and cell offsets are kept as 32-bit offsets from the
// tag's first source / destination cell (fewer registers, more resident warps).
template <class T>
__global__ void __launch_bounds__(256, 3) k_copy_tags_multi(TagList L, long long nchunks,
                                                            int ncomp) {
  pdl_begin();
  constexpr int U = kTagChunkN / 32;
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (w >= nchunks) return;
  const int lane = threadIdx.x & 31;
  TagSeg S = L.one;
  if (L.n > 1) S = L.segs[find_tagseg(L.segs, L.n, w)];
  const int2 ch = S.chunks[w - S.chunk_begin];
  const DTag t = S.tags[ch.x];
  const int r1 = min(ch.y + tag_chunk_rows(t.ex, ncomp, (int)sizeof(T)), t.ey * t.ez);
  const int ncell = (r1 - ch.y) * t.ex;
  const T* __restrict__ src = (const T*)S.base + t.src;
  T* __restrict__ dst = (T*)S.base + t.dst;
  for (int i0 = lane; i0 < ncell; i0 += 32 * U) {
    int so[U], d[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = min(i0 + 32 * u, ncell - 1);  // tail lanes repeat the last cell
      const int x = i % t.ex, r = ch.y + i / t.ex;
      const int y = r % t.ey, z = r / t.ey;
      so[u] = x * t.ssx + y * t.ssy + z * t.ssz;
      d[u] = x + y * t.dsy + z * t.dsz;
    }
    T v[4][U];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int u = 0; u < U; ++u)
        v[c][u] = c < ncomp ? tag_value(src + so[u] + c * t.scs, t.sign) : T(0);
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (c < ncomp) dst[d[u] + c * t.dcs] = v[c][u];
  }
}

// ---------------------------------------------------------------------------------------
// Flush per-warp maxima: each warp stores (slot, max); thread 0 merges equal slots.
__device__ __forceinline__ void flush_block_max(unsigned long long mx, int cur,
                                                unsigned long long* norms) {
  __shared__ unsigned long long s_max[kWarps];
  __shared__ int s_sol[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  mx = warp_max(mx);
  if (lane == 0) { s_max[warp] = mx; s_sol[warp] = cur; }
  __syncthreads();
  if (threadIdx.x == 0) {
    int sol = -1;
    unsigned long long acc = 0;
    for (int w = 0; w < kWarps; ++w) {
      if (s_sol[w] < 0) continue;
      if (s_sol[w] != sol) {
        if (sol >= 0 && acc) atomicMax(&norms[sol], acc);
        sol = s_sol[w];
        acc = 0;
      }
      acc = s_max[w] > acc ? s_max[w] : acc;
    }
    if (sol >= 0 && acc) atomicMax(&norms[sol], acc);
  }
}

// Red-black Gauss-Seidel half-sweep: cells with (i+j+k) mod 2 == color (global indices)
// take phi = (s - h^2 rhs) / 6.  G lanes per x-line (16 for wide boxes, fewer for narrow
// ones so that every lane has two cells): lane l updates cells par + 2l + 4Gk and
// par + 2l + 4Gk + 2G together.
// DIRECT: box-face neighbours through DRow::nbd / nbf (rows without that information read
// their ghost cells); else ghost cells, through plain offsets.
// MODE 1 (norms != null, single-segment launches, DIRECT only): also the max-norm of the
// residual of every updated cell just after its update, into norms[slot + solve].  The
// neighbour sum of the update serves, since the other colour's cells are unchanged by this
// half-sweep -- except where a read is the cell's own value negated (a Dirichlet face):
// those cells sum again, reading their new value.  (With an odd periodic extent an image
// could be the cell's own colour; callers use this on even periodic extents only.)
// MODE 2 (same conditions): the max-norm of the residual of every updated cell just BEFORE
// its update -- the neighbour sum of the update is exactly the one that residual needs,
// Dirichlet reads included, since they read the cell's value before the update -- and the
// value before the update saved to v[2], so that the half-sweep can be undone
// (k_restore_colour).
// MODE 3 (same conditions, no norm): the residual of every updated cell just after its update
// (as MODE 1 takes it) stored to v[2], for the residual + restriction that follows
// (k_residual_restrict with STORED).
// MODE 4 (plain, as MODE 0): four cells of a lane per step with all loads first, for FP32
// launches over rows of 64 to 127 cells (measured on GB300: 64-wide boxes, 256^3 FP32
// half-sweep 45.5 -> 42.5 us; the two-cell form is faster on 32-wide rows, and on 128-wide
// ones: 512^3 454 against 492 us).
// v[2] of MODE 2 / 3 is a one-colour view: cell x of row (y, z) at element x / 2 of the row
// (two cells of one colour are never neighbours in x), so that a warp's stores fill whole
// sectors instead of every other element of sectors it has not read.
// Resident blocks per SM the half-sweep is built for (register budget): the norm variants
// hold more live values.
// (Measured on GB300 at 256^3: 3 blocks per SM for the norm / store variants, without
// spills, made the solve 1% slower than 4 with a few spilled registers.)
constexpr int kSweepMinBlocks = 4, kNormMinBlocks = 4;
template <class T, bool DIRECT, int MODE, int G>
__global__ void __launch_bounds__(kThreads, MODE ? kNormMinBlocks : kSweepMinBlocks)
    k_rbgs_half(SegList L, long long nrows, long long per, int color, unsigned long long* norms) {
  pdl_begin();
  // A lane updates cells x and x + 2G of a pair step together (both of this colour: their
  // neighbours are of the other colour and unchanged, so both loads go first -- two
  // independent FP64 chains per lane).
  const int sub = threadIdx.x & (G - 1);
  unsigned long long mx = 0;
  int cur = -1;
  for_rows<32 / G>(L, nrows, per, [&](const DRow& R, long long lr, int slot) {
    const int n0 = R.n[0], n1 = R.n[1];
    const int y = (int)lr % n1, z = (int)lr / n1;
    T* phi = line<T>(R.v[0], y, z);
    const T* rhs = line<T>(R.v[1], y, z);
    T* save = MODE == 2 || MODE == 3 ? line<T>(R.v[2], y, z) : nullptr;  // saved values / residuals
    const T h2 = level_const<T>(R.h2), ih2 = level_const<T>(R.ih2);
    const int par = (color + R.lo[0] + R.lo[1] + y + R.lo[2] + z) & 1;
    cur = slot + R.solve;
    auto norm = [&](T s, T u, T r) {
      const unsigned long long k = Ar<T>::abskey(residual_of(s, u, r, ih2));
      mx = k > mx ? k : mx;
    };
    auto sweep = [&](auto&& sum, auto&& resum) {
      if constexpr (MODE == 4) {
        // four cells of a lane per step, all loads first
        for (int x = par + 2 * sub; x < n0; x += 8 * G) {
          T sv[4], rv[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int xq = x + 2 * G * q;
            sv[q] = xq < n0 ? sum(xq) : T(0);
            rv[q] = xq < n0 ? rhs[xq] : T(0);
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int xq = x + 2 * G * q;
            if (xq < n0) phi[xq] = gs_update(sv[q], rv[q], h2);
          }
        }
        return;
      }
      for (int x = par + 2 * sub; x < n0; x += 4 * G) {
        const int x2 = x + 2 * G;
        const bool two = x2 < n0;
        const T s1 = sum(x);
        const T s2 = two ? sum(x2) : T(0);
        const T r1 = rhs[x];
        const T r2 = two ? rhs[x2] : T(0);
        T o1 = T(0), o2 = T(0);
        if (MODE == 2) {
          o1 = phi[x];
          o2 = two ? phi[x2] : T(0);
        }
        const T u1 = gs_update(s1, r1, h2);
        if (MODE == 2) {
          norm(s1, o1, r1);
          save[x >> 1] = o1;
        }
        phi[x] = u1;
        if (MODE == 1) norm(resum(x, s1), u1, r1);
        if (MODE == 3) save[x >> 1] = residual_of(resum(x, s1), u1, r1, ih2);
        if (two) {
          const T u2 = gs_update(s2, r2, h2);
          if (MODE == 2) {
            norm(s2, o2, r2);
            save[x2 >> 1] = o2;
          }
          phi[x2] = u2;
          if (MODE == 1) norm(resum(x2, s2), u2, r2);
          if (MODE == 3) save[x2 >> 1] = residual_of(resum(x2, s2), u2, r2, ih2);
        }
      }
    };
    if constexpr (DIRECT) {
      const Nbr<T> nb = nbr_rows<T>(R, phi, y, z);
      // cells with a negated read of their own value sum again after their update
      auto resum = [&](int x, T s) {
        const bool own = (nb.neg & 60u) || (x == 0 && (nb.neg & 1u)) || (x == n0 - 1 && (nb.neg & 2u));
        return own ? nbr_sum_rows<true>(phi, x, n0, nb) : s;
      };
      if ((nb.neg & 60u) == 0) sweep([&](int x) { return nbr_sum_rows<false>(phi, x, n0, nb); }, resum);
      else sweep([&](int x) { return nbr_sum_rows<true>(phi, x, n0, nb); }, resum);
    } else {
      const int pitch = R.v[0].pitch;
      const long long plane = R.v[0].plane;
      sweep([&](int x) { return nbr_sum(phi + x, pitch, plane); }, [](int, T s) { return s; });
    }
  });
  if (MODE == 1 || MODE == 2) flush_block_max(Ar<T>::key_to_f64bits(warp_max(mx)), cur, norms);
}

// Undo of a MODE 2 half-sweep: cells of colour `color` take back their saved values
// (v[0] = phi, v[2] = the saved values, one-colour view).
template <class T>
__global__ void __launch_bounds__(kThreads) k_restore_colour(SegList L, long long nrows, long long per,
                                                             int color) {
  pdl_begin();
  const int lane = threadIdx.x & 31;
  for_rows(L, nrows, per, [&](const DRow& R, long long lr, int) {
    const int n0 = R.n[0], n1 = R.n[1];
    const int y = (int)lr % n1, z = (int)lr / n1;
    T* phi = line<T>(R.v[0], y, z);
    const T* save = line<T>(R.v[2], y, z);
    const int par = (color + R.lo[0] + R.lo[1] + y + R.lo[2] + z) & 1;
    for (int x = par + 2 * lane; x < n0; x += 64) phi[x] = save[x >> 1];
  });
}

// Residual r = rhs - (s - 6 phi) / h^2, optionally stored, with a fused max-norm into
// norms[slot + solve].
template <class T, bool DIRECT>
__global__ void __launch_bounds__(kThreads, DIRECT ? 4 : 6) k_residual(SegList L, long long nrows, long long per,
                                                       unsigned long long* norms, int color) {
  pdl_begin();
  const int lane = threadIdx.x & 31;
  unsigned long long mx = 0;
  int cur = -1;
  for_rows(L, nrows, per, [&](const DRow& R, long long lr, int slot) {
    const int idx = slot + R.solve;
    if (idx != cur) {
      if (cur >= 0 && norms) {
        unsigned long long m = Ar<T>::key_to_f64bits(warp_max(mx));
        if (lane == 0 && m) atomicMax(&norms[cur], m);
      }
      cur = idx;
      mx = 0;
    }
    const int n0 = R.n[0], n1 = R.n[1];
    const int y = (int)lr % n1, z = (int)lr / n1;
    const T* phi = line<T>(R.v[0], y, z);
    const T* rhs = line<T>(R.v[1], y, z);
    T* r = R.v[2].p ? line<T>(R.v[2], y, z) : nullptr;
    const T ih2 = level_const<T>(R.ih2);
    const Nbr<T> nb = DIRECT ? nbr_rows<T>(R, phi, y, z) : Nbr<T>{};
    auto cell = [&](int x, T s) {
      T v = residual_of(s, phi[x], rhs[x], ih2);
      if (r) r[x] = v;
      unsigned long long k = Ar<T>::abskey(v);
      mx = k > mx ? k : mx;
    };
    // color < 0: every cell; else the cells of that colour only
    const int x0 = color < 0 ? lane : ((color + R.lo[0] + R.lo[1] + y + R.lo[2] + z) & 1) + 2 * lane;
    const int dx = color < 0 ? 32 : 64;
    if constexpr (DIRECT) {
      if ((nb.neg & 60u) == 0) {
        for (int x = x0; x < n0; x += dx) cell(x, nbr_sum_rows<false>(phi, x, n0, nb));
      } else {
        for (int x = x0; x < n0; x += dx) cell(x, nbr_sum_rows<true>(phi, x, n0, nb));
      }
    } else {
      for (int x = x0; x < n0; x += dx) cell(x, nbr_sum(phi + x, R.v[0].pitch, R.v[0].plane));
    }
  });
  if (norms) flush_block_max(Ar<T>::key_to_f64bits(warp_max(mx)), cur, norms);
}

// Fused residual + restriction.  G lanes per coarse x-line (32, or fewer for narrow boxes):
// lane l produces coarse cells X = l, l+G, ...: the 8 child residuals summed x fastest,
// times 1/8.
// STORED: the children of colour 1 (black) take the residual that the preceding black
// half-sweep stored in v[2] (k_rbgs_half MODE 3, the same value; one-colour view, so that
// the black child of fine row (2Y + j, 2Z + k) is element X) instead of computing it.
// (FP32: a register budget for 3 blocks per SM, with a few spills, made 512 batched problems
// 4.6% faster than the 2 blocks of 100 registers; FP64 was unchanged.)
template <class T, bool DIRECT, int G, bool STORED = false>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 2) k_residual_restrict(SegList L, long long nrows,
                                                                long long per) {
  pdl_begin();
  const int lane = threadIdx.x & (G - 1);
  for_rows<32 / G>(L, nrows, per, [&](const DRow& R, long long lr, int) {
    const int nc0 = R.n[0] >> 1, nc1 = R.n[1] >> 1;
    const int Y = (int)lr % nc1, Z = (int)lr / nc1;
    const DView vp = R.v[0], vr = R.v[1];
    const T ih2 = level_const<T>(R.ih2);
    T* crhs = line<T>(R.c[0], Y, Z);
    T* cphi = R.c[1].p ? line<T>(R.c[1], Y, Z) : nullptr;
    const int n0 = R.n[0];
    for (int X = lane; X < nc0; X += G) {
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const T* row = line<T>(vp, 2 * Y + j, 2 * Z + k);
          const Nbr<T> nb = DIRECT ? nbr_rows<T>(R, row, 2 * Y + j, 2 * Z + k) : Nbr<T>{};
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            T v;
            if (STORED && ((R.lo[0] + R.lo[1] + R.lo[2] + i + j + k) & 1)) {
              v = line<T>(R.v[2], 2 * Y + j, 2 * Z + k)[X];
            } else {
              const T* q = line<T>(vr, 2 * Y + j, 2 * Z + k) + 2 * X + i;
              T s = !DIRECT ? nbr_sum(row + 2 * X + i, vp.pitch, vp.plane)
                            : (nb.neg & 60u) ? nbr_sum_rows<true>(row, 2 * X + i, n0, nb)
                                             : nbr_sum_rows<false>(row, 2 * X + i, n0, nb);
              v = residual_of(s, row[2 * X + i], q[0], ih2);
            }
            acc = (i | j | k) ? Ar<T>::add(acc, v) : v;
          }
        }
      crhs[X] = Ar<T>::mul(acc, (T)0.125);
      if (cphi) cphi[X] = T(0);
    }
  });
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_restrict(SegList L, long long nrows, long long per) {
  pdl_begin();
  const int lane = threadIdx.x & 31;
  for_rows(L, nrows, per, [&](const DRow& R, long long lr, int) {
    const int nc0 = R.n[0] >> 1, nc1 = R.n[1] >> 1;
    const int Y = (int)lr % nc1, Z = (int)lr / nc1;
    T* c = line<T>(R.c[0], Y, Z);
    for (int X = lane; X < nc0; X += 32) {
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            T v = line<T>(R.v[0], 2 * Y + j, 2 * Z + k)[2 * X + i];
            acc = (i | j | k) ? Ar<T>::add(acc, v) : v;
          }
      c[X] = Ar<T>::mul(acc, (T)0.125);
    }
  });
}

// fine(c) += coarse(floor(c / 2)); c[0] addresses coarse cell floor(lo / 2).  G lanes per
// fine x-line.
template <class T, int G>
__global__ void __launch_bounds__(kThreads) k_prolong_add(SegList L, long long nrows, long long per) {
  pdl_begin();
  const int lane = threadIdx.x & (G - 1);
  for_rows<32 / G>(L, nrows, per, [&](const DRow& R, long long lr, int) {
    const int n0 = R.n[0], n1 = R.n[1];
    const int y = (int)lr % n1, z = (int)lr / n1;
    const int ox = R.lo[0] & 1, oy = R.lo[1] & 1, oz = R.lo[2] & 1;
    T* f = line<T>(R.v[0], y, z);
    const T* c = line<T>(R.c[0], (y + oy) >> 1, (z + oz) >> 1);
    if constexpr (sizeof(T) == 4) {
      // FP32: four cells of a lane per step, all loads first (measured on GB300: 512
      // batched problems 2242 -> 2345 solves/s; the FP64 form keeps one cell per step, as
      // four made the 256^3 FP64 solve 3% slower)
      for (int x = lane; x < n0; x += 4 * G) {
        T a[4], b[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int xq = x + G * q;
          a[q] = xq < n0 ? f[xq] : T(0);
          b[q] = xq < n0 ? c[(xq + ox) >> 1] : T(0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int xq = x + G * q;
          if (xq < n0) f[xq] = Ar<T>::add(a[q], b[q]);
        }
      }
    } else {
      for (int x = lane; x < n0; x += G) f[x] = Ar<T>::add(f[x], c[(x + ox) >> 1]);
    }
  });
}

// Trilinear form: fine(c) += e(c), e interpolated between the parent P (weight 3/4) and P's
// neighbour on c's side (1/4) in each dimension -- x, then y, then z, each step
// fma(1/4, b, 3/4 * a) -- from the coarse field's first ghost layer where P is a boundary
// cell of its box (filled beforehand).  G lanes per fine x-line.
template <class T>
__device__ __forceinline__ T lerp34(T a, T b) {
  return Ar<T>::fma(T(0.25), b, Ar<T>::mul(T(0.75), a));
}
template <class T, int G>
__global__ void __launch_bounds__(kThreads) k_prolong_trilinear(SegList L, long long nrows, long long per) {
  pdl_begin();
  const int lane = threadIdx.x & (G - 1);
  for_rows<32 / G>(L, nrows, per, [&](const DRow& R, long long lr, int) {
    const int n0 = R.n[0], n1 = R.n[1];
    const int y = (int)lr % n1, z = (int)lr / n1;
    const int ox = R.lo[0] & 1, oy = R.lo[1] & 1, oz = R.lo[2] & 1;
    T* f = line<T>(R.v[0], y, z);
    const T* c = line<T>(R.c[0], (y + oy) >> 1, (z + oz) >> 1);
    // the neighbouring coarse row / plane on this fine row's side of its parents
    const long long dy = ((y + oy) & 1) ? R.c[0].pitch : -(long long)R.c[0].pitch;
    const long long dz = ((z + oz) & 1) ? R.c[0].plane : -R.c[0].plane;
    for (int x = lane; x < n0; x += G) {
      const T* q = c + ((x + ox) >> 1);
      const int dx = ((x + ox) & 1) ? 1 : -1;
      const T ux00 = lerp34(q[0], q[dx]);
      const T ux10 = lerp34(q[dy], q[dy + dx]);
      const T ux01 = lerp34(q[dz], q[dz + dx]);
      const T ux11 = lerp34(q[dy + dz], q[dy + dz + dx]);
      f[x] = Ar<T>::add(f[x], lerp34(lerp34(ux00, ux10), lerp34(ux01, ux11)));
    }
  });
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_set_valid(SegList L, long long nrows, long long per,
                                                        T value) {
  pdl_begin();
  const int lane = threadIdx.x & 31;
  for_rows(L, nrows, per, [&](const DRow& R, long long lr, int) {
    const int n0 = R.n[0], n1 = R.n[1];
    const int y = (int)lr % n1, z = (int)lr / n1;
    T* f = line<T>(R.v[0], y, z);
    for (int x = lane; x < n0; x += 32) f[x] = value;
  });
}

// STREAM triad a = b + s c (one fma) on valid cells: the calibration kernel of Sec. 3.1-3.2,
// run either as one launch over all boxes or as one launch per box.  G lanes per x-line.
template <class T, int G>
__global__ void __launch_bounds__(kThreads) k_triad(SegList L, long long nrows, long long per, T s) {
  pdl_begin();
  const int lane = threadIdx.x & (G - 1);
  for_rows<32 / G>(L, nrows, per, [&](const DRow& R, long long lr, int) {
    const int n0 = R.n[0], n1 = R.n[1];
    const int y = (int)lr % n1, z = (int)lr / n1;
    T* __restrict__ a = line<T>(R.v[0], y, z);
    const T* __restrict__ b = line<T>(R.v[1], y, z);
    const T* __restrict__ c = line<T>(R.v[2], y, z);
    for (int x = lane; x < n0; x += G) a[x] = Ar<T>::fma(s, __ldg(c + x), __ldg(b + x));
  });
}

// FP64 throughput probe: 8 independent chains of fused multiply-adds per thread (a -> a b + c
// converges to c / (1 - b), so the values stay normal).  The result is stored only if it
// equals an impossible value, which keeps the chains alive without a memory write.
__device__ double g_probe_sink;
constexpr int kProbeChains = 8;
__global__ void __launch_bounds__(256) k_fp64_probe(int iters, double b, double c) {
  pdl_begin();
  double a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = 1e-3 * threadIdx.x + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = __fma_rn(a[k], b, c);
  }
  double s = a[0];
#pragma unroll
  for (int k = 1; k < kProbeChains; ++k) s = __dadd_rn(s, a[k]);
  if (s == -1.0) g_probe_sink = s;
}

// a += b on valid cells: v[0] = a, v[1] = b.
template <class T>
__global__ void __launch_bounds__(kThreads) k_add_valid(SegList L, long long nrows, long long per) {
  pdl_begin();
  const int lane = threadIdx.x & 31;
  for_rows(L, nrows, per, [&](const DRow& R, long long lr, int) {
    const int n0 = R.n[0], n1 = R.n[1];
    const int y = (int)lr % n1, z = (int)lr / n1;
    T* a = line<T>(R.v[0], y, z);
    const T* b = line<T>(R.v[1], y, z);
    for (int x = lane; x < n0; x += 32) a[x] = Ar<T>::add(a[x], b[x]);
  });
}

template <class T>
__global__ void k_set_flat(T* p, long long n, T value) {
  pdl_begin();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = value;
}

// Exact bottom solve: one block per job, rhs gathered to shared memory in FP64.
template <class T>
__global__ void k_bottom(const BottomJob* __restrict__ jobs) {
  pdl_begin();
  extern __shared__ double sb[];
  const BottomJob J = jobs[blockIdx.x];
  const T* rhs = (const T*)J.rhs;
  T* phi = (T*)J.phi;
  for (int j = threadIdx.x; j < J.N; j += blockDim.x) sb[j] = (double)rhs[J.off_rhs[j]];
  __syncthreads();
  for (int i = threadIdx.x; i < J.N; i += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < J.N; ++j) s = __dadd_rn(s, __dmul_rn(J.Mt[(long long)j * J.N + i], sb[j]));
    phi[J.off_phi[i]] = (T)s;
  }
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_dense_copy(SegList L, long long nrows, long long per,
                                                         T* dense, int3 dlo, int3 dn, int ncomp,
                                                         int to_dense) {
  pdl_begin();
  const int lane = threadIdx.x & 31;
  const long long dplane = (long long)dn.x * dn.y, dcomp = dplane * dn.z;
  for_rows(L, nrows, per, [&](const DRow& R, long long lr, int) {
    const int n0 = R.n[0], n1 = R.n[1];
    const int y = (int)lr % n1, z = (int)lr / n1;
    T* f = line<T>(R.v[0], y, z);
    T* d = dense + (long long)(R.lo[2] + z - dlo.z) * dplane +
           (long long)(R.lo[1] + y - dlo.y) * dn.x + (R.lo[0] - dlo.x);
    for (int c = 0; c < ncomp; ++c) {
      T* fc = f + c * R.v[0].cstride;
      T* dc = d + c * dcomp;
      if (to_dense) {
        for (int x = lane; x < n0; x += 32) dc[x] = fc[x];
      } else {
        for (int x = lane; x < n0; x += 32) fc[x] = dc[x];
      }
    }
  });
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_maxabs(SegList L, long long nrows, long long per,
                                                     unsigned long long* norms) {
  pdl_begin();
  const int lane = threadIdx.x & 31;
  unsigned long long mx = 0;
  int cur = -1;
  for_rows(L, nrows, per, [&](const DRow& R, long long lr, int slot) {
    const int idx = slot + R.solve;
    if (idx != cur) {
      if (cur >= 0) {
        unsigned long long m = Ar<T>::key_to_f64bits(warp_max(mx));
        if (lane == 0 && m) atomicMax(&norms[cur], m);
      }
      cur = idx;
      mx = 0;
    }
    const int n0 = R.n[0], n1 = R.n[1];
    const int y = (int)lr % n1, z = (int)lr / n1;
    const T* f = line<T>(R.v[0], y, z);
    for (int x = lane; x < n0; x += 32) {
      unsigned long long k = Ar<T>::abskey(f[x]);
      mx = k > mx ? k : mx;
    }
  });
  flush_block_max(Ar<T>::key_to_f64bits(warp_max(mx)), cur, norms);
}

__device__ __forceinline__ double norm_of(const unsigned long long* norms, int idx) {
  return __longlong_as_double((long long)norms[idx]);
}
// 2^e with 2^e <= s < 2^(e+1), and its inverse; both exact powers of two (bit operations)
__device__ __forceinline__ double pow2_floor(double s) { return bits::pow2(bits::floor_log2(s)); }
__device__ __forceinline__ double pow2_floor_inv(double s) { return bits::pow2(-bits::floor_log2(s)); }

// r32 = float(r * 2^-e) with 2^e <= ||r||_inf < 2^(e+1), from the FP64 residual stored by the
// preceding norm check (the same values the norm was taken over), and the FP32 correction's
// initial guess e32 = 0.  G lanes per x-line, kScaleCells cells per lane step, loads first
// (measured: 4 beats 8, which halves the lanes per row and the bytes per load instruction).
constexpr int kScaleCells = 4;
template <int G>
__global__ void __launch_bounds__(kThreads) k_scale_residual_f32(SegList L, long long nrows,
                                                                 long long per,
                                                                 const unsigned long long* norms) {
  pdl_begin();
  const int sub = threadIdx.x & (G - 1);
  for_rows<32 / G>(L, nrows, per, [&](const DRow& R, long long lr, int slot) {
    const int n0 = R.n[0], n1 = R.n[1];
    const int y = (int)lr % n1, z = (int)lr / n1;
    const double* __restrict__ r = line<double>(R.v[0], y, z);
    float* __restrict__ r32 = line<float>(R.c[0], y, z);
    float* __restrict__ e32 = line<float>(R.c[1], y, z);
    const double s = norm_of(norms, slot + R.solve);
    const int e = bits::floor_log2(s);
    const double down = pow2_floor_inv(s);
    for (int x = sub; x < n0; x += kScaleCells * G) {
      double v[kScaleCells];
#pragma unroll
      for (int k = 0; k < kScaleCells; ++k)
        if (x + G * k < n0) v[k] = __ldg(r + x + G * k);
#pragma unroll
      for (int k = 0; k < kScaleCells; ++k) {
        if (x + G * k >= n0) continue;
        // the exact scaling and the rounding in integer operations where they apply
        float f;
        if (!bits::scale_to_f32(v[k], e, &f)) f = __double2float_rn(__dmul_rn(v[k], down));
        r32[x + G * k] = f;
        e32[x + G * k] = 0.0f;
      }
    }
  });
}

// phi += 2^e * e32 (one rounding).  2^e * e32 is exact in binary64 (a float times a power of
// two), so where the bit form applies one rounded addition gives the fma's result.  G lanes
// per x-line, kCorrectCells cells per lane step, loads first (measured: 8 beats 4 here, 59
// against 62 us at 256^3).
constexpr int kCorrectCells = 8;
template <int G>
__global__ void __launch_bounds__(kThreads) k_correct_add(SegList L, long long nrows, long long per,
                                                          const unsigned long long* norms) {
  pdl_begin();
  const int sub = threadIdx.x & (G - 1);
  for_rows<32 / G>(L, nrows, per, [&](const DRow& R, long long lr, int slot) {
    const int n0 = R.n[0], n1 = R.n[1];
    const int y = (int)lr % n1, z = (int)lr / n1;
    double* __restrict__ phi = line<double>(R.v[0], y, z);
    const float* __restrict__ e = line<float>(R.c[0], y, z);
    const double s = norm_of(norms, slot + R.solve);
    const int ex = bits::floor_log2(s);
    const double up = pow2_floor(s);
    for (int x = sub; x < n0; x += kCorrectCells * G) {
      double p[kCorrectCells];
      float v[kCorrectCells];
#pragma unroll
      for (int k = 0; k < kCorrectCells; ++k)
        if (x + G * k < n0) {
          p[k] = phi[x + G * k];
          v[k] = __ldg(e + x + G * k);
        }
#pragma unroll
      for (int k = 0; k < kCorrectCells; ++k) {
        if (x + G * k >= n0) continue;
        double t;
        phi[x + G * k] = bits::scaled_f32_to_f64(v[k], ex, &t) ? __dadd_rn(p[k], t)
                                                               : __fma_rn(up, (double)v[k], p[k]);
      }
    }
  });
}

struct Grid {
  long long per;
  unsigned blocks;
};

// rows_per_pass: rows a block takes at once (kWarps x lane groups per warp); per is a
// multiple of it so that only a launch's last block has idle groups.
Grid row_grid(long long nrows, int blocks_per_sm, int rows_per_pass = kWarps) {
  long long target = (long long)num_sms() * blocks_per_sm;
  long long per = (nrows + target - 1) / target;
  per = (per + rows_per_pass - 1) / rows_per_pass * rows_per_pass;
  Grid g;
  g.per = per;
  g.blocks = (unsigned)((nrows + per - 1) / per);
  return g;
}

}  // namespace

static std::atomic<long long> g_launches{0};
void count_launches(long long n) { g_launches += n; }
bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("GBMG_NO_PDL");
    return !(e && e[0] == '1');
  }();
  return on;
}
long long launches_so_far() { return g_launches.load(); }

cudaError_t opt_in_smem(const void* kernel, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> opted;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t& o = opted[{kernel, dev}];
  if (smem <= o) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) o = smem;
  return e;
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 1;
  }
  return n;
}

#define GB_DISPATCH(dt, KERNEL, GRID, BLOCK, SMEM, STREAM, ...)                       \
  do {                                                                                 \
    if ((dt) == DT_F64) launch_k(KERNEL<double>, GRID, BLOCK, SMEM, STREAM, __VA_ARGS__);    \
    else launch_k(KERNEL<float>, GRID, BLOCK, SMEM, STREAM, __VA_ARGS__);                    \
  } while (0)
#define GB_DISPATCH_D(dt, direct, KERNEL, GRID, BLOCK, SMEM, STREAM, ...)                  \
  do {                                                                                   \
    if ((dt) == DT_F64) {                                                                \
      if (direct) launch_k(KERNEL<double, true>, GRID, BLOCK, SMEM, STREAM, __VA_ARGS__);       \
      else launch_k(KERNEL<double, false>, GRID, BLOCK, SMEM, STREAM, __VA_ARGS__);             \
    } else {                                                                             \
      if (direct) launch_k(KERNEL<float, true>, GRID, BLOCK, SMEM, STREAM, __VA_ARGS__);        \
      else launch_k(KERNEL<float, false>, GRID, BLOCK, SMEM, STREAM, __VA_ARGS__);              \
    }                                                                                    \
  } while (0)

cudaError_t launch_copy_tags_l(int dt, const TagList& L, long long nchunks, int ncomp, cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  unsigned blocks = (unsigned)((nchunks + 7) / 8);
  // 2 to 4 components: all components' loads first (measured on the 4-component microbench:
  // 99 us against 120 us per fill)
  const bool multi = ncomp > 1 && ncomp <= 4;
  if (dt == DT_F64) {
    if (ncomp == 1) launch_k(k_copy_tags<double, 1>, blocks, 256, 0, s, L, nchunks, ncomp);
    else if (multi) launch_k(k_copy_tags_multi<double>, blocks, 256, 0, s, L, nchunks, ncomp);
    else launch_k(k_copy_tags<double, 0>, blocks, 256, 0, s, L, nchunks, ncomp);
  } else {
    if (ncomp == 1) launch_k(k_copy_tags<float, 1>, blocks, 256, 0, s, L, nchunks, ncomp);
    else if (multi) launch_k(k_copy_tags_multi<float>, blocks, 256, 0, s, L, nchunks, ncomp);
    else launch_k(k_copy_tags<float, 0>, blocks, 256, 0, s, L, nchunks, ncomp);
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_copy_tags(int dt, const DTag* tags, const int2* chunks, int nchunks, void* base,
                             int ncomp, cudaStream_t s) {
  TagList L{};
  L.one.tags = tags;
  L.one.chunks = chunks;
  L.one.base = base;
  L.one.chunk_begin = 0;
  L.one.nchunks = nchunks;
  L.n = 1;
  return launch_copy_tags_l(dt, L, nchunks, ncomp, s);
}

namespace {
// Blocks per SM the stencil row kernels aim for (measured: 16 beats 8 and 4 on both the
// finest and the coarser levels).
constexpr int kRowBlocksPerSM = 16;
// Launches over boxes at most 32 cells wide (rows of a pass or two per block) take twice as
// many, smaller blocks: measured on GB300, 512 batched problems of 32^3 boxes 2045 -> 2090
// solves/s and the 512 x 32^3 triad 126 -> 120 us, with the 256^3 solve unchanged (4 or 8
// blocks per SM made both slower).
inline int row_blocks_per_sm(int width) {
  return width > 0 && width <= 32 ? 2 * kRowBlocksPerSM : kRowBlocksPerSM;
}

// Lanes per x-line for a launch whose widest line holds `width` cells (0 = unknown): the
// smallest group (of those the kernels are built for) whose lanes each get `cells`
// consecutive-pass cells at most, i.e. width / cells lanes rounded up.
int group_lanes(int width, int cells, int lo, int hi) {
  if (width <= 0) return hi;
  int g = lo;
  while (g < hi && g * cells < width) g *= 2;
  return g;
}

template <class T, bool DIRECT, int MODE = 0>
void rbgs_half_g(int G, const Grid& g, cudaStream_t s, const SegList& L, long long nrows, int color,
                 unsigned long long* norms) {
  if (G == 16) launch_k(k_rbgs_half<T, DIRECT, MODE, 16>, g.blocks, kThreads, 0, s, L, nrows, g.per, color, norms);
  else if (G == 8) launch_k(k_rbgs_half<T, DIRECT, MODE, 8>, g.blocks, kThreads, 0, s, L, nrows, g.per, color, norms);
  else launch_k(k_rbgs_half<T, DIRECT, MODE, 4>, g.blocks, kThreads, 0, s, L, nrows, g.per, color, norms);
}
template <class T, int MODE>
void rbgs_half_norm_g(int G, const Grid& g, cudaStream_t s, const SegList& L, long long nrows, int color,
                      unsigned long long* norms) {
  if (G == 16) launch_k(k_rbgs_half<T, true, MODE, 16>, g.blocks, kThreads, 0, s, L, nrows, g.per, color, norms);
  else launch_k(k_rbgs_half<T, true, MODE, 8>, g.blocks, kThreads, 0, s, L, nrows, g.per, color, norms);
}
}  // namespace

cudaError_t launch_rbgs_half_l(int dt, const SegList& L, long long nrows, int color, cudaStream_t s,
                               bool direct, unsigned long long* norms, bool pre) {
  if (nrows <= 0) return cudaSuccess;
  if (norms && (L.n != 1 || !direct)) return cudaErrorInvalidValue;
  if (pre && !norms) return cudaErrorInvalidValue;
  // a line of w cells holds w / 2 of one colour; two per lane (four on FP32 rows of 64 to
  // 127 cells)
  const bool quad = dt == DT_F32 && !norms && L.width >= 64 && L.width < 128;
  const int G = quad ? group_lanes(L.width, 8, 4, 16) : group_lanes(L.width, 4, norms ? 8 : 4, 16);
  const Grid g = row_grid(nrows, row_blocks_per_sm(L.width), kWarps * (32 / G));
  if (norms) {
    if (dt == DT_F64) {
      if (pre) rbgs_half_norm_g<double, 2>(G, g, s, L, nrows, color, norms);
      else rbgs_half_norm_g<double, 1>(G, g, s, L, nrows, color, norms);
    } else {
      if (pre) rbgs_half_norm_g<float, 2>(G, g, s, L, nrows, color, norms);
      else rbgs_half_norm_g<float, 1>(G, g, s, L, nrows, color, norms);
    }
  } else if (dt == DT_F64) {
    if (direct) rbgs_half_g<double, true>(G, g, s, L, nrows, color, norms);
    else rbgs_half_g<double, false>(G, g, s, L, nrows, color, norms);
  } else if (quad) {
    if (direct) rbgs_half_g<float, true, 4>(G, g, s, L, nrows, color, norms);
    else rbgs_half_g<float, false, 4>(G, g, s, L, nrows, color, norms);
  } else {
    if (direct) rbgs_half_g<float, true>(G, g, s, L, nrows, color, norms);
    else rbgs_half_g<float, false>(G, g, s, L, nrows, color, norms);
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_residual_l(int dt, const SegList& L, long long nrows, unsigned long long* norms,
                              cudaStream_t s, bool direct, int color) {
  if (nrows <= 0) return cudaSuccess;
  Grid g = row_grid(nrows, 16);
  GB_DISPATCH_D(dt, direct, k_residual, g.blocks, kThreads, 0, s, L, nrows, g.per, norms, color);
  count_launches(1);
  return cudaGetLastError();
}

namespace {
template <class T, bool DIRECT>
void residual_restrict_g(int G, const Grid& g, cudaStream_t s, const SegList& L, long long nrows) {
  if (G == 32) launch_k(k_residual_restrict<T, DIRECT, 32>, g.blocks, kThreads, 0, s, L, nrows, g.per);
  else if (G == 16) launch_k(k_residual_restrict<T, DIRECT, 16>, g.blocks, kThreads, 0, s, L, nrows, g.per);
  else launch_k(k_residual_restrict<T, DIRECT, 8>, g.blocks, kThreads, 0, s, L, nrows, g.per);
}
template <class T>
void prolong_add_g(int G, const Grid& g, cudaStream_t s, const SegList& L, long long nrows) {
  if (G == 32) launch_k(k_prolong_add<T, 32>, g.blocks, kThreads, 0, s, L, nrows, g.per);
  else if (G == 16) launch_k(k_prolong_add<T, 16>, g.blocks, kThreads, 0, s, L, nrows, g.per);
  else launch_k(k_prolong_add<T, 8>, g.blocks, kThreads, 0, s, L, nrows, g.per);
}
}  // namespace

cudaError_t launch_residual_restrict_l(int dt, const SegList& L, long long nrows, cudaStream_t s,
                                       bool direct, bool stored) {
  if (nrows <= 0) return cudaSuccess;
  // rows are coarse lines of width / 2 cells, one per lane
  const int G = group_lanes(L.width, 2, 8, 32);
  const Grid g = row_grid(nrows, row_blocks_per_sm(L.width), kWarps * (32 / G));
  if (stored) {
    if (dt != DT_F64 || !direct) return cudaErrorInvalidValue;
    if (G == 32) launch_k(k_residual_restrict<double, true, 32, true>, g.blocks, kThreads, 0, s, L, nrows, g.per);
    else if (G == 16) launch_k(k_residual_restrict<double, true, 16, true>, g.blocks, kThreads, 0, s, L, nrows, g.per);
    else launch_k(k_residual_restrict<double, true, 8, true>, g.blocks, kThreads, 0, s, L, nrows, g.per);
    count_launches(1);
    return cudaGetLastError();
  }
  if (dt == DT_F64) {
    if (direct) residual_restrict_g<double, true>(G, g, s, L, nrows);
    else residual_restrict_g<double, false>(G, g, s, L, nrows);
  } else {
    if (direct) residual_restrict_g<float, true>(G, g, s, L, nrows);
    else residual_restrict_g<float, false>(G, g, s, L, nrows);
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_prolong_trilinear_l(int dt, const SegList& L, long long nrows, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  const int G = group_lanes(L.width, 1, 8, 32);
  const Grid g = row_grid(nrows, row_blocks_per_sm(L.width), kWarps * (32 / G));
  if (dt == DT_F64) {
    if (G == 32) launch_k(k_prolong_trilinear<double, 32>, g.blocks, kThreads, 0, s, L, nrows, g.per);
    else if (G == 16) launch_k(k_prolong_trilinear<double, 16>, g.blocks, kThreads, 0, s, L, nrows, g.per);
    else launch_k(k_prolong_trilinear<double, 8>, g.blocks, kThreads, 0, s, L, nrows, g.per);
  } else {
    if (G == 32) launch_k(k_prolong_trilinear<float, 32>, g.blocks, kThreads, 0, s, L, nrows, g.per);
    else if (G == 16) launch_k(k_prolong_trilinear<float, 16>, g.blocks, kThreads, 0, s, L, nrows, g.per);
    else launch_k(k_prolong_trilinear<float, 8>, g.blocks, kThreads, 0, s, L, nrows, g.per);
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_prolong_add_l(int dt, const SegList& L, long long nrows, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  const int G = group_lanes(L.width, dt == DT_F64 ? 1 : 4, 8, 32);  // cells per lane step
  const Grid g = row_grid(nrows, row_blocks_per_sm(L.width), kWarps * (32 / G));
  if (dt == DT_F64) prolong_add_g<double>(G, g, s, L, nrows);
  else prolong_add_g<float>(G, g, s, L, nrows);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_triad_l(int dt, const SegList& L, long long nrows, double sc, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  const int G = group_lanes(L.width, 1, 8, 32);
  const Grid g = row_grid(nrows, row_blocks_per_sm(L.width), kWarps * (32 / G));
  if (dt == DT_F64) {
    if (G == 32) launch_k(k_triad<double, 32>, g.blocks, kThreads, 0, s, L, nrows, g.per, sc);
    else if (G == 16) launch_k(k_triad<double, 16>, g.blocks, kThreads, 0, s, L, nrows, g.per, sc);
    else launch_k(k_triad<double, 8>, g.blocks, kThreads, 0, s, L, nrows, g.per, sc);
  } else {
    const float f = (float)sc;
    if (G == 32) launch_k(k_triad<float, 32>, g.blocks, kThreads, 0, s, L, nrows, g.per, f);
    else if (G == 16) launch_k(k_triad<float, 16>, g.blocks, kThreads, 0, s, L, nrows, g.per, f);
    else launch_k(k_triad<float, 8>, g.blocks, kThreads, 0, s, L, nrows, g.per, f);
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fp64_probe(int iters, long long* lane_ops, cudaStream_t s) {
  if (iters < 1) return cudaErrorInvalidValue;
  const int blocks = num_sms() * 8;
  launch_k(k_fp64_probe, blocks, 256, 0, s, iters, 0.999999, 1e-7);
  if (lane_ops) *lane_ops = (long long)blocks * 256 * kProbeChains * iters;
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_set_valid_l(int dt, const SegList& L, long long nrows, double value, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  Grid g = row_grid(nrows, 16);
  if (dt == DT_F64) launch_k(k_set_valid<double>, g.blocks, kThreads, 0, s, L, nrows, g.per, value);
  else launch_k(k_set_valid<float>, g.blocks, kThreads, 0, s, L, nrows, g.per, (float)value);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_maxabs_l(int dt, const SegList& L, long long nrows, unsigned long long* norms,
                            cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  Grid g = row_grid(nrows, 4);
  GB_DISPATCH(dt, k_maxabs, g.blocks, kThreads, 0, s, L, nrows, g.per, norms);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_scale_residual_f32_l(const SegList& L, long long nrows,
                                        const unsigned long long* norms, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  const int G = group_lanes(L.width, kScaleCells, 8, 32);
  const Grid g = row_grid(nrows, row_blocks_per_sm(L.width), kWarps * (32 / G));
  if (G == 32) launch_k(k_scale_residual_f32<32>, g.blocks, kThreads, 0, s, L, nrows, g.per, norms);
  else if (G == 16) launch_k(k_scale_residual_f32<16>, g.blocks, kThreads, 0, s, L, nrows, g.per, norms);
  else launch_k(k_scale_residual_f32<8>, g.blocks, kThreads, 0, s, L, nrows, g.per, norms);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_correct_add_l(const SegList& L, long long nrows, const unsigned long long* norms,
                                 cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  const int G = group_lanes(L.width, kCorrectCells, 8, 32);
  const Grid g = row_grid(nrows, row_blocks_per_sm(L.width), kWarps * (32 / G));
  if (G == 32) launch_k(k_correct_add<32>, g.blocks, kThreads, 0, s, L, nrows, g.per, norms);
  else if (G == 16) launch_k(k_correct_add<16>, g.blocks, kThreads, 0, s, L, nrows, g.per, norms);
  else launch_k(k_correct_add<8>, g.blocks, kThreads, 0, s, L, nrows, g.per, norms);
  count_launches(1);
  return cudaGetLastError();
}

// ---- single-table launchers (one segment) ------------------------------------------------

cudaError_t launch_rbgs_half(int dt, const DRow* rows, int nbox, long long nrows, int color,
                             cudaStream_t s, bool direct, unsigned long long* norms, int width,
                             bool pre) {
  return launch_rbgs_half_l(dt, one_seg(rows, nbox, 0, width), nrows, color, s, direct, norms, pre);
}

cudaError_t launch_restore_colour(int dt, const DRow* rows, int nbox, long long nrows, int color,
                                  cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  Grid g = row_grid(nrows, 16);
  GB_DISPATCH(dt, k_restore_colour, g.blocks, kThreads, 0, s, one_seg(rows, nbox), nrows, g.per, color);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_residual(int dt, const DRow* rows, int nbox, long long nrows,
                            unsigned long long* norms, cudaStream_t s, bool direct, int color) {
  return launch_residual_l(dt, one_seg(rows, nbox), nrows, norms, s, direct, color);
}

cudaError_t launch_residual_restrict(int dt, const DRow* rows, int nbox, long long nrows,
                                     cudaStream_t s, bool direct, int width, bool stored) {
  return launch_residual_restrict_l(dt, one_seg(rows, nbox, 0, width), nrows, s, direct, stored);
}

cudaError_t launch_rbgs_half_store(const DRow* rows, int nbox, long long nrows, int color,
                                   cudaStream_t s, int width) {
  if (nrows <= 0) return cudaSuccess;
  const SegList L = one_seg(rows, nbox, 0, width);
  const int G = group_lanes(L.width, 4, 8, 16);
  const Grid g = row_grid(nrows, row_blocks_per_sm(L.width), kWarps * (32 / G));
  rbgs_half_norm_g<double, 3>(G, g, s, L, nrows, color, nullptr);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_restrict(int dt, const DRow* rows, int nbox, long long nrows, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  Grid g = row_grid(nrows, 16);
  GB_DISPATCH(dt, k_restrict, g.blocks, kThreads, 0, s, one_seg(rows, nbox), nrows, g.per);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_prolong_add(int dt, const DRow* rows, int nbox, long long nrows,
                               cudaStream_t s, int width) {
  return launch_prolong_add_l(dt, one_seg(rows, nbox, 0, width), nrows, s);
}

cudaError_t launch_prolong_trilinear(int dt, const DRow* rows, int nbox, long long nrows,
                                     cudaStream_t s, int width) {
  return launch_prolong_trilinear_l(dt, one_seg(rows, nbox, 0, width), nrows, s);
}

cudaError_t launch_bottom(int dt, const BottomJob* jobs, int njobs, int maxN, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  int threads = maxN < 32 ? 32 : (maxN > 1024 ? 1024 : (maxN + 31) / 32 * 32);
  size_t smem = (size_t)maxN * sizeof(double);
  if (dt == DT_F64) launch_k(k_bottom<double>, njobs, threads, smem, s, jobs);
  else launch_k(k_bottom<float>, njobs, threads, smem, s, jobs);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_add_valid(int dt, const DRow* rows, int nbox, long long nrows, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  Grid g = row_grid(nrows, 16);
  GB_DISPATCH(dt, k_add_valid, g.blocks, kThreads, 0, s, one_seg(rows, nbox), nrows, g.per);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_set_valid(int dt, const DRow* rows, int nbox, long long nrows, double value,
                             cudaStream_t s) {
  return launch_set_valid_l(dt, one_seg(rows, nbox), nrows, value, s);
}

cudaError_t launch_set_flat(int dt, void* p, long long n, double value, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  long long cap = (long long)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  if (dt == DT_F64) launch_k(k_set_flat<double>, (unsigned)blocks, 256, 0, s, (double*)p, n, value);
  else launch_k(k_set_flat<float>, (unsigned)blocks, 256, 0, s, (float*)p, n, (float)value);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_dense_copy(int dt, const DRow* rows, int nbox, long long nrows, void* dense,
                              const int dom_lo[3], const int dom_n[3], int ncomp, int to_dense,
                              cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  Grid g = row_grid(nrows, 16);
  int3 lo = make_int3(dom_lo[0], dom_lo[1], dom_lo[2]);
  int3 n = make_int3(dom_n[0], dom_n[1], dom_n[2]);
  if (dt == DT_F64)
    launch_k(k_dense_copy<double>, g.blocks, kThreads, 0, s, one_seg(rows, nbox), nrows, g.per, (double*)dense, lo, n, ncomp, to_dense);
  else
    launch_k(k_dense_copy<float>, g.blocks, kThreads, 0, s, one_seg(rows, nbox), nrows, g.per, (float*)dense, lo, n, ncomp, to_dense);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_maxabs(int dt, const DRow* rows, int nbox, long long nrows,
                          unsigned long long* norms, cudaStream_t s) {
  return launch_maxabs_l(dt, one_seg(rows, nbox), nrows, norms, s);
}

cudaError_t launch_scale_residual_f32(const DRow* rows, int nbox, long long nrows,
                                      const unsigned long long* norms, cudaStream_t s, int width) {
  return launch_scale_residual_f32_l(one_seg(rows, nbox, 0, width), nrows, norms, s);
}

cudaError_t launch_correct_add(const DRow* rows, int nbox, long long nrows,
                               const unsigned long long* norms, cudaStream_t s, int width) {
  return launch_correct_add_l(one_seg(rows, nbox, 0, width), nrows, norms, s);
}

}  // namespace gbmg
