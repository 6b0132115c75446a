// The coarse end of the V-cycle in one launch.
//
// Below a few thousand cells a level's stage kernels finish in a microsecond or two, so the
// cycle there is bound by launch latency (about 20 dependent launches per level).  This
// kernel runs the whole sub-cycle from level lc down to the bottom and back inside ONE CTA:
// each level is copied into shared memory as a single dense box with one ghost layer
// (results of this multigrid are independent of the box decomposition), and every stage --
// face ghost fill, red and black half-sweeps, fused residual + restriction, exact bottom
// solve, prolongation -- is the same arithmetic, in the same order, as the per-stage
// kernels, so the result is bit-identical to the multi-launch path.
#include <cuda_runtime.h>

#include <mutex>

#include "mg_kernels.hpp"

namespace gbmg {

namespace {

template <class T>
struct A;
template <>
struct A<double> {
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
  static __device__ __forceinline__ double neg(double a) {
    return __longlong_as_double(__double_as_longlong(a) ^ (long long)0x8000000000000000ull);
  }
};
template <>
struct A<float> {
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
  static __device__ __forceinline__ float neg(float a) {
    return __int_as_float(__float_as_int(a) ^ (int)0x80000000u);
  }
};

template <class T>
__device__ __forceinline__ T gs_update(T s, T rhs, T h2) {
  constexpr T inv6 = T(1) / T(6);
  return A<T>::mul(A<T>::fma(A<T>::neg(h2), rhs, s), inv6);
}
template <class T>
__device__ __forceinline__ T residual_of(T s, T phi, T rhs, T ih2) {
  return A<T>::fma(A<T>::neg(ih2), A<T>::fma(T(-6), phi, s), rhs);
}

// Dense level in shared memory: phi with one ghost layer, rhs without.
template <class T>
struct Lev {
  T* phi;
  T* rhs;
  int n0, n1, n2, p0, p1;  // extents; p0 = n0 + 2, p1 = n1 + 2
  int lo;                  // lo0 + lo1 + lo2 of the level domain (colour parity)
  T h2, ih2;
  __device__ __forceinline__ int at(int x, int y, int z) const {
    return ((z + 1) * p1 + (y + 1)) * p0 + (x + 1);
  }
  __device__ __forceinline__ int cells() const { return n0 * n1 * n2; }
};

template <class T>
__device__ __forceinline__ T nsum(const Lev<T> L, int o) {
  const int pl = L.p0 * L.p1;
  T s = L.phi[o - 1];
  s = A<T>::add(s, L.phi[o + 1]);
  s = A<T>::add(s, L.phi[o - L.p0]);
  s = A<T>::add(s, L.phi[o + L.p0]);
  s = A<T>::add(s, L.phi[o - pl]);
  s = A<T>::add(s, L.phi[o + pl]);
  return s;
}

// Face ghosts of a single box covering the level domain: periodic image or -(mirror).
template <class T>
__device__ void fill_faces(const Lev<T> L, const int3 per) {
  const int periodic[3] = {per.x, per.y, per.z};
  const int n[3] = {L.n0, L.n1, L.n2};
  for (int d = 0; d < 3; ++d) {
    const int a = d == 0 ? 1 : 0, b = d == 2 ? 1 : 2;  // the two other dimensions
    const int na = n[a], nb = n[b];
    for (int t = threadIdx.x; t < 2 * na * nb; t += blockDim.x) {
      const int side = t / (na * nb), r = t % (na * nb);
      int c[3];
      c[a] = r % na;
      c[b] = r / na;
      c[d] = side ? n[d] : -1;                       // ghost
      int m[3] = {c[0], c[1], c[2]};
      if (periodic[d]) m[d] = side ? 0 : n[d] - 1;    // image
      else m[d] = side ? n[d] - 1 : 0;                // mirror
      T v = L.phi[L.at(m[0], m[1], m[2])];
      L.phi[L.at(c[0], c[1], c[2])] = periodic[d] ? v : A<T>::neg(v);
    }
  }
}

// Threads are mapped to the cells of one colour only (x = x0 + 2k on each line), so no lane
// of an issued FP64 instruction is idle.
template <class T>
__device__ void half_sweep(const Lev<T> L, int color) {
  const int hx = (L.n0 + 1) >> 1;
  const int nt = hx * L.n1 * L.n2;
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    const int k = t % hx, r = t / hx, y = r % L.n1, z = r / L.n1;
    const int x = ((color + L.lo + y + z) & 1) + 2 * k;
    if (x >= L.n0) continue;
    const int o = L.at(x, y, z);
    L.phi[o] = gs_update(nsum(L, o), L.rhs[(z * L.n1 + y) * L.n0 + x], L.h2);
  }
}

template <class T>
__device__ void smooth(const Lev<T> L, const int3 periodic, int sweeps) {
  for (int s = 0; s < sweeps; ++s)
    for (int color = 0; color < 2; ++color) {
      fill_faces(L, periodic);
      __syncthreads();
      half_sweep(L, color);
      __syncthreads();
    }
}

// rhs of C = mean of the 8 child residuals of F (x fastest); phi of C = 0.
template <class T>
__device__ void residual_restrict(const Lev<T> F, const Lev<T> C) {
  const int nc = C.cells();
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    const int X = i % C.n0, q = i / C.n0, Y = q % C.n1, Z = q / C.n1;
    T acc = T(0);
    for (int k = 0; k < 2; ++k)
      for (int j = 0; j < 2; ++j)
        for (int ii = 0; ii < 2; ++ii) {
          const int x = 2 * X + ii, y = 2 * Y + j, z = 2 * Z + k;
          const int o = F.at(x, y, z);
          const T v = residual_of(nsum(F, o), F.phi[o], F.rhs[(z * F.n1 + y) * F.n0 + x], F.ih2);
          acc = (ii | j | k) ? A<T>::add(acc, v) : v;
        }
    C.rhs[i] = A<T>::mul(acc, (T)0.125);
    C.phi[C.at(X, Y, Z)] = T(0);
  }
}

template <class T>
__device__ void prolong_add(const Lev<T> C, const Lev<T> F) {
  const int nf = F.cells();
  for (int i = threadIdx.x; i < nf; i += blockDim.x) {
    const int x = i % F.n0, q = i / F.n0, y = q % F.n1, z = q / F.n1;
    const int o = F.at(x, y, z);
    F.phi[o] = A<T>::add(F.phi[o], C.phi[C.at(x >> 1, y >> 1, z >> 1)]);
  }
}

template <class T>
__device__ void bottom(const Lev<T> B, const double* __restrict__ Mt, int N) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < N; ++j) s = __dadd_rn(s, __dmul_rn(Mt[(long long)j * N + i], (double)B.rhs[j]));
    const int x = i % B.n0, q = i / B.n0, y = q % B.n1, z = q / B.n1;
    B.phi[B.at(x, y, z)] = (T)s;
  }
}

// 512 threads for FP64 (128 registers each), 1024 for FP32.
template <class T>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : 1024, 1) k_coarse_cycle(const CoarseJob* __restrict__ jobs) {
  pdl_begin();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Lev<T> L[kMaxCoarseLevels];
  const CoarseJob& J = jobs[blockIdx.x];
  T* arena = (T*)smem_raw;
  const int nl = J.nlev;
  const int3 per = make_int3(J.periodic[0], J.periodic[1], J.periodic[2]);
  if (threadIdx.x < nl) {
    const CoarseLevel& c = J.lev[threadIdx.x];
    Lev<T> v;
    v.phi = arena + c.off_phi;
    v.rhs = arena + c.off_rhs;
    v.n0 = c.n[0];
    v.n1 = c.n[1];
    v.n2 = c.n[2];
    v.p0 = c.n[0] + 2;
    v.p1 = c.n[1] + 2;
    v.lo = c.lo[0] + c.lo[1] + c.lo[2];
    v.h2 = (T)c.h2;
    v.ih2 = (T)c.ih2;
    L[threadIdx.x] = v;
  }
  __syncthreads();
  // gather phi (the current guess) and rhs of level lc
  T* const gphi = (T*)J.phi;
  const T* const grhs = (const T*)J.rhs;
  {
    const Lev<T> F = L[0];
    const int nc = F.cells();
    for (int i = threadIdx.x; i < nc; i += blockDim.x) {
      const int x = i % F.n0, q = i / F.n0, y = q % F.n1, z = q / F.n1;
      F.rhs[i] = grhs[J.off_rhs[i]];
      F.phi[F.at(x, y, z)] = gphi[J.off_phi[i]];
    }
  }
  __syncthreads();
  for (int k = 0; k + 1 < nl; ++k) {
    smooth(L[k], per, J.nu1);
    fill_faces(L[k], per);
    __syncthreads();
    residual_restrict(L[k], L[k + 1]);
    __syncthreads();
  }
  bottom(L[nl - 1], J.Mt, J.N);
  __syncthreads();
  for (int k = nl - 2; k >= 0; --k) {
    prolong_add(L[k + 1], L[k]);
    __syncthreads();
    smooth(L[k], per, J.nu2);
  }
  // scatter phi of level lc back
  {
    const Lev<T> F = L[0];
    const int nc = F.cells();
    for (int i = threadIdx.x; i < nc; i += blockDim.x) {
      const int x = i % F.n0, q = i / F.n0, y = q % F.n1, z = q / F.n1;
      gphi[J.off_phi[i]] = F.phi[F.at(x, y, z)];
    }
  }
}

}  // namespace

size_t coarse_smem_bytes(int dt, const int (*n)[3], int nlev) {
  size_t es = dt == DT_F64 ? 8 : 4, elems = 0;
  for (int k = 0; k < nlev; ++k)
    elems += (size_t)(n[k][0] + 2) * (n[k][1] + 2) * (n[k][2] + 2) + (size_t)n[k][0] * n[k][1] * n[k][2];
  return elems * es;
}

cudaError_t coarse_opt_in(int dt, size_t smem) {
  return dt == DT_F64 ? opt_in_smem((const void*)k_coarse_cycle<double>, smem)
                      : opt_in_smem((const void*)k_coarse_cycle<float>, smem);
}

cudaError_t launch_coarse_cycle(int dt, const CoarseJob* jobs, int njobs, size_t smem,
                                cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  if (smem > kCoarseSmemMax) return cudaErrorInvalidValue;
  cudaError_t e = coarse_opt_in(dt, smem);
  if (e != cudaSuccess) return e;
  if (dt == DT_F64) launch_k(k_coarse_cycle<double>, njobs, 512, smem, s, jobs);
  else launch_k(k_coarse_cycle<float>, njobs, 1024, smem, s, jobs);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace gbmg
