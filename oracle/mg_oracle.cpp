// Oracle for the cell-centered multigrid Poisson path -- TEST INFRASTRUCTURE ONLY.
//
// This file is the plain, slow, obviously correct CPU restatement that the CUDA path is
// checked against.  Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
// reference legs may load it.  It shares no code, header or table with the CUDA library.
//
// What it computes (paper: AMReX/pyAMReX review, arXiv 2403.12179):
//   * Sec. 2 names "linear solvers for cell-centered and nodal data" and ghost cell exchange
//     as a cached communication pattern; Sec. 3.4 names fused max/sum reductions.  The paper
//     describes no solver algorithm, so every numerical choice below is a stated reading:
//       - 7-point Laplacian, (A phi)_c = (sum of 6 neighbours - 6 phi_c) / h^2, solve A phi = rhs
//       - periodic faces: ghost = value of the periodic image
//       - homogeneous Dirichlet faces: ghost = -(mirror cell across the face); a ghost cell
//         outside the domain in two or more non-periodic directions is 0
//       - red-black Gauss-Seidel, colour (i+j+k) mod 2 on global indices, red (0) first,
//         ghost fill before each colour, sum order x-,x+,y-,y+,z-,z+; the update is
//         phi = fma(-h^2, rhs, s) * (1/6) with 1/6 rounded once
//       - residual r = fma(-1/h^2, fma(-6, phi, s), rhs), max-norm
//       - restriction = mean of the 8 children (x fastest sum order), coarse guess 0,
//         coarse operator rediscretised with h_{l+1} = 2 h_l
//       - prolongation = piecewise-constant injection added to phi (default), or trilinear:
//         weights 3/4 (parent) and 1/4 (its neighbour towards the fine cell) per dimension,
//         applied x, then y, then z, each step fma(1/4, b, 3/4 * a), from filled coarse ghosts
//       - bottom = exact solve by the closed-form (pseudo-)inverse built from the discrete
//         sine / Fourier eigenvectors of the 1-D operators
//       - V(nu1, nu2) cycle, stop when ||rhs - A phi||_inf <= tol ||rhs||_inf
//       - mixed form: FP64 outer residual / correction, FP32 inner V-cycle on r * 2^-e with
//         2^e <= ||r||_inf < 2^(e+1) (an exact rescaling), FP64 bottom,
//         phi = fma(2^e, e_inner, phi)
//   * Parity of these functions is pinned by mathematics, not by the paper: closed-form
//     eigenvalues, a dense brute-force solve, transfer identities, decomposition
//     invariance and second-order convergence (tests/test_oracle_pins.py).
//
// Data layout (oracle's own): a level's field is the concatenation of one array per box,
// each (nx+2g)(ny+2g)(nz+2g) per component, x fastest, then y, z, component; no padding.
// Box bounds are inclusive global indices (lo, hi).
//
// Compiled with -ffp-contract=off so every + - * / is a single IEEE-rounded operation.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <cstdio>
#include <vector>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int kMaxBottomCells = 1024;

struct Box {
  int lo[3];
  int hi[3];
};

inline int ext(const Box& b, int d) { return b.hi[d] - b.lo[d] + 1; }
inline long long npts(const Box& b) { return (long long)ext(b, 0) * ext(b, 1) * ext(b, 2); }

// Floor division and non-negative modulo for possibly negative global indices.
inline int floordiv2(int a) { return (a >= 0) ? a / 2 : -((-a + 1) / 2); }
inline int pmod(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

struct Level {
  int dlo[3], dhi[3];
  int periodic[3];
  double h;
  std::vector<Box> boxes;
  std::vector<int> owner;  // owner box of every domain cell (x fastest)
};

inline int dext(const Level& L, int d) { return L.dhi[d] - L.dlo[d] + 1; }

inline long long dom_index(const Level& L, int x, int y, int z) {
  return ((long long)(z - L.dlo[2]) * dext(L, 1) + (y - L.dlo[1])) * dext(L, 0) + (x - L.dlo[0]);
}

// Owner map: every domain cell records which box holds it.  Fails if boxes overlap, leave
// the domain, or leave a hole.
bool build_owner(Level& L) {
  long long n = (long long)dext(L, 0) * dext(L, 1) * dext(L, 2);
  L.owner.assign(n, -1);
  for (size_t b = 0; b < L.boxes.size(); ++b) {
    const Box& B = L.boxes[b];
    for (int d = 0; d < 3; ++d)
      if (B.lo[d] < L.dlo[d] || B.hi[d] > L.dhi[d] || B.lo[d] > B.hi[d]) return false;
    for (int z = B.lo[2]; z <= B.hi[2]; ++z)
      for (int y = B.lo[1]; y <= B.hi[1]; ++y)
        for (int x = B.lo[0]; x <= B.hi[0]; ++x) {
          long long i = dom_index(L, x, y, z);
          if (L.owner[i] != -1) return false;
          L.owner[i] = (int)b;
        }
  }
  for (long long i = 0; i < n; ++i)
    if (L.owner[i] < 0) return false;
  return true;
}

// Per-box offsets of a field with ng ghosts and nc components.
std::vector<long long> fab_offsets(const Level& L, int ng, int nc) {
  std::vector<long long> off(L.boxes.size() + 1, 0);
  for (size_t b = 0; b < L.boxes.size(); ++b) {
    const Box& B = L.boxes[b];
    long long sz = (long long)(ext(B, 0) + 2 * ng) * (ext(B, 1) + 2 * ng) * (ext(B, 2) + 2 * ng) * nc;
    off[b + 1] = off[b] + sz;
  }
  return off;
}

inline long long cell(const Box& B, int ng, int x, int y, int z, int c) {
  long long sx = ext(B, 0) + 2 * ng, sy = ext(B, 1) + 2 * ng, sz = ext(B, 2) + 2 * ng;
  return (((long long)c * sz + (z - B.lo[2] + ng)) * sy + (y - B.lo[1] + ng)) * sx + (x - B.lo[0] + ng);
}

template <class R>
struct Field {
  const Level* L;
  int ng, nc;
  std::vector<long long> off;
  R* data;
  R& at(int b, int x, int y, int z, int c = 0) const {
    return data[off[b] + cell(L->boxes[b], ng, x, y, z, c)];
  }
};

template <class R>
Field<R> make_field(const Level& L, int ng, int nc, R* data) {
  Field<R> f;
  f.L = &L; f.ng = ng; f.nc = nc; f.off = fab_offsets(L, ng, nc); f.data = data;
  return f;
}

// ---------------------------------------------------------------------------------------
// Ghost fill (Sec. 2: ghost cell exchange).  Brute force: every ghost cell looks up the box
// that owns its (periodically wrapped) position in the owner map.  Reading from valid cells
// only, so the order in which ghosts are written does not matter.
template <class R>
bool fill(const Field<R>& f) {
  const Level& L = *f.L;
  const int ng = f.ng;
  for (int d = 0; d < 3; ++d)
    if (!L.periodic[d] && ng > dext(L, d)) return false;  // mirror would leave the domain
  bool ok = true;
#pragma omp parallel for schedule(dynamic)
  for (long long b = 0; b < (long long)L.boxes.size(); ++b) {
    const Box& B = L.boxes[b];
    for (int z = B.lo[2] - ng; z <= B.hi[2] + ng; ++z)
      for (int y = B.lo[1] - ng; y <= B.hi[1] + ng; ++y)
        for (int x = B.lo[0] - ng; x <= B.hi[0] + ng; ++x) {
          bool inside = x >= B.lo[0] && x <= B.hi[0] && y >= B.lo[1] && y <= B.hi[1] &&
                        z >= B.lo[2] && z <= B.hi[2];
          if (inside) continue;
          int p[3] = {x, y, z};
          int nout = 0, od = -1;
          for (int d = 0; d < 3; ++d) {
            if (L.periodic[d]) {
              p[d] = L.dlo[d] + pmod(p[d] - L.dlo[d], dext(L, d));
            } else if (p[d] < L.dlo[d] || p[d] > L.dhi[d]) {
              ++nout;
              od = d;
            }
          }
          for (int c = 0; c < f.nc; ++c) {
            R v;
            if (nout == 0) {
              int s = L.owner[dom_index(L, p[0], p[1], p[2])];
              v = f.at(s, p[0], p[1], p[2], c);
            } else if (nout == 1) {
              int q[3] = {p[0], p[1], p[2]};
              q[od] = (p[od] < L.dlo[od]) ? 2 * L.dlo[od] - 1 - p[od] : 2 * L.dhi[od] + 1 - p[od];
              int s = L.owner[dom_index(L, q[0], q[1], q[2])];
              v = -f.at(s, q[0], q[1], q[2], c);
            } else {
              v = (R)0;
            }
            f.at((int)b, x, y, z, c) = v;
          }
        }
  }
  return ok;
}

// Sum of the six neighbours in the fixed order x-, x+, y-, y+, z-, z+.
template <class R>
inline R nbr_sum(const Field<R>& f, int b, int x, int y, int z) {
  R s = f.at(b, x - 1, y, z);
  s = s + f.at(b, x + 1, y, z);
  s = s + f.at(b, x, y - 1, z);
  s = s + f.at(b, x, y + 1, z);
  s = s + f.at(b, x, y, z - 1);
  s = s + f.at(b, x, y, z + 1);
  return s;
}

// One red-black Gauss-Seidel half-sweep of colour `color` (0 = red): every cell with
// (x+y+z) mod 2 == color takes phi = (s - h^2 rhs) / 6, evaluated as
// fma(-h^2, rhs, s) * (1/6).  phi's ghosts must be filled.
template <class R>
void rbgs(const Field<R>& phi, const Field<R>& rhs, int color) {
  const Level& L = *phi.L;
  const R h2 = (R)(L.h * L.h);
  const R inv6 = R(1) / R(6);
#pragma omp parallel for schedule(dynamic)
  for (long long b = 0; b < (long long)L.boxes.size(); ++b) {
    const Box& B = L.boxes[b];
    for (int z = B.lo[2]; z <= B.hi[2]; ++z)
      for (int y = B.lo[1]; y <= B.hi[1]; ++y)
        for (int x = B.lo[0]; x <= B.hi[0]; ++x) {
          if (pmod(x + y + z, 2) != color) continue;
          R s = nbr_sum(phi, (int)b, x, y, z);
          phi.at((int)b, x, y, z) = std::fma(-h2, rhs.at((int)b, x, y, z), s) * inv6;
        }
  }
}

// Residual r = rhs - (s - 6 phi) / h^2, evaluated as fma(-1/h^2, fma(-6, phi, s), rhs), on
// valid cells (r may be null); returns
// max |r| (NaN if any residual is NaN).  phi's ghosts must be filled.
template <class R>
double residual(const Field<R>& phi, const Field<R>& rhs, const Field<R>* r) {
  const Level& L = *phi.L;
  const R ih2 = (R)(1.0 / (L.h * L.h));
  double mx = 0.0;
  bool nan = false;
#pragma omp parallel for schedule(dynamic) reduction(max : mx) reduction(|| : nan)
  for (long long b = 0; b < (long long)L.boxes.size(); ++b) {
    const Box& B = L.boxes[b];
    for (int z = B.lo[2]; z <= B.hi[2]; ++z)
      for (int y = B.lo[1]; y <= B.hi[1]; ++y)
        for (int x = B.lo[0]; x <= B.hi[0]; ++x) {
          R s = nbr_sum(phi, (int)b, x, y, z);
          R v = std::fma(-ih2, std::fma((R)-6, phi.at((int)b, x, y, z), s), rhs.at((int)b, x, y, z));
          if (r) r->at((int)b, x, y, z) = v;
          double a = std::fabs((double)v);
          if (std::isnan(a)) nan = true;
          if (a > mx) mx = a;
        }
  }
  return nan ? NAN : mx;
}

// Restriction: coarse(I) = (sum of the 8 children, x fastest) * 1/8.  Children are found
// through the fine owner map.
template <class R>
void restrict_avg(const Field<R>& fine, const Field<R>& coarse) {
  const Level& F = *fine.L;
  const Level& C = *coarse.L;
#pragma omp parallel for schedule(dynamic)
  for (long long b = 0; b < (long long)C.boxes.size(); ++b) {
    const Box& B = C.boxes[b];
    for (int Z = B.lo[2]; Z <= B.hi[2]; ++Z)
      for (int Y = B.lo[1]; Y <= B.hi[1]; ++Y)
        for (int X = B.lo[0]; X <= B.hi[0]; ++X) {
          R s = (R)0;
          bool first = true;
          for (int k = 0; k < 2; ++k)
            for (int j = 0; j < 2; ++j)
              for (int i = 0; i < 2; ++i) {
                int x = 2 * X + i, y = 2 * Y + j, z = 2 * Z + k;
                int o = F.owner[dom_index(F, x, y, z)];
                R v = fine.at(o, x, y, z);
                s = first ? v : s + v;
                first = false;
              }
          coarse.at((int)b, X, Y, Z) = s * (R)0.125;
        }
  }
}

// Prolongation: phi_fine(c) += e_coarse(parent(c)), piecewise constant.
template <class R>
void prolong_add(const Field<R>& coarse, const Field<R>& fine) {
  const Level& F = *fine.L;
  const Level& C = *coarse.L;
#pragma omp parallel for schedule(dynamic)
  for (long long b = 0; b < (long long)F.boxes.size(); ++b) {
    const Box& B = F.boxes[b];
    for (int z = B.lo[2]; z <= B.hi[2]; ++z)
      for (int y = B.lo[1]; y <= B.hi[1]; ++y)
        for (int x = B.lo[0]; x <= B.hi[0]; ++x) {
          int X = floordiv2(x), Y = floordiv2(y), Z = floordiv2(z);
          int o = C.owner[dom_index(C, X, Y, Z)];
          fine.at((int)b, x, y, z) = fine.at((int)b, x, y, z) + coarse.at(o, X, Y, Z);
        }
  }
}

// Trilinear prolongation: phi_fine(c) += e(c), where e interpolates the coarse correction
// linearly in each dimension between the parent P (weight 3/4) and P's neighbour on c's side
// (weight 1/4) -- the cell-centred linear interpolation, fine centres lying a quarter of a
// coarse cell from P's centre.  Dimension by dimension, x then y then z, each step
// lerp(a, b) = fma(1/4, b, 3/4 * a).  Reads the coarse ghosts as they are (fill first).
template <class R>
R lerp34(R a, R b) { return std::fma((R)0.25, b, (R)0.75 * a); }

template <class R>
void prolong_add_trilinear(const Field<R>& coarse, const Field<R>& fine) {
  const Level& F = *fine.L;
  const Level& C = *coarse.L;
#pragma omp parallel for schedule(dynamic)
  for (long long b = 0; b < (long long)F.boxes.size(); ++b) {
    const Box& B = F.boxes[b];
    for (int z = B.lo[2]; z <= B.hi[2]; ++z)
      for (int y = B.lo[1]; y <= B.hi[1]; ++y)
        for (int x = B.lo[0]; x <= B.hi[0]; ++x) {
          const int X = floordiv2(x), Y = floordiv2(y), Z = floordiv2(z);
          const int sx = (x - 2 * X) ? 1 : -1, sy = (y - 2 * Y) ? 1 : -1, sz = (z - 2 * Z) ? 1 : -1;
          const int o = C.owner[dom_index(C, X, Y, Z)];
          auto v = [&](int i, int j, int k) { return coarse.at(o, X + i * sx, Y + j * sy, Z + k * sz); };
          const R ux00 = lerp34(v(0, 0, 0), v(1, 0, 0));
          const R ux10 = lerp34(v(0, 1, 0), v(1, 1, 0));
          const R ux01 = lerp34(v(0, 0, 1), v(1, 0, 1));
          const R ux11 = lerp34(v(0, 1, 1), v(1, 1, 1));
          const R u = lerp34(lerp34(ux00, ux10), lerp34(ux01, ux11));
          fine.at((int)b, x, y, z) = fine.at((int)b, x, y, z) + u;
        }
  }
}

// ---------------------------------------------------------------------------------------
// Bottom solve.  The 1-D operators (u_{i-1} - 2u_i + u_{i+1})/h^2 with either periodic or
// reflecting (ghost = -mirror) ends have known orthonormal eigenvectors:
//   Dirichlet: q_m(i) = sin(pi m (i+1/2)/n), m = 1..n, mu_m = -(4/h^2) sin^2(pi m / (2n))
//   periodic : 1, cos(2 pi m i/n), sin(2 pi m i/n) (1 <= m < n/2), (-1)^i (n even),
//              mu_m = -(4/h^2) sin^2(pi m / n)
// The 3-D operator is their Kronecker sum, so its (pseudo-)inverse is
//   M = sum over modes with lambda != 0 of v v^T / lambda,  v = q_a (x) q_b (x) q_c.
void eig1d(int n, int periodic, double h, std::vector<double>& Q /* n*n, [m][i] */,
           std::vector<double>& mu) {
  Q.assign((size_t)n * n, 0.0);
  mu.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  const double s4 = 4.0 / (h * h);
  if (!periodic) {
    for (int m = 1; m <= n; ++m) {
      double nrm = 0;
      for (int i = 0; i < n; ++i) {
        double v = std::sin(pi * m * (i + 0.5) / n);
        Q[(size_t)(m - 1) * n + i] = v;
        nrm += v * v;
      }
      nrm = std::sqrt(nrm);
      for (int i = 0; i < n; ++i) Q[(size_t)(m - 1) * n + i] /= nrm;
      double sn = std::sin(pi * m / (2.0 * n));
      mu[m - 1] = -s4 * sn * sn;
    }
    return;
  }
  int row = 0;
  for (int i = 0; i < n; ++i) Q[i] = 1.0 / std::sqrt((double)n);
  mu[row++] = 0.0;
  for (int m = 1; 2 * m < n; ++m) {
    double sn = std::sin(pi * m / n);
    for (int t = 0; t < 2; ++t) {
      double nrm = 0;
      for (int i = 0; i < n; ++i) {
        double a = 2.0 * pi * m * i / n;
        double v = t == 0 ? std::cos(a) : std::sin(a);
        Q[(size_t)row * n + i] = v;
        nrm += v * v;
      }
      nrm = std::sqrt(nrm);
      for (int i = 0; i < n; ++i) Q[(size_t)row * n + i] /= nrm;
      mu[row++] = -s4 * sn * sn;
    }
  }
  if (n % 2 == 0) {
    for (int i = 0; i < n; ++i) Q[(size_t)row * n + i] = (i % 2 ? -1.0 : 1.0) / std::sqrt((double)n);
    mu[row++] = -s4;
  }
}

bool bottom_matrix(const int n[3], const int periodic[3], double h, std::vector<double>& M) {
  long long N = (long long)n[0] * n[1] * n[2];
  if (N <= 0 || N > kMaxBottomCells) return false;
  std::vector<double> Q[3], mu[3];
  for (int d = 0; d < 3; ++d) eig1d(n[d], periodic[d], h, Q[d], mu[d]);
  M.assign((size_t)N * N, 0.0);
  std::vector<double> v(N);
  for (int c = 0; c < n[2]; ++c)
    for (int b = 0; b < n[1]; ++b)
      for (int a = 0; a < n[0]; ++a) {
        double lam = mu[0][a] + mu[1][b] + mu[2][c];
        if (lam == 0.0) continue;  // the constant mode of a fully periodic problem
        for (int z = 0; z < n[2]; ++z)
          for (int y = 0; y < n[1]; ++y)
            for (int x = 0; x < n[0]; ++x)
              v[((long long)z * n[1] + y) * n[0] + x] =
                  Q[0][(size_t)a * n[0] + x] * Q[1][(size_t)b * n[1] + y] * Q[2][(size_t)c * n[2] + z];
        for (long long i = 0; i < N; ++i) {
          double vi = v[i] / lam;
          double* Mi = &M[(size_t)i * N];
          for (long long j = 0; j < N; ++j) Mi[j] += vi * v[j];
        }
      }
  return true;
}

// e = M rhs on the bottom level: gather rhs in domain order (x fastest) through the owner
// map, dot products in index order, scatter to the level's phi (valid cells only).
template <class R>
void bottom_apply(const std::vector<double>& M, const Field<R>& rhs, const Field<R>& phi) {
  const Level& L = *rhs.L;
  long long N = (long long)dext(L, 0) * dext(L, 1) * dext(L, 2);
  std::vector<double> b(N), e(N);
  for (int z = L.dlo[2]; z <= L.dhi[2]; ++z)
    for (int y = L.dlo[1]; y <= L.dhi[1]; ++y)
      for (int x = L.dlo[0]; x <= L.dhi[0]; ++x) {
        long long i = dom_index(L, x, y, z);
        b[i] = (double)rhs.at(L.owner[i], x, y, z);
      }
  for (long long i = 0; i < N; ++i) {
    double s = 0.0;
    for (long long j = 0; j < N; ++j) s = s + M[(size_t)i * N + j] * b[j];
    e[i] = s;
  }
  for (int z = L.dlo[2]; z <= L.dhi[2]; ++z)
    for (int y = L.dlo[1]; y <= L.dhi[1]; ++y)
      for (int x = L.dlo[0]; x <= L.dhi[0]; ++x) {
        long long i = dom_index(L, x, y, z);
        phi.at(L.owner[i], x, y, z) = (R)e[i];
      }
}

// ---------------------------------------------------------------------------------------
// Level hierarchy.  Level l+1 exists while every domain edge of level l is even and >= 4
// (and the domain lo is even).  Its boxes are the level-l boxes coarsened by 2, unless some
// level-l box has an odd lo or odd (hi+1), or some coarsened box edge would fall below 2:
// then level l+1 is one box covering the coarse domain.  The sequence of level domains thus
// depends on the domain only, never on how it is split into boxes.
bool boxes_aligned(const Level& L) {
  for (const Box& B : L.boxes)
    for (int d = 0; d < 3; ++d)
      if (pmod(B.lo[d], 2) != 0 || pmod(B.hi[d] + 1, 2) != 0) return false;
  return true;
}

bool can_coarsen(const Level& L) {
  for (int d = 0; d < 3; ++d) {
    int n = dext(L, d);
    if (n % 2 != 0 || n < 4) return false;
    if (pmod(L.dlo[d], 2) != 0) return false;
  }
  return true;
}

Level coarsen_level(const Level& F) {
  Level C;
  for (int d = 0; d < 3; ++d) {
    C.dlo[d] = floordiv2(F.dlo[d]);
    C.dhi[d] = floordiv2(F.dhi[d] + 1) - 1;
    C.periodic[d] = F.periodic[d];
  }
  C.h = 2.0 * F.h;
  bool small = !boxes_aligned(F);
  for (const Box& B : F.boxes) {
    Box c;
    for (int d = 0; d < 3; ++d) {
      c.lo[d] = floordiv2(B.lo[d]);
      c.hi[d] = floordiv2(B.hi[d] + 1) - 1;
      if (c.hi[d] - c.lo[d] + 1 < 2) small = true;
    }
    C.boxes.push_back(c);
  }
  if (small) {
    Box one;
    for (int d = 0; d < 3; ++d) { one.lo[d] = C.dlo[d]; one.hi[d] = C.dhi[d]; }
    C.boxes.assign(1, one);
  }
  return C;
}

bool build_hierarchy(const Level& L0, std::vector<Level>& levels) {
  levels.clear();
  levels.push_back(L0);
  if (!build_owner(levels.back())) return false;
  while (can_coarsen(levels.back())) {
    Level C = coarsen_level(levels.back());
    levels.push_back(C);
    if (!build_owner(levels.back())) return false;
  }
  const Level& B = levels.back();
  long long nb = (long long)dext(B, 0) * dext(B, 1) * dext(B, 2);
  return nb <= kMaxBottomCells;
}

Level make_level(const int dlo[3], const int dhi[3], const int periodic[3], double h, int nbox,
                 const int* lohi) {
  Level L;
  for (int d = 0; d < 3; ++d) {
    L.dlo[d] = dlo[d]; L.dhi[d] = dhi[d]; L.periodic[d] = periodic[d] ? 1 : 0;
  }
  L.h = h;
  for (int b = 0; b < nbox; ++b) {
    Box B;
    for (int d = 0; d < 3; ++d) { B.lo[d] = lohi[6 * b + d]; B.hi[d] = lohi[6 * b + 3 + d]; }
    L.boxes.push_back(B);
  }
  return L;
}

// ---------------------------------------------------------------------------------------
// The V-cycle and the solve loop.

template <class R>
struct LevelData {
  std::vector<R> phi, rhs, r;
  Field<R> fphi, frhs, fr;
};

template <class R>
void alloc_levels(const std::vector<Level>& levels, std::vector<LevelData<R>>& D) {
  D.resize(levels.size());
  for (size_t l = 0; l < levels.size(); ++l) {
    const Level& L = levels[l];
    std::vector<long long> o1 = fab_offsets(L, 1, 1), o0 = fab_offsets(L, 0, 1);
    D[l].phi.assign(o1.back(), (R)0);
    D[l].rhs.assign(o0.back(), (R)0);
    D[l].r.assign(o0.back(), (R)0);
    D[l].fphi = make_field(L, 1, 1, D[l].phi.data());
    D[l].frhs = make_field(L, 0, 1, D[l].rhs.data());
    D[l].fr = make_field(L, 0, 1, D[l].r.data());
  }
}

template <class R>
void zero_valid(const Field<R>& f) {
  const Level& L = *f.L;
  for (size_t b = 0; b < L.boxes.size(); ++b) {
    const Box& B = L.boxes[b];
    for (int z = B.lo[2]; z <= B.hi[2]; ++z)
      for (int y = B.lo[1]; y <= B.hi[1]; ++y)
        for (int x = B.lo[0]; x <= B.hi[0]; ++x) f.at((int)b, x, y, z) = (R)0;
  }
}

template <class R>
void smooth(const Field<R>& phi, const Field<R>& rhs, int nsweeps) {
  for (int s = 0; s < nsweeps; ++s) {
    fill(phi);
    rbgs(phi, rhs, 0);
    fill(phi);
    rbgs(phi, rhs, 1);
  }
}

template <class R>
void vcycle(std::vector<LevelData<R>>& D, const std::vector<std::vector<double>>& Mb, size_t l,
            int nu1, int nu2, bool trilinear) {
  size_t bottom = D.size() - 1;
  if (l == bottom) {
    bottom_apply(Mb[0], D[l].frhs, D[l].fphi);
    return;
  }
  smooth(D[l].fphi, D[l].frhs, nu1);
  fill(D[l].fphi);
  residual(D[l].fphi, D[l].frhs, &D[l].fr);
  restrict_avg(D[l].fr, D[l + 1].frhs);
  zero_valid(D[l + 1].fphi);
  vcycle(D, Mb, l + 1, nu1, nu2, trilinear);
  if (trilinear) {
    fill(D[l + 1].fphi);
    prolong_add_trilinear(D[l + 1].fphi, D[l].fphi);
  } else {
    prolong_add(D[l + 1].fphi, D[l].fphi);
  }
  smooth(D[l].fphi, D[l].frhs, nu2);
}

// Gather / scatter between a dense domain array (x fastest) and a level field.
template <class R, class S>
void scatter_dense(const Level& L, const S* g, const Field<R>& f) {
  for (size_t b = 0; b < L.boxes.size(); ++b) {
    const Box& B = L.boxes[b];
    for (int z = B.lo[2]; z <= B.hi[2]; ++z)
      for (int y = B.lo[1]; y <= B.hi[1]; ++y)
        for (int x = B.lo[0]; x <= B.hi[0]; ++x) f.at((int)b, x, y, z) = (R)g[dom_index(L, x, y, z)];
  }
}
template <class R, class S>
void gather_dense(const Level& L, const Field<R>& f, S* g) {
  for (size_t b = 0; b < L.boxes.size(); ++b) {
    const Box& B = L.boxes[b];
    for (int z = B.lo[2]; z <= B.hi[2]; ++z)
      for (int y = B.lo[1]; y <= B.hi[1]; ++y)
        for (int x = B.lo[0]; x <= B.hi[0]; ++x) g[dom_index(L, x, y, z)] = (S)f.at((int)b, x, y, z);
  }
}

double max_abs_valid(const Field<double>& f) {
  const Level& L = *f.L;
  double mx = 0.0;
  bool nan = false;
  for (size_t b = 0; b < L.boxes.size(); ++b) {
    const Box& B = L.boxes[b];
    for (int z = B.lo[2]; z <= B.hi[2]; ++z)
      for (int y = B.lo[1]; y <= B.hi[1]; ++y)
        for (int x = B.lo[0]; x <= B.hi[0]; ++x) {
          double a = std::fabs(f.at((int)b, x, y, z));
          if (std::isnan(a)) nan = true;
          if (a > mx) mx = a;
        }
  }
  return nan ? NAN : mx;
}

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_NOT_CONVERGED = -4, ORC_ENAN = -7 };

}  // namespace

// =======================================================================================
// C entry points used by oracle/__init__.py.  Box lists are int[6*nbox] = lo0 lo1 lo2 hi0
// hi1 hi2 per box (inclusive).  Level fields use the oracle layout described above.

extern "C" {

// Chop the domain into boxes of edge <= max_box per dimension: pieces of max_box from lo,
// the remainder last.  Boxes are ordered x fastest.  Returns the box count, or -1 if cap is
// too small.
int orc_chop(const int dlo[3], const int dhi[3], const int maxb[3], int cap, int* lohi) {
  std::vector<int> cuts[3];
  for (int d = 0; d < 3; ++d) {
    if (maxb[d] <= 0 || dhi[d] < dlo[d]) return -1;
    for (int s = dlo[d]; s <= dhi[d]; s += maxb[d]) cuts[d].push_back(s);
  }
  int nb = 0;
  for (size_t k = 0; k < cuts[2].size(); ++k)
    for (size_t j = 0; j < cuts[1].size(); ++j)
      for (size_t i = 0; i < cuts[0].size(); ++i) {
        if (nb >= cap) return -1;
        int st[3] = {cuts[0][i], cuts[1][j], cuts[2][k]};
        for (int d = 0; d < 3; ++d) {
          lohi[6 * nb + d] = st[d];
          lohi[6 * nb + 3 + d] = std::min(st[d] + maxb[d] - 1, dhi[d]);
        }
        ++nb;
      }
  return nb;
}

// Level hierarchy.  Writes per level: domain (6 ints) into dom_out, box count into nbox_out,
// boxes into lohi_out (concatenated).  Returns the level count, or -1 (invalid / caps).
int orc_hierarchy(const int dlo[3], const int dhi[3], int nbox, const int* lohi, int cap_levels,
                  int cap_boxes, int* dom_out, int* nbox_out, int* lohi_out) {
  int per[3] = {0, 0, 0};
  Level L0 = make_level(dlo, dhi, per, 1.0, nbox, lohi);
  std::vector<Level> levels;
  if (!build_hierarchy(L0, levels)) return -1;
  if ((int)levels.size() > cap_levels) return -1;
  int k = 0;
  for (size_t l = 0; l < levels.size(); ++l) {
    for (int d = 0; d < 3; ++d) {
      dom_out[6 * l + d] = levels[l].dlo[d];
      dom_out[6 * l + 3 + d] = levels[l].dhi[d];
    }
    nbox_out[l] = (int)levels[l].boxes.size();
    for (const Box& B : levels[l].boxes) {
      if (k >= cap_boxes) return -1;
      for (int d = 0; d < 3; ++d) { lohi_out[6 * k + d] = B.lo[d]; lohi_out[6 * k + 3 + d] = B.hi[d]; }
      ++k;
    }
  }
  return (int)levels.size();
}

int orc_fill(const int dlo[3], const int dhi[3], const int periodic[3], int nbox, const int* lohi,
             int ng, int ncomp, double* data) {
  Level L = make_level(dlo, dhi, periodic, 1.0, nbox, lohi);
  if (!build_owner(L) || ng < 0 || ncomp < 1) return ORC_EINVAL;
  return fill(make_field(L, ng, ncomp, data)) ? ORC_OK : ORC_EINVAL;
}

int orc_fill_f32(const int dlo[3], const int dhi[3], const int periodic[3], int nbox,
                 const int* lohi, int ng, int ncomp, float* data) {
  Level L = make_level(dlo, dhi, periodic, 1.0, nbox, lohi);
  if (!build_owner(L) || ng < 0 || ncomp < 1) return ORC_EINVAL;
  return fill(make_field(L, ng, ncomp, data)) ? ORC_OK : ORC_EINVAL;
}

// One half-sweep; phi's ghosts are used as they are (fill first).
int orc_rbgs(const int dlo[3], const int dhi[3], int nbox, const int* lohi, double h, int ng_phi,
             double* phi, int ng_rhs, const double* rhs, int color) {
  int per[3] = {0, 0, 0};
  Level L = make_level(dlo, dhi, per, h, nbox, lohi);
  if (!build_owner(L) || ng_phi < 1) return ORC_EINVAL;
  rbgs(make_field(L, ng_phi, 1, phi), make_field(L, ng_rhs, 1, const_cast<double*>(rhs)), color);
  return ORC_OK;
}

int orc_rbgs_f32(const int dlo[3], const int dhi[3], int nbox, const int* lohi, double h,
                 int ng_phi, float* phi, int ng_rhs, const float* rhs, int color) {
  int per[3] = {0, 0, 0};
  Level L = make_level(dlo, dhi, per, h, nbox, lohi);
  if (!build_owner(L) || ng_phi < 1) return ORC_EINVAL;
  rbgs(make_field(L, ng_phi, 1, phi), make_field(L, ng_rhs, 1, const_cast<float*>(rhs)), color);
  return ORC_OK;
}

// Residual into r (ng_r ghosts, may be null); max-norm into *norm.
int orc_residual(const int dlo[3], const int dhi[3], int nbox, const int* lohi, double h,
                 int ng_phi, const double* phi, int ng_rhs, const double* rhs, int ng_r, double* r,
                 double* norm) {
  int per[3] = {0, 0, 0};
  Level L = make_level(dlo, dhi, per, h, nbox, lohi);
  if (!build_owner(L) || ng_phi < 1) return ORC_EINVAL;
  Field<double> fr = make_field(L, ng_r, 1, r);
  *norm = residual(make_field(L, ng_phi, 1, const_cast<double*>(phi)),
                   make_field(L, ng_rhs, 1, const_cast<double*>(rhs)), r ? &fr : nullptr);
  return ORC_OK;
}

int orc_restrict(const int fdlo[3], const int fdhi[3], int fnbox, const int* flohi, int ng_f,
                 const double* fine, const int cdlo[3], const int cdhi[3], int cnbox,
                 const int* clohi, int ng_c, double* coarse) {
  int per[3] = {0, 0, 0};
  Level F = make_level(fdlo, fdhi, per, 1.0, fnbox, flohi);
  Level C = make_level(cdlo, cdhi, per, 2.0, cnbox, clohi);
  if (!build_owner(F) || !build_owner(C)) return ORC_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (2 * C.dlo[d] != F.dlo[d] || 2 * C.dhi[d] + 1 != F.dhi[d]) return ORC_EINVAL;
  restrict_avg(make_field(F, ng_f, 1, const_cast<double*>(fine)), make_field(C, ng_c, 1, coarse));
  return ORC_OK;
}

// trilinear != 0: the trilinear form, reading the coarse ghosts as they are (fill first).
int orc_prolong(const int cdlo[3], const int cdhi[3], int cnbox, const int* clohi, int ng_c,
                const double* coarse, const int fdlo[3], const int fdhi[3], int fnbox,
                const int* flohi, int ng_f, double* fine, int trilinear) {
  int per[3] = {0, 0, 0};
  Level F = make_level(fdlo, fdhi, per, 1.0, fnbox, flohi);
  Level C = make_level(cdlo, cdhi, per, 2.0, cnbox, clohi);
  if (!build_owner(F) || !build_owner(C)) return ORC_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (2 * C.dlo[d] != F.dlo[d] || 2 * C.dhi[d] + 1 != F.dhi[d]) return ORC_EINVAL;
  if (trilinear) {
    if (ng_c < 1) return ORC_EINVAL;
    prolong_add_trilinear(make_field(C, ng_c, 1, const_cast<double*>(coarse)), make_field(F, ng_f, 1, fine));
  } else {
    prolong_add(make_field(C, ng_c, 1, const_cast<double*>(coarse)), make_field(F, ng_f, 1, fine));
  }
  return ORC_OK;
}

// Threads of the oracle's OpenMP loops from now on (n >= 1); returns the count in effect.
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

int orc_bottom_matrix(const int n[3], const int periodic[3], double h, double* M) {
  std::vector<double> m;
  if (!bottom_matrix(n, periodic, h, m)) return ORC_EINVAL;
  std::memcpy(M, m.data(), m.size() * sizeof(double));
  return ORC_OK;
}

// Full solve.  rhs_g / phi_g are dense domain arrays (x fastest); phi_g is the initial guess
// on entry and the result on exit.  fixed_vcycles >= 0 runs exactly that many V-cycles with
// no stop test.  mixed != 0 selects the FP64-outer / FP32-inner form.  hist receives the
// relative residual before each V-cycle and after the last (hist_cap entries at most).
// trilinear != 0 selects the trilinear prolongation.  inner (>= 1): FP32 V-cycles per outer
// iteration of the mixed form, the later ones continuing from the correction so far.
// Returns ORC_OK, ORC_NOT_CONVERGED, ORC_ENAN or ORC_EINVAL.
int orc_solve(const int dlo[3], const int dhi[3], const int periodic[3], int nbox, const int* lohi,
              double h, const double* rhs_g, double* phi_g, double tol, int max_iter, int nu1,
              int nu2, int fixed_vcycles, int mixed, int* vcycles, double* hist, int hist_cap,
              int trilinear, int inner) {
  if (inner < 1) return ORC_EINVAL;
  Level L0 = make_level(dlo, dhi, periodic, h, nbox, lohi);
  std::vector<Level> levels;
  if (!build_hierarchy(L0, levels)) return ORC_EINVAL;
  for (size_t l = 1; l < levels.size(); ++l) levels[l].h = 2.0 * levels[l - 1].h;
  const Level& Lb = levels.back();
  int nb[3] = {dext(Lb, 0), dext(Lb, 1), dext(Lb, 2)};
  std::vector<std::vector<double>> Mb(1);
  if (!bottom_matrix(nb, Lb.periodic, Lb.h, Mb[0])) return ORC_EINVAL;

  std::vector<LevelData<double>> D;
  alloc_levels(levels, D);
  scatter_dense(levels[0], rhs_g, D[0].frhs);
  scatter_dense(levels[0], phi_g, D[0].fphi);
  double rhsnorm = max_abs_valid(D[0].frhs);
  *vcycles = 0;
  if (std::isnan(rhsnorm)) return ORC_ENAN;
  if (rhsnorm == 0.0) {
    zero_valid(D[0].fphi);
    gather_dense(levels[0], D[0].fphi, phi_g);
    if (hist_cap > 0) hist[0] = 0.0;
    return ORC_OK;
  }

  std::vector<LevelData<float>> Df;
  if (mixed) alloc_levels(levels, Df);

  int status = ORC_OK;
  for (int it = 0;; ++it) {
    fill(D[0].fphi);
    double rn = residual(D[0].fphi, D[0].frhs, mixed ? &D[0].fr : nullptr);
    if (it < hist_cap) hist[it] = rn / rhsnorm;
    if (std::isnan(rn)) { status = ORC_ENAN; break; }
    if (fixed_vcycles >= 0) {
      if (it == fixed_vcycles) break;
    } else {
      if (rn <= tol * rhsnorm) break;
      if (it == max_iter) { status = ORC_NOT_CONVERGED; break; }
    }
    if (!mixed) {
      vcycle(D, Mb, 0, nu1, nu2, trilinear != 0);
    } else {
      // Inner FP32 V-cycle on the residual scaled by 2^-e, 2^e <= ||r|| < 2^(e+1) (exact),
      // FP64 correction add.
      const double up = std::ldexp(1.0, std::ilogb(rn));
      const double down = std::ldexp(1.0, -std::ilogb(rn));
      const Level& L = levels[0];
      for (size_t b = 0; b < L.boxes.size(); ++b) {
        const Box& B = L.boxes[b];
        for (int z = B.lo[2]; z <= B.hi[2]; ++z)
          for (int y = B.lo[1]; y <= B.hi[1]; ++y)
            for (int x = B.lo[0]; x <= B.hi[0]; ++x)
              Df[0].frhs.at((int)b, x, y, z) = (float)(D[0].fr.at((int)b, x, y, z) * down);
      }
      zero_valid(Df[0].fphi);
      for (int k = 0; k < inner; ++k) vcycle(Df, Mb, 0, nu1, nu2, trilinear != 0);
      for (size_t b = 0; b < L.boxes.size(); ++b) {
        const Box& B = L.boxes[b];
        for (int z = B.lo[2]; z <= B.hi[2]; ++z)
          for (int y = B.lo[1]; y <= B.hi[1]; ++y)
            for (int x = B.lo[0]; x <= B.hi[0]; ++x)
              D[0].fphi.at((int)b, x, y, z) =
                  std::fma(up, (double)Df[0].fphi.at((int)b, x, y, z), D[0].fphi.at((int)b, x, y, z));
      }
    }
    *vcycles = it + 1;
  }
  gather_dense(levels[0], D[0].fphi, phi_g);
  return status;
}

}  // extern "C"
