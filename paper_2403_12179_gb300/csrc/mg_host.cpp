// Host-side planning: box algebra, hierarchy, copy tags, layouts, bottom matrix.
// Ghost exchange as a cached, precomputed communication pattern follows Sec. 2 of the
// AMReX/pyAMReX review (arXiv 2403.12179); the concrete rules are documented per function.
#include "mg_host.hpp"

#include <algorithm>
#include <cmath>
#include <cstdio>

namespace gbmg {

Box intersect(const Box& a, const Box& b) {
  Box r;
  for (int d = 0; d < 3; ++d) {
    r.lo[d] = std::max(a.lo[d], b.lo[d]);
    r.hi[d] = std::min(a.hi[d], b.hi[d]);
  }
  return r;
}

Box grow(const Box& b, int g) {
  Box r = b;
  for (int d = 0; d < 3; ++d) { r.lo[d] -= g; r.hi[d] += g; }
  return r;
}

Box shift(const Box& b, const int s[3]) {
  Box r = b;
  for (int d = 0; d < 3; ++d) { r.lo[d] += s[d]; r.hi[d] += s[d]; }
  return r;
}

bool contains(const Box& b, int x, int y, int z) {
  return x >= b.lo[0] && x <= b.hi[0] && y >= b.lo[1] && y <= b.hi[1] && z >= b.lo[2] &&
         z <= b.hi[2];
}

long long BoxArray::cells() const {
  long long n = 0;
  for (const Box& b : boxes) n += b.npts();
  return n;
}

static std::string fmt_box(const Box& b) {
  char buf[128];
  std::snprintf(buf, sizeof buf, "[(%d,%d,%d)-(%d,%d,%d)]", b.lo[0], b.lo[1], b.lo[2], b.hi[0],
                b.hi[1], b.hi[2]);
  return buf;
}

bool chop(const Box& dom, const int max_box[3], BoxArray* out, std::string* err) {
  if (dom.empty()) { *err = "empty domain"; return false; }
  std::vector<int> starts[3];
  for (int d = 0; d < 3; ++d) {
    if (max_box[d] < 1) { *err = "max_box must be >= 1"; return false; }
    for (long long s = dom.lo[d]; s <= dom.hi[d]; s += max_box[d]) starts[d].push_back((int)s);
  }
  out->dom = dom;
  out->boxes.clear();
  for (int k : starts[2])
    for (int j : starts[1])
      for (int i : starts[0]) {
        Box b;
        int st[3] = {i, j, k};
        for (int d = 0; d < 3; ++d) {
          b.lo[d] = st[d];
          b.hi[d] = (int)std::min<long long>((long long)st[d] + max_box[d] - 1, dom.hi[d]);
        }
        out->boxes.push_back(b);
      }
  return true;
}

bool validate(const BoxArray& ba, std::string* err) {
  if (ba.dom.empty()) { *err = "empty domain"; return false; }
  if (ba.boxes.empty()) { *err = "no boxes"; return false; }
  for (const Box& b : ba.boxes) {
    if (b.empty()) { *err = "empty box " + fmt_box(b); return false; }
    // the device kernels index a box's x-rows (ghosts included) with 32-bit integers
    if ((int64_t)(b.len(1) + 8) * (b.len(2) + 8) >= ((int64_t)1 << 30)) {
      *err = "box " + fmt_box(b) + " has too many x-rows";
      return false;
    }
    Box i = intersect(b, ba.dom);
    if (i.npts() != b.npts() || i.empty()) {
      *err = "box " + fmt_box(b) + " leaves the domain " + fmt_box(ba.dom);
      return false;
    }
  }
  // Pairwise disjoint (sweep over boxes sorted by lo.x) and total volume equals the domain.
  std::vector<int> order(ba.boxes.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::sort(order.begin(), order.end(),
            [&](int a, int b) { return ba.boxes[a].lo[0] < ba.boxes[b].lo[0]; });
  for (size_t a = 0; a < order.size(); ++a) {
    const Box& A = ba.boxes[order[a]];
    for (size_t b = a + 1; b < order.size(); ++b) {
      const Box& B = ba.boxes[order[b]];
      if (B.lo[0] > A.hi[0]) break;
      if (!intersect(A, B).empty()) {
        *err = "boxes " + fmt_box(A) + " and " + fmt_box(B) + " overlap";
        return false;
      }
    }
  }
  if (ba.cells() != ba.dom.npts()) { *err = "boxes do not cover the domain"; return false; }
  return true;
}

bool aligned(const BoxArray& ba) {
  for (const Box& b : ba.boxes)
    for (int d = 0; d < 3; ++d)
      if ((b.lo[d] & 1) != 0 || ((b.hi[d] + 1) & 1) != 0) return false;
  return true;
}

bool build_levels(const BoxArray& fine, std::vector<BoxArray>* levels, std::string* err) {
  levels->clear();
  levels->push_back(fine);
  for (;;) {
    const BoxArray& F = levels->back();
    bool more = true;
    for (int d = 0; d < 3; ++d) {
      int n = F.dom.len(d);
      if (n % 2 != 0 || n < 4 || (F.dom.lo[d] & 1) != 0) more = false;
    }
    if (!more) break;
    BoxArray C;
    for (int d = 0; d < 3; ++d) {
      C.dom.lo[d] = fdiv2(F.dom.lo[d]);
      C.dom.hi[d] = fdiv2(F.dom.hi[d] + 1) - 1;
    }
    bool merge = !aligned(F);
    if (!merge) {
      for (const Box& b : F.boxes) {
        Box c;
        for (int d = 0; d < 3; ++d) {
          c.lo[d] = fdiv2(b.lo[d]);
          c.hi[d] = fdiv2(b.hi[d] + 1) - 1;
          if (c.len(d) < 2) merge = true;
        }
        C.boxes.push_back(c);
      }
    }
    if (merge) C.boxes.assign(1, C.dom);
    levels->push_back(C);
  }
  if (levels->back().dom.npts() > kMaxBottomCells) {
    *err = "bottom level " + fmt_box(levels->back().dom) + " has more than 1024 cells "
           "(domain edges must reduce to <= 1024 cells by halving)";
    return false;
  }
  return true;
}

// One dimension of a ghost region split into pieces that are inside the domain (after a
// periodic shift), below it, or above it.
struct Piece {
  int a, b;    // range in the destination's index space
  int kind;    // 0 inside (after shift), -1 below the domain, +1 above
  int shift;   // added to reach the domain (periodic image)
};

static void split_dim(int a, int b, int dlo, int dhi, bool periodic, std::vector<Piece>* out) {
  out->clear();
  int n = dhi - dlo + 1;
  if (periodic) {
    int x = a;
    while (x <= b) {
      int k = (x - dlo) >= 0 ? (x - dlo) / n : -((dlo - x + n - 1) / n);  // image index
      int end = std::min(b, dlo + (k + 1) * n - 1);
      out->push_back({x, end, 0, -k * n});
      x = end + 1;
    }
    return;
  }
  if (a < dlo) out->push_back({a, std::min(b, dlo - 1), -1, 0});
  if (std::max(a, dlo) <= std::min(b, dhi)) out->push_back({std::max(a, dlo), std::min(b, dhi), 0, 0});
  if (b > dhi) out->push_back({std::max(a, dhi + 1), b, +1, 0});
}

bool make_copy_tags(const BoxArray& ba, const int periodic[3], int g, std::vector<CopyTag>* tags,
                    std::string* err) {
  tags->clear();
  if (g < 0) { *err = "negative ghost width"; return false; }
  if (g == 0) return true;
  for (int d = 0; d < 3; ++d)
    if (!periodic[d] && g > ba.dom.len(d)) {
      *err = "ghost width exceeds a Dirichlet domain extent";
      return false;
    }
  const Box& D = ba.dom;
  std::vector<Piece> pcs[3];
  for (size_t bi = 0; bi < ba.boxes.size(); ++bi) {
    const Box& B = ba.boxes[bi];
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (!dx && !dy && !dz) continue;
          int dir[3] = {dx, dy, dz};
          for (int d = 0; d < 3; ++d) {
            int a = dir[d] < 0 ? B.lo[d] - g : dir[d] > 0 ? B.hi[d] + 1 : B.lo[d];
            int b = dir[d] < 0 ? B.lo[d] - 1 : dir[d] > 0 ? B.hi[d] + g : B.hi[d];
            split_dim(a, b, D.lo[d], D.hi[d], periodic[d] != 0, &pcs[d]);
          }
          for (const Piece& pz : pcs[2])
            for (const Piece& py : pcs[1])
              for (const Piece& px : pcs[0]) {
                const Piece* p[3] = {&px, &py, &pz};
                int nout = 0, od = -1;
                for (int d = 0; d < 3; ++d)
                  if (p[d]->kind != 0) { ++nout; od = d; }
                Box dst;
                for (int d = 0; d < 3; ++d) { dst.lo[d] = p[d]->a; dst.hi[d] = p[d]->b; }
                if (nout >= 2) {
                  CopyTag t{};
                  t.src_box = -1;
                  t.dst_box = (int)bi;
                  for (int d = 0; d < 3; ++d) {
                    t.dst_lo[d] = dst.lo[d];
                    t.src_first[d] = 0;
                    t.dir[d] = 1;
                    t.ext[d] = dst.len(d);
                  }
                  t.sign = 0;
                  tags->push_back(t);
                  continue;
                }
                // Source region inside the domain: periodic shift, plus the mirror across
                // the one Dirichlet face if the piece lies outside it.
                Box src;
                for (int d = 0; d < 3; ++d) {
                  if (d == od) {
                    int m = p[d]->kind < 0 ? 2 * D.lo[d] - 1 : 2 * D.hi[d] + 1;  // x -> m - x
                    src.lo[d] = m - dst.hi[d];
                    src.hi[d] = m - dst.lo[d];
                  } else {
                    src.lo[d] = dst.lo[d] + p[d]->shift;
                    src.hi[d] = dst.hi[d] + p[d]->shift;
                  }
                }
                for (size_t si = 0; si < ba.boxes.size(); ++si) {
                  Box I = intersect(src, ba.boxes[si]);
                  if (I.empty()) continue;
                  CopyTag t{};
                  t.src_box = (int)si;
                  t.dst_box = (int)bi;
                  for (int d = 0; d < 3; ++d) {
                    t.ext[d] = I.len(d);
                    if (d == od) {
                      int m = p[d]->kind < 0 ? 2 * D.lo[d] - 1 : 2 * D.hi[d] + 1;
                      t.dst_lo[d] = m - I.hi[d];
                      t.src_first[d] = I.hi[d];
                      t.dir[d] = -1;
                    } else {
                      t.dst_lo[d] = I.lo[d] - p[d]->shift;
                      t.src_first[d] = I.lo[d];
                      t.dir[d] = 1;
                    }
                  }
                  t.sign = nout == 1 ? -1 : 1;
                  tags->push_back(t);
                }
              }
        }
  }
  return true;
}

FabLayout make_layout(const BoxArray& ba, int ncomp, int g, int esize) {
  FabLayout L;
  L.ncomp = ncomp;
  L.g = g;
  L.esize = esize;
  const int row_align = 16 / esize;   // rows start on 16-byte boundaries
  const int box_align = 256 / esize;  // boxes start on 256-byte boundaries
  long long cur = 0;
  for (const Box& b : ba.boxes) {
    int pitch = (b.len(0) + 2 * g + row_align - 1) / row_align * row_align;
    long long plane = (long long)pitch * (b.len(1) + 2 * g);
    long long cs = plane * (b.len(2) + 2 * g);
    cur = (cur + box_align - 1) / box_align * box_align;
    L.off.push_back(cur);
    L.pitch.push_back(pitch);
    L.plane.push_back(plane);
    L.cstride.push_back(cs);
    cur += cs * ncomp;
  }
  L.total = (cur + box_align - 1) / box_align * box_align;
  return L;
}

// Bottom matrix from 1-D spectral projectors.  With P_m(i,i') the projector of the 1-D
// operator onto its eigenspace m (eigenvalue mu_m), the 3-D operator's (pseudo-)inverse is
//   M(c,c') = sum over (a,b,c) with lambda != 0 of Pa(x,x') Pb(y,y') Pc(z,z') / lambda,
//   lambda = mu_a + mu_b + mu_c.
// Periodic ends: m = 0..n-1, P_m(i,i') = cos(2 pi m (i-i')/n) / n, mu_m = -(4/h^2) sin^2(pi m/n)
// (the real part of the Fourier projector; m and n-m are summed separately).
// Reflecting ends: m = 1..n, P_m(i,i') = (2/n) w_m sin(pi m (i+1/2)/n) sin(pi m (i'+1/2)/n),
// w_m = 1 for m < n and 1/2 for m = n, mu_m = -(4/h^2) sin^2(pi m/(2n)).
bool bottom_matrix(const int n[3], const int periodic[3], double h, std::vector<double>* M,
                   std::string* err) {
  long long N = (long long)n[0] * n[1] * n[2];
  if (n[0] < 1 || n[1] < 1 || n[2] < 1 || N > kMaxBottomCells) {
    *err = "bottom size out of range";
    return false;
  }
  const double pi = 3.141592653589793238462643;
  const double s4 = 4.0 / (h * h);
  std::vector<double> P[3], mu[3];
  for (int d = 0; d < 3; ++d) {
    int m_ = n[d];
    P[d].assign((size_t)m_ * m_ * m_, 0.0);
    mu[d].assign(m_, 0.0);
    for (int k = 0; k < m_; ++k) {
      double* Pk = &P[d][(size_t)k * m_ * m_];
      if (periodic[d]) {
        double s = std::sin(pi * k / m_);
        mu[d][k] = -s4 * s * s;
        for (int i = 0; i < m_; ++i)
          for (int j = 0; j < m_; ++j) Pk[i * m_ + j] = std::cos(2.0 * pi * k * (i - j) / m_) / m_;
      } else {
        int m = k + 1;
        double s = std::sin(pi * m / (2.0 * m_));
        mu[d][k] = -s4 * s * s;
        double w = (m == m_) ? 0.5 : 1.0;
        for (int i = 0; i < m_; ++i)
          for (int j = 0; j < m_; ++j)
            Pk[i * m_ + j] = 2.0 / m_ * w * std::sin(pi * m * (i + 0.5) / m_) *
                             std::sin(pi * m * (j + 0.5) / m_);
      }
    }
  }
  const int nx = n[0], ny = n[1], nz = n[2];
  M->assign((size_t)N * N, 0.0);
  std::vector<double> G((size_t)nz * nz);
  for (int a = 0; a < nx; ++a)
    for (int b = 0; b < ny; ++b) {
      // G(z,z') = sum_c Pc(z,z') / (mu_a + mu_b + mu_c), skipping the null mode
      std::fill(G.begin(), G.end(), 0.0);
      bool any = false;
      for (int c = 0; c < nz; ++c) {
        double lam = mu[0][a] + mu[1][b] + mu[2][c];
        if (lam == 0.0) continue;
        any = true;
        const double* Pc = &P[2][(size_t)c * nz * nz];
        for (int t = 0; t < nz * nz; ++t) G[t] += Pc[t] / lam;
      }
      if (!any) continue;
      const double* Pa = &P[0][(size_t)a * nx * nx];
      const double* Pb = &P[1][(size_t)b * ny * ny];
      for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
          for (int x = 0; x < nx; ++x) {
            double* row = &(*M)[(size_t)(((long long)z * ny + y) * nx + x) * N];
            for (int z2 = 0; z2 < nz; ++z2) {
              double gz = G[z * nz + z2];
              for (int y2 = 0; y2 < ny; ++y2) {
                double gyz = Pb[y * ny + y2] * gz;
                double* r = row + ((long long)z2 * ny + y2) * nx;
                for (int x2 = 0; x2 < nx; ++x2) r[x2] += Pa[x * nx + x2] * gyz;
              }
            }
          }
    }
  return true;
}

}  // namespace gbmg
