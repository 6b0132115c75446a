// Host-side planning for the multigrid path: box algebra, box arrays, the multigrid level
// hierarchy, copy tags for the ghost fill, fab layouts and the closed-form bottom matrix.
// Nothing here touches the GPU.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace gbmg {

constexpr int kMaxBottomCells = 1024;

struct Box {
  int lo[3];
  int hi[3];
  int len(int d) const { return hi[d] - lo[d] + 1; }
  bool empty() const { return hi[0] < lo[0] || hi[1] < lo[1] || hi[2] < lo[2]; }
  long long npts() const { return empty() ? 0 : (long long)len(0) * len(1) * len(2); }
};

Box intersect(const Box& a, const Box& b);
Box grow(const Box& b, int g);
Box shift(const Box& b, const int s[3]);
bool contains(const Box& b, int x, int y, int z);

struct BoxArray {
  Box dom;
  std::vector<Box> boxes;
  long long cells() const;
};

// Floor division by 2 and non-negative modulo for possibly negative indices.
inline int fdiv2(int a) { return a >= 0 ? a / 2 : -((1 - a) / 2); }
inline int pmod(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

// Pieces of max_box from lo, remainder last, x fastest.
bool chop(const Box& dom, const int max_box[3], BoxArray* out, std::string* err);
// Boxes must be non-empty, inside the domain, pairwise disjoint and cover it.
bool validate(const BoxArray& ba, std::string* err);

// Multigrid levels: level l+1 exists while every domain edge of level l is even and >= 4 and
// the domain lo is even.  Its boxes are the level-l boxes coarsened by 2, unless some
// level-l box has odd bounds or some coarsened edge is below 2 -- then it is one box over
// the coarse domain.  The last level must hold <= kMaxBottomCells cells.
bool build_levels(const BoxArray& fine, std::vector<BoxArray>* levels, std::string* err);

// True if every box has even lo and even hi+1 (so each 2x2x2 child group lies in one box).
bool aligned(const BoxArray& ba);

// A ghost-fill copy tag: destination cells dst_lo + (i,j,k) for 0 <= (i,j,k) < ext receive
// sign * src(src_first + dir * (i,j,k)); sign 0 means "write 0".
struct CopyTag {
  int src_box, dst_box;
  int src_first[3];
  int dst_lo[3];
  int dir[3];
  int ext[3];
  int sign;
};

// Tags filling every ghost cell (grow(box, g) minus box) of every box: periodic images and
// other boxes by box intersection; -(mirror) across a single Dirichlet face; 0 when the
// ghost is outside the domain in two or more non-periodic dimensions.
bool make_copy_tags(const BoxArray& ba, const int periodic[3], int g, std::vector<CopyTag>* tags,
                    std::string* err);

// Per-box storage of a fab: x fastest, rows padded to 16 bytes, planes and components
// contiguous, each box 256-byte aligned in one allocation.  Offsets are in elements.
struct FabLayout {
  int ncomp = 1, g = 0, esize = 8;
  std::vector<long long> off;
  std::vector<int> pitch;
  std::vector<long long> plane, cstride;
  long long total = 0;  // elements
  // element offset of cell (x,y,z) comp c of box b
  long long at(const BoxArray& ba, int b, int x, int y, int z, int c = 0) const {
    const Box& B = ba.boxes[b];
    return off[b] + c * cstride[b] + (long long)(z - B.lo[2] + g) * plane[b] +
           (long long)(y - B.lo[1] + g) * pitch[b] + (x - B.lo[0] + g);
  }
};
FabLayout make_layout(const BoxArray& ba, int ncomp, int g, int esize);

// Closed-form (pseudo-)inverse of the 7-point operator on an n0 x n1 x n2 box (x fastest),
// per-dimension periodic or reflecting (ghost = -mirror) ends, cell size h.
bool bottom_matrix(const int n[3], const int periodic[3], double h, std::vector<double>* M,
                   std::string* err);

}  // namespace gbmg
