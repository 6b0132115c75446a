"""Independent dense restatements used to pin the oracle (tests only).

The 7-point operator is assembled entry by entry from its definition: each of the six
neighbours contributes 1/h^2; a neighbour across a periodic face wraps; a neighbour across a
homogeneous Dirichlet face is the ghost -phi(c) (its mirror across the face is c itself), so
it contributes -1/h^2 to the diagonal; the centre contributes -6/h^2.  Unknowns are ordered
x fastest.
"""
import numpy as np


def assemble(n, periodic, h):
    nx, ny, nz = (int(v) for v in n)
    N = nx * ny * nz
    A = np.zeros((N, N))
    ih2 = 1.0 / (h * h)

    def idx(x, y, z):
        return (z * ny + y) * nx + x

    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                c = idx(x, y, z)
                A[c, c] -= 6.0 * ih2
                for d, dlt in ((0, -1), (0, 1), (1, -1), (1, 1), (2, -1), (2, 1)):
                    q = [x, y, z]
                    q[d] += dlt
                    ext = (nx, ny, nz)[d]
                    if 0 <= q[d] < ext:
                        A[c, idx(*q)] += ih2
                    elif periodic[d]:
                        q[d] %= ext
                        A[c, idx(*q)] += ih2
                    else:
                        A[c, c] -= ih2
    return A


def eigenvalue(n, m, periodic, h):
    """Closed-form eigenvalue of the 7-point operator for mode m (per-dim indices)."""
    lam = 0.0
    for d in range(3):
        if periodic[d]:
            lam += -4.0 / (h * h) * np.sin(np.pi * m[d] / n[d]) ** 2
        else:
            lam += -4.0 / (h * h) * np.sin(np.pi * m[d] / (2.0 * n[d])) ** 2
    return lam


def mode(n, m, periodic):
    """Eigenvector: sin(2 pi m (i+1/2)/n) per periodic dim, sin(pi m (i+1/2)/n) per
    Dirichlet dim; shaped (nz, ny, nx)."""
    f = []
    for d in range(3):
        i = np.arange(n[d]) + 0.5
        f.append(np.sin((2.0 if periodic[d] else 1.0) * np.pi * m[d] * i / n[d]))
    return f[2][:, None, None] * f[1][None, :, None] * f[0][None, None, :]


# ---- one V(nu1, nu2) cycle composed from dense per-level operators ----------------------
#
# A second statement of the solver's cycle, written from the documented schedule alone (it
# calls nothing under oracle/), so that the oracle's cycle can be checked against it:
#
# * levels: level l+1 has half the extents of level l and exists while every extent of level
#   l is even and at least 4; h doubles per level; the same face kinds on every level;
# * half-sweep of colour c ((i+j+k) mod 2 == c): every cell of that colour takes
#   (sum of its six neighbours - h^2 rhs) / 6 with fresh neighbour values (a fill precedes
#   each colour), and a ghost across a Dirichlet face holds -(the cell itself).  Written
#   with the assembled matrix A (whose diagonal already carries those ghosts) this is
#   phi <- phi + (h^2 / 6) D_c (A phi - rhs), D_c the colour mask; cells of one colour
#   only couple to the other colour when every periodic extent is even, so the colour's
#   updates are simultaneous;
# * a sweep is red (0) then black (1); nu1 sweeps before the coarse correction, nu2 after;
# * coarse right-hand side: the mean of the 8 children of the residual rhs - A phi;
#   coarse initial guess 0;
# * bottom: the exact solution (pseudo-inverse, mean-zero answer, when every face is
#   periodic);
# * correction: the coarse value added to each of its 8 children (injection).

def level_extents(n):
    out = [tuple(int(v) for v in n)]
    while all(e % 2 == 0 and e >= 4 for e in out[-1]):
        out.append(tuple(e // 2 for e in out[-1]))
    return out


def colour_mask(n, c):
    nx, ny, nz = n
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return ((i + j + k) % 2 == c).ravel()


def restriction_matrix(nf):
    """(coarse cells x fine cells): each coarse cell gets 1/8 of each of its 8 children."""
    nc = tuple(e // 2 for e in nf)
    Nf, Nc = nf[0] * nf[1] * nf[2], nc[0] * nc[1] * nc[2]
    R = np.zeros((Nc, Nf))
    for z in range(nf[2]):
        for y in range(nf[1]):
            for x in range(nf[0]):
                I = ((z // 2) * nc[1] + y // 2) * nc[0] + x // 2
                R[I, (z * nf[1] + y) * nf[0] + x] = 0.125
    return R


class DenseVCycle:
    def __init__(self, n, periodic, h, nu1=2, nu2=2):
        self.ext = level_extents(n)
        self.periodic = tuple(int(p) for p in periodic)
        self.nu1, self.nu2 = nu1, nu2
        self.A, self.h2, self.masks, self.R = [], [], [], []
        for l, e in enumerate(self.ext):
            hl = h * 2.0 ** l
            self.A.append(assemble(e, self.periodic, hl))
            self.h2.append(hl * hl)
            self.masks.append((colour_mask(e, 0), colour_mask(e, 1)))
            if l + 1 < len(self.ext):
                self.R.append(restriction_matrix(e))
        Ab = self.A[-1]
        self.bottom = np.linalg.pinv(Ab, rcond=1e-10) if all(self.periodic) else np.linalg.inv(Ab)

    def half_sweep(self, l, phi, rhs, c):
        m = self.masks[l][c]
        upd = phi + self.h2[l] / 6.0 * (self.A[l] @ phi - rhs)
        return np.where(m, upd, phi)

    def sweeps(self, l, phi, rhs, count):
        for _ in range(count):
            phi = self.half_sweep(l, phi, rhs, 0)
            phi = self.half_sweep(l, phi, rhs, 1)
        return phi

    def cycle(self, l, phi, rhs):
        if l == len(self.ext) - 1:
            return self.bottom @ rhs
        phi = self.sweeps(l, phi, rhs, self.nu1)
        rc = self.R[l] @ (rhs - self.A[l] @ phi)
        ec = self.cycle(l + 1, np.zeros_like(rc), rc)
        phi = phi + 8.0 * (self.R[l].T @ ec)  # 8 R^T is the injection
        return self.sweeps(l, phi, rhs, self.nu2)

    def run(self, phi0, rhs, k):
        """k V-cycles from phi0 on dense (nz, ny, nx) arrays."""
        phi, b = np.asarray(phi0, np.float64).ravel().copy(), np.asarray(rhs, np.float64).ravel()
        for _ in range(k):
            phi = self.cycle(0, phi, b)
        return phi.reshape(np.asarray(rhs).shape)
