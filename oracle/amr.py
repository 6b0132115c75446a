"""Two-level AMR composite Poisson oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference legs
may import this module; the product library never loads it and shares no code with it.

What it computes (AMReX/pyAMReX review, arXiv 2403.12179: Sec. 1 and Sec. 2 describe the
block-structured AMR hierarchy -- a coarse level covering the domain and finer levels covering
sub-regions, with inter-level operations between them -- and name the framework's linear
solvers for cell-centered data; the paper gives no coarse/fine discretisation, so every choice
below is a stated reading):

* Two levels, refinement ratio 2.  Level 0 covers the domain with n0 cells per dimension
  (h0 = 1 / n0[0]); level 1 covers one box region R = [A, B) of coarse cells, at least one
  coarse cell away from every domain face, with cells of size h1 = h0 / 2 (fine cells
  [2A, 2B)).
* Unknowns: every fine cell and every coarse cell outside R.  Coarse cells under R are not
  unknowns of the composite problem.
* Fine operator: the 7-point Laplacian with h1.  A fine neighbour across the coarse/fine
  boundary is a ghost value interpolated quadratically: first in the two tangential
  directions over the 3 x 3 coarse cells of the layer just outside R around the ghost's
  parent cell (3-point Lagrange weights at the fine centre's offset of -1/4 or +1/4 coarse
  cells; the lower-numbered tangential dimension first), then in the normal direction through
  that value (one fine cell width outside the face) and the first two fine cells inside:
  g = 8/15 c + 2/3 f1 - 1/5 f2.
* Coarse operator (cells outside R): the 7-point Laplacian with h0, except that the flux
  through a face shared with R is the mean of the four fine fluxes (phi_in - g) / h1 through
  the fine faces that make it up (flux matching, so the composite operator is conservative).
* Domain faces: homogeneous Dirichlet (ghost = -mirror) or periodic, as on a single level.

Functions work on dense arrays: coarse fields (nz0, ny0, nx0), fine fields (nz1, ny1, nx1)
over R refined, x fastest.  ``apply`` evaluates the operator with vectorised numpy;
``assemble`` builds the same operator as a sparse matrix entry by entry (a second, independent
statement); ``solve`` is the exact composite solution by a sparse direct solve.
"""
from __future__ import annotations

import numpy as np

W_NORMAL = (8.0 / 15.0, 2.0 / 3.0, -1.0 / 5.0)  # coarse value, first, second fine cell


def tangential_weights(delta):
    """3-point Lagrange weights of the nodes -1, 0, +1 at offset delta."""
    return (delta * (delta - 1.0) / 2.0, 1.0 - delta * delta, delta * (delta + 1.0) / 2.0)


W_LO = tangential_weights(-0.25)   # fine cell in the lower half of its parent
W_HI = tangential_weights(0.25)


class Geometry:
    """n0: coarse cells per dimension (x, y, z); A, B: the refined region [A, B) in coarse
    indices; periodic: per-dimension flags (else homogeneous Dirichlet)."""

    def __init__(self, n0, A, B, periodic=(0, 0, 0)):
        self.n0 = tuple(int(v) for v in n0)
        self.A = tuple(int(v) for v in A)
        self.B = tuple(int(v) for v in B)
        self.periodic = tuple(int(p) for p in periodic)
        for d in range(3):
            if not (1 <= self.A[d] < self.B[d] <= self.n0[d] - 1):
                raise ValueError("the refined region must keep one coarse cell from every face")
        self.h0 = 1.0 / self.n0[0]
        self.h1 = self.h0 / 2.0
        self.n1 = tuple(2 * (self.B[d] - self.A[d]) for d in range(3))

    def covered(self):
        """Boolean (nz0, ny0, nx0) mask of the coarse cells under R."""
        m = np.zeros(self.n0[::-1], bool)
        m[self.A[2]:self.B[2], self.A[1]:self.B[1], self.A[0]:self.B[0]] = True
        return m


# ---- the operator, vectorised ---------------------------------------------------------

def _coarse_padded(phi0, g):
    """phi0 with one ghost layer from the domain faces (periodic image / -mirror)."""
    p = np.pad(phi0, 1)
    for ax, d in ((2, 0), (1, 1), (0, 2)):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax], hi[ax] = 0, -1
        a = [slice(None)] * 3
        b = [slice(None)] * 3
        if g.periodic[d]:
            a[ax], b[ax] = -2, 1
            p[tuple(lo)] = p[tuple(a)]
            p[tuple(hi)] = p[tuple(b)]
        else:
            a[ax], b[ax] = 1, -2
            p[tuple(lo)] = -p[tuple(a)]
            p[tuple(hi)] = -p[tuple(b)]
    return p


def cf_ghosts(phi0, phi1, g):
    """The fine field with one ghost layer whose face cells hold the coarse/fine
    interpolation (edge and corner ghosts, unused by the 7-point stencil, are NaN)."""
    n1 = g.n1
    p = np.full((n1[2] + 2, n1[1] + 2, n1[0] + 2), np.nan)
    p[1:-1, 1:-1, 1:-1] = phi1
    for d in range(3):                       # normal dimension (x, y, z)
        t = [e for e in range(3) if e != d]  # tangential dimensions, lower first
        for side in (0, 1):
            X = g.A[d] - 1 if side == 0 else g.B[d]          # coarse layer outside R
            # every fine ghost of this face: fine tangential indices (i, j) over R refined
            ti = np.arange(n1[t[0]])
            tj = np.arange(n1[t[1]])
            I, J = np.meshgrid(ti, tj, indexing="ij")      # I along t[0], J along t[1]
            P0 = g.A[t[0]] + I // 2                        # parent coarse indices
            P1 = g.A[t[1]] + J // 2
            w0 = np.where((I % 2)[..., None] == 0, np.array(W_LO), np.array(W_HI))
            w1 = np.where((J % 2)[..., None] == 0, np.array(W_LO), np.array(W_HI))
            c = np.zeros(I.shape)
            for q in range(3):                             # along t[1]
                cq = np.zeros(I.shape)
                for pp in range(3):                        # along t[0]
                    idx = [0, 0, 0]
                    idx[d] = X
                    idx[t[0]] = P0 + pp - 1
                    idx[t[1]] = P1 + q - 1
                    cq = cq + w0[..., pp] * phi0[idx[2], idx[1], idx[0]]
                c = c + w1[..., q] * cq
            # the first two fine cells inside, along the normal
            f = []
            for k in (0, 1):
                idx = [None, None, None]
                idx[d] = k if side == 0 else n1[d] - 1 - k
                idx[t[0]] = I
                idx[t[1]] = J
                f.append(phi1[idx[2], idx[1], idx[0]])
            gval = W_NORMAL[0] * c + W_NORMAL[1] * f[0] + W_NORMAL[2] * f[1]
            idx = [None, None, None]
            idx[d] = 0 if side == 0 else n1[d] + 1
            idx[t[0]] = I + 1
            idx[t[1]] = J + 1
            p[idx[2], idx[1], idx[0]] = gval
    return p


def apply(phi0, phi1, g):
    """(A phi) on fine cells and on coarse cells; covered coarse entries are 0."""
    h0, h1 = g.h0, g.h1
    pf = cf_ghosts(phi0, phi1, g)
    c = pf[1:-1, 1:-1, 1:-1]
    a1 = (pf[1:-1, 1:-1, :-2] + pf[1:-1, 1:-1, 2:] + pf[1:-1, :-2, 1:-1] + pf[1:-1, 2:, 1:-1] +
          pf[:-2, 1:-1, 1:-1] + pf[2:, 1:-1, 1:-1] - 6.0 * c) / (h1 * h1)
    pc = _coarse_padded(phi0, g)
    # fluxes through the +x, +y, +z faces of every coarse cell (face i between i and i+1)
    fx = (pc[1:-1, 1:-1, 1:] - pc[1:-1, 1:-1, :-1]) / h0   # (nz, ny, nx + 1)
    fy = (pc[1:-1, 1:, 1:-1] - pc[1:-1, :-1, 1:-1]) / h0
    fz = (pc[1:, 1:-1, 1:-1] - pc[:-1, 1:-1, 1:-1]) / h0
    # faces shared with R: the mean of the four fine fluxes
    ff = [(pf[1:-1, 1:-1, 1:] - pf[1:-1, 1:-1, :-1]) / h1,
          (pf[1:-1, 1:, 1:-1] - pf[1:-1, :-1, 1:-1]) / h1,
          (pf[1:, 1:-1, 1:-1] - pf[:-1, 1:-1, 1:-1]) / h1]
    for d, F in ((0, fx), (1, fy), (2, fz)):
        t = [e for e in range(3) if e != d]
        for side in (0, 1):
            fi = 0 if side == 0 else g.n1[d]          # fine face index along d
            ci = g.A[d] if side == 0 else g.B[d]      # coarse face index (between ci-1, ci)
            fine_face = np.take(ff[d], fi, axis=2 - d)  # (fine tangential, z-major order)
            # mean over 2 x 2 blocks in the tangential dims
            s = fine_face.reshape(fine_face.shape[0] // 2, 2, fine_face.shape[1] // 2, 2).mean(axis=(1, 3))
            sl = [slice(None)] * 3
            sl[2 - d] = ci
            sl[2 - t[0]] = slice(g.A[t[0]], g.B[t[0]])
            sl[2 - t[1]] = slice(g.A[t[1]], g.B[t[1]])
            F[tuple(sl)] = s
    a0 = ((fx[:, :, 1:] - fx[:, :, :-1]) + (fy[:, 1:, :] - fy[:, :-1, :]) +
          (fz[1:, :, :] - fz[:-1, :, :])) / h0
    a0 = np.where(g.covered(), 0.0, a0)
    return a0, a1


def residual(phi0, phi1, f0, f1, g):
    """Composite residual (covered coarse entries 0) and its max-norm."""
    a0, a1 = apply(phi0, phi1, g)
    r0 = np.where(g.covered(), 0.0, f0 - a0)
    r1 = f1 - a1
    return r0, r1, max(float(np.abs(r0).max()), float(np.abs(r1).max()))


# ---- the same operator as a sparse matrix, entry by entry -----------------------------

def unknowns(g):
    """Index maps: fine cell -> row, uncovered coarse cell -> row (fine cells first)."""
    n1, n0 = g.n1, g.n0
    nf = n1[0] * n1[1] * n1[2]
    cov = g.covered()
    cidx = -np.ones(n0[::-1], np.int64)
    free = np.flatnonzero(~cov.ravel())
    cidx.ravel()[free] = nf + np.arange(free.size)
    fidx = np.arange(nf).reshape(n1[::-1])
    return fidx, cidx, nf + free.size


def assemble(g):
    """Sparse composite matrix over [fine cells, uncovered coarse cells] (x fastest)."""
    import scipy.sparse as sp
    fidx, cidx, N = unknowns(g)
    rows, cols, vals = [], [], []
    h0, h1 = g.h0, g.h1
    n0, n1, A, B = g.n0, g.n1, g.A, g.B

    def add(r, c, v):
        rows.append(r)
        cols.append(c)
        vals.append(v)

    def coarse_nb(X, dim, step, r, w):
        """w * (coarse neighbour value) into row r, through the domain faces."""
        q = list(X)
        q[dim] += step
        if 0 <= q[dim] < n0[dim]:
            add(r, cidx[q[2], q[1], q[0]], w)
        elif g.periodic[dim]:
            q[dim] %= n0[dim]
            add(r, cidx[q[2], q[1], q[0]], w)
        else:
            add(r, cidx[X[2], X[1], X[0]], -w)      # ghost = -(the cell itself)

    def ghost_terms(fcell, dim, side):
        """The C/F ghost beside fine cell fcell across face (dim, side): list of
        (column, weight)."""
        t = [e for e in range(3) if e != dim]
        X = A[dim] - 1 if side == 0 else B[dim]
        terms = []
        par = [A[e] + fcell[e] // 2 for e in range(3)]
        w0 = W_LO if fcell[t[0]] % 2 == 0 else W_HI
        w1 = W_LO if fcell[t[1]] % 2 == 0 else W_HI
        for q in range(3):
            for p in range(3):
                c = [0, 0, 0]
                c[dim] = X
                c[t[0]] = par[t[0]] + p - 1
                c[t[1]] = par[t[1]] + q - 1
                terms.append((cidx[c[2], c[1], c[0]], W_NORMAL[0] * w0[p] * w1[q]))
        for k, wn in ((0, W_NORMAL[1]), (1, W_NORMAL[2])):
            f = list(fcell)
            f[dim] = k if side == 0 else n1[dim] - 1 - k
            terms.append((fidx[f[2], f[1], f[0]], wn))
        return terms

    # fine rows
    for k in range(n1[2]):
        for j in range(n1[1]):
            for i in range(n1[0]):
                r = fidx[k, j, i]
                cellf = (i, j, k)
                add(r, r, -6.0 / h1 ** 2)
                for dim in range(3):
                    for side, step in ((0, -1), (1, 1)):
                        q = list(cellf)
                        q[dim] += step
                        if 0 <= q[dim] < n1[dim]:
                            add(r, fidx[q[2], q[1], q[0]], 1.0 / h1 ** 2)
                        else:
                            for col, w in ghost_terms(cellf, dim, side):
                                add(r, col, w / h1 ** 2)
    # coarse rows (uncovered cells)
    cov = g.covered()
    for Z in range(n0[2]):
        for Y in range(n0[1]):
            for X in range(n0[0]):
                if cov[Z, Y, X]:
                    continue
                r = cidx[Z, Y, X]
                C = (X, Y, Z)
                for dim in range(3):
                    for side, step in ((0, -1), (1, 1)):
                        q = list(C)
                        q[dim] += step
                        inside = all(0 <= q[e] < n0[e] for e in range(3))
                        if inside and cov[q[2], q[1], q[0]]:
                            # the face shared with R: mean of the four fine fluxes, taken in
                            # the outward direction of this coarse cell
                            fs = 0 if step > 0 else 1   # R's face: low side when R is at +step
                            t = [e for e in range(3) if e != dim]
                            base = [0, 0, 0]
                            base[dim] = 0 if fs == 0 else n1[dim] - 1
                            for a in range(2):
                                for b in range(2):
                                    f = list(base)
                                    f[t[0]] = 2 * (C[t[0]] - A[t[0]]) + a
                                    f[t[1]] = 2 * (C[t[1]] - A[t[1]]) + b
                                    # outward flux (phi_f - g_f) / h1 divided by h0, mean of 4
                                    w = 0.25 / (h1 * h0)
                                    add(r, fidx[f[2], f[1], f[0]], w)
                                    for col, wg in ghost_terms(tuple(f), dim, fs):
                                        add(r, col, -w * wg)
                        else:
                            add(r, r, -1.0 / h0 ** 2)
                            coarse_nb(C, dim, step, r, 1.0 / h0 ** 2)
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))


def pack(phi0, phi1, g):
    fidx, cidx, N = unknowns(g)
    v = np.zeros(N)
    v[fidx.ravel()] = phi1.ravel()
    m = cidx >= 0
    v[cidx[m]] = phi0[m]
    return v


def unpack(v, g):
    fidx, cidx, N = unknowns(g)
    phi1 = v[fidx.ravel()].reshape(g.n1[::-1])
    phi0 = np.zeros(g.n0[::-1])
    m = cidx >= 0
    phi0[m] = v[cidx[m]]
    return phi0, phi1


def solve(f0, f1, g):
    """Exact composite solution (sparse LU).  Covered coarse entries hold the mean of their
    8 fine children.  With every face periodic the operator is singular: the answer is the
    one with zero mean over the composite cells (volume-weighted)."""
    import scipy.sparse.linalg as sla
    Amat = assemble(g)
    b = pack(f0, f1, g)
    if all(g.periodic):
        # append the volume-weighted mean constraint as a Lagrange multiplier
        import scipy.sparse as sp
        fidx, cidx, N = unknowns(g)
        w = np.zeros(N)
        w[:fidx.size] = g.h1 ** 3
        w[fidx.size:] = g.h0 ** 3
        K = sp.bmat([[Amat, sp.csr_matrix(w[:, None])], [sp.csr_matrix(w[None, :]), None]], format="csc")
        x = sla.spsolve(K, np.concatenate([b, [0.0]]))[:N]
    else:
        x = sla.spsolve(Amat.tocsc(), b)
    phi0, phi1 = unpack(x, g)
    return average_down(phi0, phi1, g), phi1


def average_down(phi0, phi1, g):
    """phi0 with every covered cell replaced by the mean of its 8 fine children."""
    out = phi0.copy()
    n1 = g.n1
    m = phi1.reshape(n1[2] // 2, 2, n1[1] // 2, 2, n1[0] // 2, 2).mean(axis=(1, 3, 5))
    out[g.A[2]:g.B[2], g.A[1]:g.B[1], g.A[0]:g.B[0]] = m
    return out


def sample(g, fn):
    """fn(x, y, z) at the coarse and fine cell centres (dense arrays)."""
    def centres(n, h, off):
        return (np.arange(n) + 0.5) * h + off
    xc = [centres(g.n0[d], g.h0, 0.0) for d in range(3)]
    xf = [centres(g.n1[d], g.h1, g.A[d] * g.h0) for d in range(3)]
    Zc, Yc, Xc = np.meshgrid(xc[2], xc[1], xc[0], indexing="ij")
    Zf, Yf, Xf = np.meshgrid(xf[2], xf[1], xf[0], indexing="ij")
    return fn(Xc, Yc, Zc), fn(Xf, Yf, Zf)


# ---- the iteration the GPU solver runs, step by step ----------------------------------

def fine_half_sweep(phi0, phi1, f1, g, color):
    """One red-black half-sweep of the fine level (colour on fine global indices), the
    coarse/fine ghosts taken from phi0 and phi1 as they are before it."""
    pf = cf_ghosts(phi0, phi1, g)
    n1 = g.n1
    k, j, i = np.meshgrid(np.arange(n1[2]), np.arange(n1[1]), np.arange(n1[0]), indexing="ij")
    col = ((i + 2 * g.A[0]) + (j + 2 * g.A[1]) + (k + 2 * g.A[2])) % 2 == color
    s = (pf[1:-1, 1:-1, :-2] + pf[1:-1, 1:-1, 2:] + pf[1:-1, :-2, 1:-1] + pf[1:-1, 2:, 1:-1] +
         pf[:-2, 1:-1, 1:-1] + pf[2:, 1:-1, 1:-1])
    return np.where(col, (s - g.h1 * g.h1 * f1) / 6.0, phi1)


def iterate(f0, f1, g, k, nu1=2, nu2=2):
    """k iterations of the composite scheme from phi = 0: composite residual; one V(nu1, nu2)
    cycle of the single-level oracle on level 0 for it (covered cells: the mean of the fine
    residual); phi0 += e0, phi1 += e0 of the parent; nu1 + nu2 fine red-black sweeps;
    covered coarse cells take the mean of their children.  Returns (phi0, phi1, history of
    the composite residual norm relative to ||f||)."""
    import oracle
    phi0, phi1 = np.zeros(g.n0[::-1]), np.zeros(g.n1[::-1])
    cov = g.covered()
    fn = max(float(np.abs(f0[~cov]).max()), float(np.abs(f1).max()))
    dlo, dhi = (0, 0, 0), tuple(v - 1 for v in g.n0)
    boxes = oracle.chop(dlo, dhi, g.n0)
    hist = []
    for _ in range(k):
        r0, r1, rn = residual(phi0, phi1, f0, f1, g)
        hist.append(rn / fn)
        rc = average_down(r0, r1, g)
        e0, st, _, _ = oracle.solve(dlo, dhi, g.periodic, boxes, g.h0, rc, fixed_vcycles=1,
                                    nu1=nu1, nu2=nu2)
        phi0 = phi0 + e0
        sub = e0[g.A[2]:g.B[2], g.A[1]:g.B[1], g.A[0]:g.B[0]]
        phi1 = phi1 + np.repeat(np.repeat(np.repeat(sub, 2, 0), 2, 1), 2, 2)
        for _s in range(nu1 + nu2):
            for color in (0, 1):
                phi1 = fine_half_sweep(phi0, phi1, f1, g, color)
        phi0 = average_down(phi0, phi1, g)
    _, _, rn = residual(phi0, phi1, f0, f1, g)
    hist.append(rn / fn)
    return phi0, phi1, np.array(hist)
