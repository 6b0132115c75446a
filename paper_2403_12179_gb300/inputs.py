"""Seeded synthetic inputs for the multigrid Poisson workloads.

This module only draws and shapes input data; it holds none of the solver's arithmetic.
Both the CUDA path and the CPU oracle are fed from here.  Every generator uses NumPy's
``PCG64`` bit generator with a fixed seed and returns dense domain arrays shaped
``(nz, ny, nx)`` (x fastest), cell ``(i, j, k)`` centred at ``((i+1/2)h, (j+1/2)h, (k+1/2)h)``
on the unit cube, ``h = 1/n``.

Workloads (unit cube, ``A phi = rhs`` with the 7-point Laplacian):

* ``periodic_sine``  64^3 periodic, 8 boxes of 32^3:
  ``rhs = -12 pi^2 prod sin(2 pi x_d) + U(-1e-3, 1e-3)``, exact mean removed.
* ``dirichlet_jacobi`` 256^3 homogeneous Dirichlet, 64 boxes of 64^3: i.i.d. N(0,1) per
  cell, then one damped-Jacobi pass ``r <- (6 r_c + sum of 6 neighbours) / 12`` with
  neighbours outside the domain taken as ``-r_c``.
* ``fill_microbench`` same layout, 4 components, 2 ghosts, periodic, values U(0,1).
* ``batched_periodic`` 512 periodic problems, edges drawn from {32,48,64,96,128},
  N(0,1) with the mean removed.
* ``gaussian_blobs`` 512^3 Dirichlet: 16 blobs ``a exp(-|x-c|^2 / (2 s^2))``,
  ``c ~ U(0,1)^3``, ``s ~ U(0.02, 0.1)``, ``a ~ N(0,1)``, plus N(0, 1e-3) noise.
* ``serving_requests`` Poisson arrivals (mean rate 200/s), edge from {32,64,128,256} with
  probabilities {0.4,0.3,0.2,0.1}, periodic / Dirichlet 50/50, box edge 32 or 64 (50/50).
"""
from __future__ import annotations

import dataclasses

import numpy as np

PI = np.pi


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def centers(n: int) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def remove_mean(a: np.ndarray) -> np.ndarray:
    """Subtract the mean (NumPy's pairwise sum over the flattened array, a fixed order)."""
    return a - np.sum(a, dtype=np.float64) / a.size


def periodic_sine(n: int = 64, seed: int = 1, noise: float = 1e-3) -> np.ndarray:
    x = centers(n)
    s = np.sin(2 * PI * x)
    rhs = -12.0 * PI * PI * (s[:, None, None] * s[None, :, None] * s[None, None, :])
    if noise:
        rhs = rhs + rng(seed).uniform(-noise, noise, size=(n, n, n))
    return np.ascontiguousarray(remove_mean(rhs))


def sine_mode(n, m, periodic=True):
    """prod_d sin(2 pi m_d x_d) (periodic) or prod_d sin(pi m_d x_d) (Dirichlet) at cell
    centres, shaped (nz, ny, nx); ``n`` and ``m`` are (nx, ny, nz) triples."""
    f = []
    for d in range(3):
        x = centers(n[d])
        f.append(np.sin((2.0 if periodic else 1.0) * PI * m[d] * x))
    return np.ascontiguousarray(f[2][:, None, None] * f[1][None, :, None] * f[0][None, None, :])


def dirichlet_jacobi(n: int = 256, seed: int = 2) -> np.ndarray:
    r = rng(seed).standard_normal(size=(n, n, n))
    p = np.empty((n + 2, n + 2, n + 2))
    p[1:-1, 1:-1, 1:-1] = r
    out = 6.0 * r
    # neighbour sum with out-of-domain neighbours = -r_c (input recipe, not the solver)
    for axis in range(3):
        for side in (-1, 1):
            nb = np.roll(r, -side, axis=axis)
            idx = [slice(None)] * 3
            idx[axis] = slice(n - 1, n) if side == 1 else slice(0, 1)
            nb[tuple(idx)] = -r[tuple(idx)]
            out += nb
    return np.ascontiguousarray(out / 12.0)


def fill_microbench(n: int = 256, box: int = 64, ncomp: int = 4, seed: int = 3) -> np.ndarray:
    return np.ascontiguousarray(rng(seed).uniform(0.0, 1.0, size=(ncomp, n, n, n)))


@dataclasses.dataclass
class Problem:
    n: int
    periodic: bool
    box: int
    seed: int

    def rhs(self) -> np.ndarray:
        r = rng(self.seed).standard_normal(size=(self.n, self.n, self.n))
        return np.ascontiguousarray(remove_mean(r) if self.periodic else r)


def batched_periodic(count: int = 512, seed: int = 4, edges=(32, 48, 64, 96, 128), box: int = 32):
    g = rng(seed)
    ns = g.choice(np.asarray(edges), size=count)
    return [Problem(int(n), True, box, seed * 100003 + i) for i, n in enumerate(ns)]


def gaussian_blobs(n: int = 512, seed: int = 5, nblob: int = 16, noise: float = 1e-3,
                   dtype=np.float64) -> np.ndarray:
    g = rng(seed)
    c = g.uniform(0.0, 1.0, size=(nblob, 3))
    s = g.uniform(0.02, 0.1, size=nblob)
    a = g.standard_normal(size=nblob)
    x = centers(n)
    out = np.zeros((n, n, n), dtype)
    for k in range(nblob):
        ex = np.exp(-((x - c[k, 0]) ** 2) / (2 * s[k] ** 2))
        ey = np.exp(-((x - c[k, 1]) ** 2) / (2 * s[k] ** 2))
        ez = np.exp(-((x - c[k, 2]) ** 2) / (2 * s[k] ** 2))
        out += (a[k] * ez)[:, None, None] * ey[None, :, None] * ex[None, None, :]
    out += g.normal(0.0, noise, size=(n, n, n))
    return np.ascontiguousarray(out)


def amr_sine(n0: int, A, B):
    """A two-level problem with known solution: level 0 covers the unit cube with n0^3
    cells, level 1 the coarse box region [A, B) refined by 2.  Returns (f0, f1, u0, u1):
    f = -3 pi^2 u and u = prod sin(pi x_d) at the cell centres of each level (dense arrays
    (nz, ny, nx); level 1 spans the refined region only)."""
    h0 = 1.0 / n0
    x0 = centers(n0)
    xs = [(np.arange(2 * (B[d] - A[d])) + 0.5) * (h0 / 2) + A[d] * h0 for d in range(3)]

    def field(xx, yy, zz):
        s = [np.sin(PI * v) for v in (xx, yy, zz)]
        return s[2][:, None, None] * s[1][None, :, None] * s[0][None, None, :]
    u0 = field(x0, x0, x0)
    u1 = field(*xs)
    return (np.ascontiguousarray(-3 * PI * PI * u0), np.ascontiguousarray(-3 * PI * PI * u1),
            np.ascontiguousarray(u0), np.ascontiguousarray(u1))


@dataclasses.dataclass
class Request:
    t_arrive: float
    n: int
    periodic: bool
    box: int
    seed: int

    def rhs(self) -> np.ndarray:
        r = rng(self.seed).standard_normal(size=(self.n, self.n, self.n))
        return np.ascontiguousarray(remove_mean(r) if self.periodic else r)

    def rhs_into(self, out: np.ndarray) -> np.ndarray:
        """The same values as rhs(), drawn into a caller's C-contiguous (n, n, n) float64
        array (e.g. pinned host memory), without a temporary of the request's size."""
        assert out.shape == (self.n,) * 3 and out.dtype == np.float64 and out.flags.c_contiguous
        rng(self.seed).standard_normal(out=out)
        if self.periodic:
            out -= np.sum(out, dtype=np.float64) / out.size
        return out


def serving_requests(count: int = 5000, rate: float = 200.0, seed: int = 6,
                     edges=(32, 64, 128, 256), probs=(0.4, 0.3, 0.2, 0.1)):
    g = rng(seed)
    t = np.cumsum(g.exponential(1.0 / rate, size=count))
    ns = g.choice(np.asarray(edges), size=count, p=np.asarray(probs))
    per = g.uniform(size=count) < 0.5
    bx = np.where(g.uniform(size=count) < 0.5, 32, 64)
    return [Request(float(t[i]), int(ns[i]), bool(per[i]), int(min(bx[i], ns[i])), seed * 1000003 + i)
            for i in range(count)]
