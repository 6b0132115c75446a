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
