"""Pins for the two-level AMR composite oracle (oracle/amr.py): checks against mathematics,
not against the oracle itself.

* the vectorised operator equals the independently assembled sparse matrix;
* exactness on quadratic polynomials: the quadratic coarse/fine interpolation and the
  flux-matched coarse cells reproduce lap(u) exactly wherever the stencil stays off the
  domain faces (a wrong interpolation weight, a dropped flux term or a wrong flux sign
  breaks it);
* conservation: on a periodic domain the volume-weighted sum of A phi vanishes for any phi
  (it does not without the flux matching, which the mutation case shows);
* second-order convergence of the exact composite solution to a smooth solution under
  refinement, and a smaller error than the coarse level alone;
* the composite null space: constants (periodic) give A phi = 0.
"""
import numpy as np
import pytest

from oracle import amr
from paper_2403_12179_gb300 import inputs

GEOMS = [((8, 8, 8), (2, 2, 2), (6, 6, 6)), ((12, 8, 10), (3, 2, 4), (8, 5, 7)),
         ((10, 10, 10), (1, 4, 2), (9, 6, 5))]
FACES = [(0, 0, 0), (1, 1, 1), (1, 0, 1)]


def _rand(g, seed):
    r = inputs.rng(seed)
    return r.standard_normal(g.n0[::-1]), r.standard_normal(g.n1[::-1])


@pytest.mark.parametrize("n0,A,B", GEOMS)
@pytest.mark.parametrize("periodic", FACES)
def test_apply_equals_assembled_matrix(n0, A, B, periodic):
    g = amr.Geometry(n0, A, B, periodic)
    p0, p1 = _rand(g, 80)
    a0, a1 = amr.apply(p0, p1, g)
    m0, m1 = amr.unpack(amr.assemble(g) @ amr.pack(p0, p1, g), g)
    cov = g.covered()
    scale = 24.0 / g.h1 ** 2
    assert np.abs(a1 - m1).max() <= 1e-14 * scale
    assert np.abs((a0 - m0)[~cov]).max() <= 1e-14 * scale


@pytest.mark.parametrize("n0,A,B", GEOMS)
def test_quadratic_exactness(n0, A, B):
    g = amr.Geometry(n0, A, B, (0, 0, 0))
    c = inputs.rng(81).standard_normal(10)

    def u(x, y, z):
        return (c[0] * x * x + c[1] * y * y + c[2] * z * z + c[3] * x * y + c[4] * y * z +
                c[5] * x * z + c[6] * x + c[7] * y + c[8] * z + c[9])
    lap = 2.0 * (c[0] + c[1] + c[2])
    u0, u1 = amr.sample(g, u)
    a0, a1 = amr.apply(u0, u1, g)
    tol = 1e-9 * (1.0 + abs(lap))
    assert np.abs(a1 - lap).max() <= tol
    # coarse cells whose stencil stays off the domain faces (those read -mirror ghosts)
    interior = np.zeros(g.n0[::-1], bool)
    interior[1:-1, 1:-1, 1:-1] = True
    m = interior & ~g.covered()
    assert np.abs(a0[m] - lap).max() <= tol


@pytest.mark.parametrize("n0,A,B", GEOMS)
def test_conservation_on_a_periodic_domain(n0, A, B):
    g = amr.Geometry(n0, A, B, (1, 1, 1))
    p0, p1 = _rand(g, 82)
    a0, a1 = amr.apply(p0, p1, g)
    cov = g.covered()
    total = g.h0 ** 3 * a0[~cov].sum() + g.h1 ** 3 * a1.sum()
    scale = g.h0 ** 3 * np.abs(a0).sum() + g.h1 ** 3 * np.abs(a1).sum()
    assert abs(total) <= 1e-13 * scale
    # without flux matching (coarse differences against the averaged-down fine values on the
    # shared faces) the composite sum does not vanish
    q0 = amr.average_down(p0, p1, g)
    pc = np.pad(q0, 1, mode="wrap")
    plain = (pc[1:-1, 1:-1, :-2] + pc[1:-1, 1:-1, 2:] + pc[1:-1, :-2, 1:-1] + pc[1:-1, 2:, 1:-1] +
             pc[:-2, 1:-1, 1:-1] + pc[2:, 1:-1, 1:-1] - 6 * q0) / g.h0 ** 2
    bad = g.h0 ** 3 * plain[~cov].sum() + g.h1 ** 3 * a1.sum()
    assert abs(bad) > 1e-6 * scale


def test_constants_are_the_periodic_null_space():
    g = amr.Geometry((8, 8, 8), (2, 3, 2), (6, 5, 7), (1, 1, 1))
    a0, a1 = amr.apply(np.full(g.n0[::-1], 3.5), np.full(g.n1[::-1], 3.5), g)
    assert np.abs(a1).max() <= 1e-11 and np.abs(a0[~g.covered()]).max() <= 1e-11


def _manufactured_error(n0):
    g = amr.Geometry((n0,) * 3, (n0 // 4,) * 3, (3 * n0 // 4,) * 3)

    def u(x, y, z):
        return np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
    f0, f1 = amr.sample(g, lambda x, y, z: -3 * np.pi ** 2 * u(x, y, z))
    u0, u1 = amr.sample(g, u)
    p0, p1 = amr.solve(f0, f1, g)
    cov = g.covered()
    return max(np.abs(p1 - u1).max(), np.abs((p0 - u0)[~cov]).max()), np.abs(p1 - u1).max()


def test_second_order_convergence_of_the_composite_solution():
    e8, _ = _manufactured_error(8)
    e16, f16 = _manufactured_error(16)
    assert 3.5 <= e8 / e16 <= 4.8
    # the refined region is more accurate than the coarse level alone: there the discrete
    # solution is u * 3 pi^2 / |lambda_h| with lambda_h = -(12 / h^2) sin^2(pi h / 2)
    h = 1.0 / 16
    coarse_only = abs(3 * np.pi ** 2 / (12 / h ** 2 * np.sin(np.pi * h / 2) ** 2) - 1.0)
    assert f16 < coarse_only


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 1, 0)])
def test_exact_solve_has_zero_residual(periodic):
    g = amr.Geometry((8, 10, 8), (2, 3, 2), (5, 7, 6), periodic)
    f0, f1 = _rand(g, 83)
    if all(periodic):
        cov = g.covered()
        mean = (g.h0 ** 3 * f0[~cov].sum() + g.h1 ** 3 * f1.sum()) / (
            g.h0 ** 3 * (~cov).sum() + g.h1 ** 3 * f1.size)
        f0, f1 = f0 - mean, f1 - mean
    p0, p1 = amr.solve(f0, f1, g)
    _, _, rn = amr.residual(p0, p1, f0, f1, g)
    assert rn <= 1e-10 * max(np.abs(f0).max(), np.abs(f1).max())
    # covered coarse cells hold the mean of their children
    np.testing.assert_allclose(p0, amr.average_down(p0, p1, g), rtol=0, atol=0)


def test_iteration_converges_to_the_exact_composite_solution():
    """The composite iteration (coarse V-cycle on the composite residual, fine sweeps with
    coarse/fine ghosts) contracts the residual by at least 4x per step and reaches the sparse
    direct solution."""
    g = amr.Geometry((16, 16, 16), (4, 4, 4), (12, 12, 12), (0, 0, 0))
    f0, f1 = _rand(g, 84)
    p0, p1, hist = amr.iterate(f0, f1, g, 12)
    assert np.all(hist[1:] <= 0.25 * hist[:-1]) and hist[-1] < 1e-10
    e0, e1 = amr.solve(f0, f1, g)
    cov = g.covered()
    assert np.abs(p1 - e1).max() <= 1e-10 * np.abs(e1).max()
    assert np.abs((p0 - e0)[~cov]).max() <= 1e-10 * np.abs(e1).max()


def test_composite_inverse_norm_bound_at_8():
    """||A^-1||_inf of the composite operator (Dirichlet unit cube, refined middle) is below
    0.1 -- the constant the GPU tests use to turn a residual into an error bound (the
    continuous problem's value is about 0.056)."""
    g = amr.Geometry((8, 8, 8), (2, 2, 2), (6, 6, 6), (0, 0, 0))
    A = amr.assemble(g).toarray()
    inv = np.linalg.inv(A)
    assert np.abs(inv).sum(axis=1).max() < 0.1
