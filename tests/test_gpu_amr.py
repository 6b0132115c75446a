"""Two-level AMR composite solve on the GPU (mg_amr2_residual, mg_amr2_solve) against the
oracle of oracle/amr.py: the composite residual (coarse/fine ghost interpolation, flux
matching) element by element, the iterates of the composite scheme after 1, 2 and 3
iterations, and the converged answer against the exact sparse solution.

Tolerances: the GPU evaluates the same formulas as the oracle with fused multiply-adds and
its own summation order, so values agree to a few units of rounding of the terms they sum:
1e-12 relative to the largest term (12 |phi| / h1^2 for the operator).  A converged answer
(||r||_inf <= tol ||f||_inf) differs from the exact solution by at most ||A^-1||_inf tol
||f||_inf, with ||A^-1||_inf < 0.1 (pinned in tests/test_amr_pins.py)."""
import numpy as np
import pytest
import torch

from oracle import amr
from paper_2403_12179_gb300 import inputs, mg
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

# (coarse cells, region A, region B, coarse max box, fine max box)
CASES = [((16, 16, 16), (4, 4, 4), (12, 12, 12), (8, 8, 8), (8, 8, 8)),
         ((16, 12, 20), (3, 2, 5), (11, 9, 14), (16, 4, 20), (6, 4, 8)),
         ((24, 16, 16), (5, 3, 1), (19, 13, 15), (8, 16, 8), (10, 8, 12))]
FACES = [(0, 0, 0), (1, 1, 1), (0, 1, 1)]


@pytest.fixture(scope="module")
def gctx():
    import paper_2403_12179_gb300.build as b
    b.build()
    assert torch.cuda.is_available()
    ctx = mg.mg_init(0)
    yield ctx
    mg.mg_finalize(ctx)


def _setup(ctx, case, periodic, seed, zero_phi=False):
    n0, A, B, mb0, mb1 = case
    g = amr.Geometry(n0, A, B, periodic)
    r = inputs.rng(seed)
    f0, f1 = r.standard_normal(g.n0[::-1]), r.standard_normal(g.n1[::-1])
    if all(periodic):
        cov = g.covered()
        m = (g.h0 ** 3 * f0[~cov].sum() + g.h1 ** 3 * f1.sum()) / (
            g.h0 ** 3 * (~cov).sum() + g.h1 ** 3 * f1.size)
        f0, f1 = f0 - m, f1 - m
    p0 = np.zeros(g.n0[::-1]) if zero_phi else r.standard_normal(g.n0[::-1])
    p1 = np.zeros(g.n1[::-1]) if zero_phi else r.standard_normal(g.n1[::-1])
    ba0 = mg.mg_box_array_create(ctx, (0, 0, 0), tuple(v - 1 for v in n0), mb0)
    flo = tuple(2 * a for a in A)
    fhi = tuple(2 * b - 1 for b in B)
    ba1 = mg.mg_box_array_create(ctx, flo, fhi, mb1)
    fabs = dict(rhs0=gu.dense_fab(ctx, ba0, f0, 0), phi0=gu.dense_fab(ctx, ba0, p0, 1),
                rhs1=gu.dense_fab(ctx, ba1, f1, 0), phi1=gu.dense_fab(ctx, ba1, p1, 1),
                r0=mg.mg_fab_alloc(ctx, ba0, 1, 0), r1=mg.mg_fab_alloc(ctx, ba1, 1, 0))
    return g, (f0, f1, p0, p1), fabs


def _free(ctx, fabs):
    for f in fabs.values():
        mg.mg_fab_free(ctx, f)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("periodic", FACES)
def test_composite_residual_matches_oracle(gctx, case, periodic):
    g, (f0, f1, p0, p1), F = _setup(gctx, case, periodic, 90)
    nrm = mg.mg_amr2_residual(gctx, F["rhs0"], F["phi0"], F["rhs1"], F["phi1"], mg.make_bc(periodic),
                              0.0, F["r0"], F["r1"])
    q0 = amr.average_down(p0, p1, g)
    o0, o1, onrm = amr.residual(q0, p1, f0, f1, g)
    o0 = amr.average_down(o0, o1, g)          # covered cells: the mean of the fine residual
    r0 = gu.fab_dense(gctx, F["r0"], o0.shape)
    r1 = gu.fab_dense(gctx, F["r1"], o1.shape)
    scale = 12.0 / g.h1 ** 2 * max(np.abs(p0).max(), np.abs(p1).max())
    assert np.abs(r1 - o1).max() <= 1e-12 * scale
    assert np.abs(r0 - o0).max() <= 1e-12 * scale
    assert abs(nrm - onrm) <= 1e-12 * scale
    # the covered coarse cells of phi0 now hold the mean of their children
    assert np.abs(gu.fab_dense(gctx, F["phi0"], q0.shape) - q0).max() <= 1e-15 * np.abs(q0).max()
    _free(gctx, F)


@pytest.mark.parametrize("case", CASES[:2])
@pytest.mark.parametrize("periodic", [(0, 0, 0), (1, 1, 1)])
def test_iterates_match_oracle(gctx, case, periodic):
    for k in (1, 2, 3):
        g, (f0, f1, _, _), F = _setup(gctx, case, periodic, 91, zero_phi=True)
        res = mg.mg_amr2_solve(gctx, F["rhs0"], F["phi0"], F["rhs1"], F["phi1"], mg.make_bc(periodic),
                               1e-10, mg.make_options(fixed_vcycles=k))
        o0, o1, hist = amr.iterate(f0, f1, g, k)
        a0 = gu.fab_dense(gctx, F["phi0"], o0.shape)
        a1 = gu.fab_dense(gctx, F["phi1"], o1.shape)
        scale = max(np.abs(o0).max(), np.abs(o1).max())
        assert res.status == mg.MG_OK and res.vcycles == k
        assert np.abs(a1 - o1).max() <= 1e-11 * scale
        assert np.abs(a0 - o0).max() <= 1e-11 * scale
        assert abs(res.rel_resid - hist[-1]) <= 1e-6 * hist[-1]
        _free(gctx, F)


@pytest.mark.parametrize("case", CASES[:2])
@pytest.mark.parametrize("periodic", [(0, 0, 0), (0, 1, 1)])
def test_solve_reaches_the_exact_composite_solution(gctx, case, periodic):
    tol = 1e-10
    g, (f0, f1, _, _), F = _setup(gctx, case, periodic, 92, zero_phi=True)
    res = mg.mg_amr2_solve(gctx, F["rhs0"], F["phi0"], F["rhs1"], F["phi1"], mg.make_bc(periodic), tol)
    assert res.status == mg.MG_OK and res.rel_resid <= tol and res.vcycles <= 20
    e0, e1 = amr.solve(f0, f1, g)
    a0 = gu.fab_dense(gctx, F["phi0"], e0.shape)
    a1 = gu.fab_dense(gctx, F["phi1"], e1.shape)
    fn = max(np.abs(f0[~g.covered()]).max(), np.abs(f1).max())
    bound = 0.1 * tol * fn
    assert np.abs(a1 - e1).max() <= bound
    assert np.abs((a0 - e0)[~g.covered()]).max() <= bound
    # the residual the oracle measures on the GPU answer meets the tolerance
    _, _, rn = amr.residual(a0, a1, f0, f1, g)
    assert rn <= 1.01 * tol * fn
    _free(gctx, F)


def test_manufactured_solution_second_order(gctx):
    """lap u = f with u = prod sin(pi x_d) on the Dirichlet unit cube, the middle half
    refined: the GPU composite answer's error against u falls about 4x when h halves."""
    errs = []
    for n0 in (16, 32):
        g = amr.Geometry((n0,) * 3, (n0 // 4,) * 3, (3 * n0 // 4,) * 3)

        def u(x, y, z):
            return np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
        f0, f1 = amr.sample(g, lambda x, y, z: -3 * np.pi ** 2 * u(x, y, z))
        u0, u1 = amr.sample(g, u)
        ba0 = mg.mg_box_array_create(gctx, (0, 0, 0), (n0 - 1,) * 3, (16,) * 3)
        ba1 = mg.mg_box_array_create(gctx, (n0 // 2,) * 3, (3 * n0 // 2 - 1,) * 3, (16,) * 3)
        F = dict(rhs0=gu.dense_fab(gctx, ba0, f0, 0), phi0=mg.mg_fab_alloc(gctx, ba0, 1, 1),
                 rhs1=gu.dense_fab(gctx, ba1, f1, 0), phi1=mg.mg_fab_alloc(gctx, ba1, 1, 1))
        res = mg.mg_amr2_solve(gctx, F["rhs0"], F["phi0"], F["rhs1"], F["phi1"], mg.make_bc((0, 0, 0)), 1e-12)
        assert res.status == mg.MG_OK
        a0 = gu.fab_dense(gctx, F["phi0"], u0.shape)
        a1 = gu.fab_dense(gctx, F["phi1"], u1.shape)
        errs.append(max(np.abs(a1 - u1).max(), np.abs((a0 - u0)[~g.covered()]).max()))
        _free(gctx, F)
    assert 3.5 <= errs[0] / errs[1] <= 4.8


def test_refused_layouts(gctx):
    ba0 = mg.mg_box_array_create(gctx, (0, 0, 0), (15, 15, 15), (8, 8, 8))
    c0, c1 = mg.mg_fab_alloc(gctx, ba0, 1, 0), mg.mg_fab_alloc(gctx, ba0, 1, 1)
    bc = mg.make_bc((0, 0, 0))
    # a refined region touching the domain face
    ba1 = mg.mg_box_array_create(gctx, (0, 8, 8), (15, 23, 23), (8, 8, 8))
    f0, f1 = mg.mg_fab_alloc(gctx, ba1, 1, 0), mg.mg_fab_alloc(gctx, ba1, 1, 1)
    with pytest.raises(mg.MgError) as e:
        mg.mg_amr2_solve(gctx, c0, c1, f0, f1, bc, 1e-10)
    assert e.value.code == mg.MG_EINVAL
    # fine boxes with odd bounds
    ba2 = mg.mg_box_array_create(gctx, (8, 8, 8), (23, 23, 23), (5, 8, 8))
    g0, g1 = mg.mg_fab_alloc(gctx, ba2, 1, 0), mg.mg_fab_alloc(gctx, ba2, 1, 1)
    with pytest.raises(mg.MgError) as e:
        mg.mg_amr2_solve(gctx, c0, c1, g0, g1, bc, 1e-10)
    assert e.value.code == mg.MG_EINVAL
    for f in (c0, c1, f0, f1, g0, g1):
        mg.mg_fab_free(gctx, f)


@pytest.mark.parametrize("periodic", [(0, 0, 0), (1, 1, 1)])
def test_graph_replay_equals_eager(gctx, periodic):
    """From the second iteration on the composite iteration is replayed as a CUDA graph; the
    answer equals, bit for bit, the one of eager launches."""
    out = []
    for use_graph in (1, 0):
        g, _, F = _setup(gctx, CASES[0], periodic, 93, zero_phi=True)
        res = mg.mg_amr2_solve(gctx, F["rhs0"], F["phi0"], F["rhs1"], F["phi1"], mg.make_bc(periodic),
                               1e-10, mg.make_options(use_graph=use_graph))
        assert res.status == mg.MG_OK and res.vcycles >= 3
        out.append((res.vcycles, res.rel_resid, gu.fab_dense(gctx, F["phi0"], g.n0[::-1]),
                    gu.fab_dense(gctx, F["phi1"], g.n1[::-1])))
        _free(gctx, F)
    (va, ra, a0, a1), (vb, rb, b0, b1) = out
    assert va == vb and ra == rb
    assert np.array_equal(a0, b0) and np.array_equal(a1, b1)
