"""Pins for the CPU oracle: checks against mathematics, not against the oracle itself.

The paper (AMReX/pyAMReX review, Sec. 2) only names cell-centered linear solvers and ghost
cell exchange, and prints no worked example for them; every check here follows from closed
forms, brute force or exact identities:

* ghost fill vs a closed-form function of global position (periodic wrap / -mirror / 0)
* operator vs closed-form eigenvalues of the discrete sine / Fourier modes (P1)
* operator vs an independently assembled dense matrix; bottom (pseudo-)inverse vs numpy (P3)
* full solve vs dense direct solve at 8^3 (P3), vs eigenmode / lambda (P1)
* exact discrete solution of the periodic sine problem, second-order error ratios (P2)
* restriction / prolongation identities and adjointness (P6)
* Gauss-Seidel property (coloured residuals vanish), decomposition invariance (P5)
* mixed-precision result within the a-priori error bound (P7)
* the V-cycle schedule (sweep counts, colour order, transfers, bottom) and the mixed form's
  outer iteration vs a dense composition of per-level matrices, one and two cycles
"""
import numpy as np
import pytest

from paper_2403_12179_gb300 import inputs
from tests import dense_ref

Z3 = (0, 0, 0)


def _dom(n):
    return Z3, tuple(int(v) - 1 for v in n)


def _field_fn(x, y, z, c):
    return x + 100.0 * y + 10000.0 * z + 1e6 * c


def _expected_ghost(p, dlo, dhi, periodic, c):
    q = list(p)
    out = []
    for d in range(3):
        n = dhi[d] - dlo[d] + 1
        if periodic[d]:
            q[d] = dlo[d] + (q[d] - dlo[d]) % n
        elif q[d] < dlo[d] or q[d] > dhi[d]:
            out.append(d)
    if not out:
        return _field_fn(*q, c)
    if len(out) == 1:
        d = out[0]
        q[d] = 2 * dlo[d] - 1 - q[d] if q[d] < dlo[d] else 2 * dhi[d] + 1 - q[d]
        return -_field_fn(*q, c)
    return 0.0


def _check_fill(orc, dlo, dhi, periodic, boxes, ng, ncomp):
    fabs = orc.new_field(boxes, ng, ncomp)
    for f, b in zip(fabs, boxes):
        f[...] = np.nan
        for c in range(ncomp):
            for k in range(b[2], b[5] + 1):
                for j in range(b[1], b[4] + 1):
                    for i in range(b[0], b[3] + 1):
                        f[c, k - b[2] + ng, j - b[1] + ng, i - b[0] + ng] = _field_fn(i, j, k, c)
    out = orc.fill_boundary(dlo, dhi, periodic, boxes, fabs, ng)
    for f, b in zip(out, boxes):
        for c in range(ncomp):
            for k in range(b[2] - ng, b[5] + ng + 1):
                for j in range(b[1] - ng, b[4] + ng + 1):
                    for i in range(b[0] - ng, b[3] + ng + 1):
                        got = f[c, k - b[2] + ng, j - b[1] + ng, i - b[0] + ng]
                        inside = (b[0] <= i <= b[3] and b[1] <= j <= b[4] and b[2] <= k <= b[5])
                        want = _field_fn(i, j, k, c) if inside else \
                            _expected_ghost((i, j, k), dlo, dhi, periodic, c)
                        assert got == want, ((i, j, k, c), got, want)


def test_chop_48_by_32(orc):
    b = orc.chop(Z3, (47, 47, 47), (32, 32, 32))
    assert len(b) == 8
    assert sorted({(int(r[0]), int(r[3])) for r in b}) == [(0, 31), (32, 47)]


@pytest.mark.parametrize("n,box", [(32, 32), (48, 32), (64, 32), (96, 32), (128, 32), (256, 64)])
def test_hierarchy_levels(orc, n, box):
    levels = orc.hierarchy(Z3, (n - 1,) * 3, orc.chop(Z3, (n - 1,) * 3, (box,) * 3))
    e, edges = n, [n]
    while e % 2 == 0 and e >= 4:
        e //= 2
        edges.append(e)
    assert [int(l[1][0]) + 1 for l in levels] == edges
    assert len(levels[-1][2]) == 1          # bottom is one box
    for (lo, hi, bx) in levels:            # boxes tile the level domain
        assert sum(int(np.prod(r[3:] - r[:3] + 1)) for r in bx) == int(np.prod(hi - lo + 1))


def test_hierarchy_independent_of_split(orc):
    dom = _dom((32, 32, 32))
    ref = [(tuple(l[0]), tuple(l[1])) for l in orc.hierarchy(*dom, orc.chop(*dom, (32, 32, 32)))]
    for mb in [(16, 16, 16), (8, 8, 8), (12, 20, 32), (6, 10, 14)]:
        got = [(tuple(l[0]), tuple(l[1])) for l in orc.hierarchy(*dom, orc.chop(*dom, mb))]
        assert got == ref


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0), (0, 1, 0), (1, 0, 1)])
def test_fill_closed_form_multibox(orc, periodic):
    dlo, dhi = (0, 0, 0), (11, 9, 7)
    boxes = orc.chop(dlo, dhi, (5, 4, 8))
    _check_fill(orc, dlo, dhi, periodic, boxes, ng=2, ncomp=2)


def test_fill_closed_form_negative_lo(orc):
    dlo, dhi = (-4, -6, 2), (3, 1, 7)
    boxes = orc.chop(dlo, dhi, (4, 3, 6))
    _check_fill(orc, dlo, dhi, (1, 0, 1), boxes, ng=1, ncomp=1)


def test_fill_single_box_self_images(orc):
    dlo, dhi = (0, 0, 0), (3, 3, 3)
    boxes = orc.chop(dlo, dhi, (4, 4, 4))
    _check_fill(orc, dlo, dhi, (1, 1, 1), boxes, ng=2, ncomp=1)
    _check_fill(orc, dlo, dhi, (0, 0, 0), boxes, ng=2, ncomp=1)
    # ghost width larger than the periodic domain: images wrap more than once
    dlo, dhi = (0, 0, 0), (1, 2, 1)
    _check_fill(orc, dlo, dhi, (1, 1, 1), orc.chop(dlo, dhi, (2, 3, 2)), ng=3, ncomp=1)


def _apply(orc, n, periodic, boxes, h, phi_dense):
    """A phi through the oracle: fill, then residual with rhs = 0 gives -A phi."""
    dlo, dhi = _dom(n)
    phi = orc.from_dense(phi_dense, boxes, dlo, 1)
    phi = orc.fill_boundary(dlo, dhi, periodic, boxes, phi, 1)
    rhs = orc.new_field(boxes, 0)
    r, _ = orc.residual(dlo, dhi, boxes, h, phi, 1, rhs, 0)
    return -orc.to_dense(r, boxes, dlo, dhi, 0)


@pytest.mark.parametrize("periodic,m", [((1, 1, 1), (1, 2, 3)), ((0, 0, 0), (1, 3, 2)),
                                        ((1, 0, 1), (2, 1, 1)), ((0, 0, 0), (16, 16, 16))])
def test_operator_eigenmodes(orc, periodic, m):
    n = (16, 16, 16)
    h = 1.0 / 16
    boxes = orc.chop(*_dom(n), (8, 4, 16))
    v = dense_ref.mode(n, m, periodic)
    lam = dense_ref.eigenvalue(n, m, periodic, h)
    Av = _apply(orc, n, periodic, boxes, h, v)
    scale = 12.0 / h ** 2
    assert np.abs(Av - lam * v).max() <= 1e-13 * max(abs(lam), 1.0) + 2e-15 * scale


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0), (0, 1, 1)])
def test_operator_vs_dense_matrix(orc, periodic):
    n, h = (8, 6, 4), 0.125
    A = dense_ref.assemble(n, periodic, h)
    v = inputs.rng(11).standard_normal((n[2], n[1], n[0]))
    boxes = orc.chop(*_dom(n), (4, 3, 4))
    Av = _apply(orc, n, periodic, boxes, h, v)
    ref = (A @ v.ravel()).reshape(v.shape)
    assert np.abs(Av - ref).max() <= 1e-14 * (12.0 / h ** 2) * np.abs(v).max()


@pytest.mark.parametrize("n", [(2, 2, 2), (3, 3, 3), (2, 3, 4), (4, 4, 4), (5, 2, 3)])
@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0), (1, 0, 1)])
def test_bottom_matrix_vs_numpy(orc, n, periodic):
    h = 0.37
    M = orc.bottom_matrix(n, periodic, h)
    A = dense_ref.assemble(n, periodic, h)
    ref = np.linalg.pinv(A, rcond=1e-10) if all(periodic) else np.linalg.inv(A)
    assert np.abs(M - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("periodic", [(0, 0, 0), (1, 1, 1), (1, 0, 0)])
def test_solve_matches_dense_direct_8(orc, periodic):
    n, h = (8, 8, 8), 0.125
    dlo, dhi = _dom(n)
    boxes = orc.chop(dlo, dhi, (4, 4, 4))
    rhs = inputs.rng(12).standard_normal((8, 8, 8))
    if all(periodic):
        rhs = inputs.remove_mean(rhs)
    phi, st, vc, hist = orc.solve(dlo, dhi, periodic, boxes, h, rhs, tol=1e-12)
    assert st == 0 and vc <= 30 and hist[-1] <= 1e-12
    A = dense_ref.assemble(n, periodic, h)
    if all(periodic):
        ref = (np.linalg.pinv(A, rcond=1e-10) @ rhs.ravel()).reshape(rhs.shape)
        phi = phi - phi.mean()
    else:
        ref = np.linalg.solve(A, rhs.ravel()).reshape(rhs.shape)
    assert np.abs(phi - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("periodic,m", [((1, 1, 1), (1, 2, 1)), ((0, 0, 0), (1, 1, 2)),
                                        ((0, 1, 0), (3, 1, 1))])
def test_solve_eigenmode(orc, periodic, m):
    n, h = (32, 32, 32), 1.0 / 32
    dlo, dhi = _dom(n)
    boxes = orc.chop(dlo, dhi, (16, 16, 16))
    v = dense_ref.mode(n, m, periodic)
    lam = dense_ref.eigenvalue(n, m, periodic, h)
    phi, st, vc, hist = orc.solve(dlo, dhi, periodic, boxes, h, lam * v)
    assert st == 0 and vc <= 30
    if all(periodic):
        phi = phi - phi.mean()
    assert np.abs(phi - v).max() <= 1e-10 * np.abs(v).max()


def _sine_error(orc, n):
    h = 1.0 / n
    dlo, dhi = _dom((n, n, n))
    boxes = orc.chop(dlo, dhi, (32, 32, 32))
    rhs = inputs.periodic_sine(n, noise=0.0)
    phi, st, vc, _ = orc.solve(dlo, dhi, (1, 1, 1), boxes, h, rhs, tol=1e-12)
    assert st == 0
    u = inputs.sine_mode((n, n, n), (1, 1, 1), True)
    return phi - phi.mean(), u, h


def test_periodic_sine_exact_discrete_solution(orc):
    # discrete solution is u * (pi h)^2 / sin^2(pi h): the 7-point eigenvalue of the m=1 mode
    phi, u, h = _sine_error(orc, 64)
    fac = (np.pi * h) ** 2 / np.sin(np.pi * h) ** 2
    assert abs(fac - 1.000803577679) < 1e-12
    assert np.abs(phi - fac * u).max() <= 1e-10


def test_second_order_convergence(orc):
    errs = []
    for n in (16, 32, 64):
        phi, u, _ = _sine_error(orc, n)
        errs.append(np.abs(phi - u).max() / np.abs(u).max())   # = (pi h)^2/sin^2(pi h) - 1
    for a, b in zip(errs, errs[1:]):
        assert abs(a / b / 4.0 - 1.0) < 0.01


def test_restriction_identities(orc):
    dlo, dhi = (0, 0, 0), (15, 7, 11)
    fine_boxes = orc.chop(dlo, dhi, (8, 4, 6))
    levels = orc.hierarchy(dlo, dhi, fine_boxes)
    F, C = levels[0], levels[1]
    # constants restrict exactly
    f = orc.new_field(F[2], 1)
    for a in f:
        a[...] = 3.25
    c = orc.restrict(F, f, 1, C, 0)
    for a in c:
        assert np.all(a == 3.25)
    # a linear function of the cell centre restricts to its coarse-centre value
    n = (16, 8, 12)
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    lin = (2 * i + 1) + 3 * (2 * j + 1) - 5 * (2 * k + 1)          # 2 * centre / h
    cn = (8, 4, 6)
    K, J, I = np.meshgrid(np.arange(cn[2]), np.arange(cn[1]), np.arange(cn[0]), indexing="ij")
    clin = 2 * (2 * I + 1) + 6 * (2 * J + 1) - 10 * (2 * K + 1)      # same function at coarse centres
    c = orc.restrict(F, orc.from_dense(lin.astype(float), F[2], dlo, 1), 1, C, 0)
    assert np.array_equal(orc.to_dense(c, C[2], C[0], C[1], 0), clin.astype(float))


def test_restriction_prolongation_adjoint(orc):
    dlo, dhi = (0, 0, 0), (11, 7, 15)
    levels = orc.hierarchy(dlo, dhi, orc.chop(dlo, dhi, (4, 8, 8)))
    F, C = levels[0], levels[1]
    g = inputs.rng(13)
    fd = g.integers(-50, 50, size=(16, 8, 12)).astype(float)
    cd = g.integers(-50, 50, size=(8, 4, 6)).astype(float)
    Rf = orc.to_dense(orc.restrict(F, orc.from_dense(fd, F[2], dlo, 0), 0, C, 0), C[2], C[0], C[1], 0)
    zero = orc.from_dense(np.zeros_like(fd), F[2], dlo, 0)
    Pg = orc.to_dense(orc.prolong_add(C, orc.from_dense(cd, C[2], C[0], 0), 0, F, zero, 0),
                      F[2], dlo, dhi, 0)
    assert 8.0 * np.sum(Rf * cd) == np.sum(fd * Pg)
    # piecewise-constant injection: every fine cell carries its parent's value
    assert np.array_equal(Pg, np.repeat(np.repeat(np.repeat(cd, 2, 0), 2, 1), 2, 2))


def test_trilinear_prolongation_reproduces_linear_and_constant(orc):
    """P6 for the trilinear option: coarse samples of a linear function interpolate to the
    function's values at the fine centres wherever the coarse stencil stays inside the domain
    (dyadic data: exact), and a constant on a periodic domain stays that constant everywhere
    (the ghosts are periodic images)."""
    dlo, dhi = (0, 0, 0), (15, 11, 7)
    levels = orc.hierarchy(dlo, dhi, orc.chop(dlo, dhi, (8, 4, 4)))
    F, C = levels[0], levels[1]
    cn = (8, 6, 4)
    K, J, I = np.meshgrid(np.arange(cn[2]), np.arange(cn[1]), np.arange(cn[0]), indexing="ij")
    f = lambda x, y, z: 1.0 + 2.0 * x - 4.0 * y + 8.0 * z        # coarse cell units
    coarse = orc.from_dense(f(I + 0.5, J + 0.5, K + 0.5), C[2], C[0], 1)
    coarse = orc.fill_boundary(C[0], C[1], (0, 0, 0), C[2], coarse, 1)
    fn = (16, 12, 8)
    k, j, i = np.meshgrid(np.arange(fn[2]), np.arange(fn[1]), np.arange(fn[0]), indexing="ij")
    base = orc.from_dense(np.full(fn[::-1], 0.5), F[2], dlo, 1)
    out = orc.to_dense(orc.prolong_add(C, coarse, 1, F, base, 1, trilinear=True), F[2], dlo, dhi, 1)
    want = 0.5 + f((i + 0.5) / 2, (j + 0.5) / 2, (k + 0.5) / 2)
    inner = (i >= 1) & (i <= fn[0] - 2) & (j >= 1) & (j <= fn[1] - 2) & (k >= 1) & (k <= fn[2] - 2)
    assert np.array_equal(out[inner], want[inner])
    assert not np.array_equal(out, want)             # the Dirichlet ghosts bend it at the faces
    # a constant through periodic ghosts, every cell
    coarse = orc.fill_boundary(C[0], C[1], (1, 1, 1), C[2],
                               orc.from_dense(np.full(cn[::-1], 3.0), C[2], C[0], 1), 1)
    zero = orc.from_dense(np.zeros(fn[::-1]), F[2], dlo, 1)
    out = orc.to_dense(orc.prolong_add(C, coarse, 1, F, zero, 1, trilinear=True), F[2], dlo, dhi, 1)
    assert np.all(out == 3.0)


def test_trilinear_vcycle_converges_to_the_same_solution(orc):
    """With trilinear prolongation the V-cycle solves the same discrete problem: every cycle
    reduces the residual (by at least 4x here; with the 8-cell-average restriction it is not
    faster than injection), and the result differs from the injection solve's by no more than
    the a-priori bound ||A^-1|| ||r|| of both (P7)."""
    n = 32
    dlo, dhi = _dom((n, n, n))
    boxes = orc.chop(dlo, dhi, (16, 16, 16))
    rhs = inputs.dirichlet_jacobi(n, seed=2)
    a, st_a, vc_a, _ = orc.solve(dlo, dhi, (0, 0, 0), boxes, 1.0 / n, rhs)
    b, st_b, vc_b, hb = orc.solve(dlo, dhi, (0, 0, 0), boxes, 1.0 / n, rhs, trilinear=True)
    assert st_a == st_b == 0 and hb[-1] <= 1e-10 < hb[-2]
    assert np.all(hb[1:] <= 0.25 * hb[:-1])
    assert np.abs(a - b).max() <= 2 * 0.06 * 1e-10 * np.abs(rhs).max()


@pytest.mark.parametrize("color", [0, 1])
def test_rbgs_zeroes_coloured_residuals(orc, color):
    n, h = (8, 8, 8), 0.125
    dlo, dhi = _dom(n)
    periodic = (0, 1, 0)
    boxes = orc.chop(dlo, dhi, (4, 8, 4))
    g = inputs.rng(14)
    phi = orc.from_dense(g.standard_normal((8, 8, 8)), boxes, dlo, 1)
    rhs = orc.from_dense(g.standard_normal((8, 8, 8)), boxes, dlo, 0)
    phi = orc.fill_boundary(dlo, dhi, periodic, boxes, phi, 1)
    before = orc.to_dense(phi, boxes, dlo, dhi, 1)
    phi = orc.rbgs(dlo, dhi, boxes, h, phi, 1, rhs, 0, color)
    after = orc.to_dense(phi, boxes, dlo, dhi, 1)
    phi = orc.fill_boundary(dlo, dhi, periodic, boxes, phi, 1)
    r, _ = orc.residual(dlo, dhi, boxes, h, phi, 1, rhs, 0)
    r = orc.to_dense(r, boxes, dlo, dhi, 0)
    k, j, i = np.meshgrid(*(np.arange(8),) * 3, indexing="ij")
    col = (i + j + k) % 2 == color
    assert np.array_equal(after[~col], before[~col])         # other colour untouched
    # a coloured cell solves its own equation exactly, except next to a Dirichlet face (x, z
    # here) where its ghost still holds -phi from before the update (ghosts are refilled
    # only before each colour)
    inner = col & (i > 0) & (i < 7) & (k > 0) & (k < 7)
    assert np.abs(r[inner]).max() <= 1e-13 * 12 / h ** 2 * np.abs(after).max()
    assert np.abs(r[col & ~inner]).max() > 1e-3
    assert np.abs(r[~col]).max() > 1e-3                      # only one colour solved


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0)])
def test_decomposition_invariance_bitwise(orc, periodic):
    n, h = (32, 32, 32), 1.0 / 32
    dlo, dhi = _dom(n)
    rhs = inputs.rng(15).standard_normal((32, 32, 32))
    if all(periodic):
        rhs = inputs.remove_mean(rhs)
    ref = None
    for mb in [(32, 32, 32), (16, 16, 16), (8, 8, 8), (12, 20, 32), (6, 10, 14)]:
        boxes = orc.chop(dlo, dhi, mb)
        phi, st, vc, hist = orc.solve(dlo, dhi, periodic, boxes, h, rhs, fixed_vcycles=3)
        assert vc == 3
        if ref is None:
            ref = (phi, hist)
        else:
            assert np.array_equal(phi, ref[0]) and np.array_equal(hist, ref[1])


def test_vcycle_convergence_rate(orc):
    n = 64
    dlo, dhi = _dom((n, n, n))
    boxes = orc.chop(dlo, dhi, (32, 32, 32))
    rhs = inputs.dirichlet_jacobi(n, seed=2)
    phi, st, vc, hist = orc.solve(dlo, dhi, (0, 0, 0), boxes, 1.0 / n, rhs)
    assert st == 0 and vc <= 12
    rates = hist[1:] / hist[:-1]
    assert rates.max() < 0.15


def test_zero_rhs_gives_zero(orc):
    dlo, dhi = _dom((8, 8, 8))
    boxes = orc.chop(dlo, dhi, (4, 4, 4))
    phi, st, vc, _ = orc.solve(dlo, dhi, (1, 1, 1), boxes, 0.125, np.zeros((8, 8, 8)),
                               phi0=np.ones((8, 8, 8)))
    assert st == 0 and vc == 0 and not phi.any()


def test_nan_rhs_reported(orc):
    dlo, dhi = _dom((8, 8, 8))
    boxes = orc.chop(dlo, dhi, (4, 4, 4))
    rhs = np.ones((8, 8, 8))
    rhs[3, 2, 1] = np.nan
    _, st, _, _ = orc.solve(dlo, dhi, (0, 0, 0), boxes, 0.125, rhs)
    assert st == orc.ENAN


def test_mixed_precision_within_error_bound(orc):
    # ||phi - phi*||_inf <= ||A^-1||_inf ||r||_inf; for the Dirichlet unit cube ||A^-1||_inf
    # is bounded by max of the solution of lap w = -1 (about 0.056), so two solves that both
    # meet tol differ by at most 2 * 0.06 * tol * ||rhs||_inf.
    n = 32
    dlo, dhi = _dom((n, n, n))
    boxes = orc.chop(dlo, dhi, (16, 16, 16))
    rhs = inputs.dirichlet_jacobi(n, seed=2)
    tol = 1e-10
    p64, s1, v1, h1 = orc.solve(dlo, dhi, (0, 0, 0), boxes, 1.0 / n, rhs, tol=tol)
    p32, s2, v2, h2 = orc.solve(dlo, dhi, (0, 0, 0), boxes, 1.0 / n, rhs, tol=tol, mixed=True)
    assert s1 == 0 and s2 == 0 and h2[-1] <= tol
    A = dense_ref.assemble((n, n, n), (0, 0, 0), 1.0 / n) if n <= 16 else None
    assert np.abs(p64 - p32).max() <= 2 * 0.06 * tol * np.abs(rhs).max()
    assert v2 <= v1 + 2
    del A


# ---- the V-cycle schedule against a dense composition of per-level operators ------------
#
# tests/dense_ref.DenseVCycle states the cycle (sweep counts, colour order, fresh neighbour
# values before every colour, residual restriction, zero coarse guess, exact bottom,
# injection) as products of dense matrices, independently of the oracle's box loops.  One
# and two oracle cycles from a random phi_0 must equal it to rounding: a swapped colour
# order, a wrong sweep count, a missing fill between colours on a multi-box level, a
# transfer operator off by a factor, or a skipped coarse correction all move the iterate
# by O(1) (the mutation test below checks that the pin sees such slips).

VC_CASES = [((8, 8, 8), (4, 4, 4)), ((8, 4, 6), (4, 4, 3))]
VC_FACES = [(0, 0, 0), (1, 1, 1), (1, 0, 1)]
VC_NU = [(2, 2), (1, 1), (0, 2)]


def _vc_problem(n, periodic, seed=21):
    g = inputs.rng(seed)
    shape = (n[2], n[1], n[0])
    rhs = g.standard_normal(shape)
    if all(periodic):
        rhs = inputs.remove_mean(rhs)
    return rhs, g.standard_normal(shape)


@pytest.mark.parametrize("n,mb", VC_CASES)
@pytest.mark.parametrize("periodic", VC_FACES)
@pytest.mark.parametrize("nu", VC_NU)
def test_vcycle_schedule_matches_dense_composition(orc, n, mb, periodic, nu):
    h = 1.0 / n[0]
    dlo, dhi = _dom(n)
    boxes = orc.chop(dlo, dhi, mb)
    rhs, phi0 = _vc_problem(n, periodic)
    ref = dense_ref.DenseVCycle(n, periodic, h, *nu)
    for k in (1, 2):
        phi, st, vc, _ = orc.solve(dlo, dhi, periodic, boxes, h, rhs, phi0=phi0,
                                   fixed_vcycles=k, nu1=nu[0], nu2=nu[1])
        d = ref.run(phi0, rhs, k)
        assert st == 0 and vc == k
        assert np.abs(phi - d).max() <= 1e-13 * np.abs(d).max()


@pytest.mark.parametrize("n,mb", VC_CASES)
@pytest.mark.parametrize("periodic", VC_FACES)
@pytest.mark.parametrize("inner", [1, 2, 3])
def test_mixed_outer_iteration_matches_dense_composition(orc, n, mb, periodic, inner):
    """The mixed form's outer iteration phi <- phi + e, e = m inner cycles on A e = r from
    e = 0 (r = rhs - A phi scaled by an exact power of two, e scaled back), equals m FP64
    dense cycles from phi -- a V-cycle is the affine map phi + B (rhs - A phi), so its m-fold
    application from 0 on the residual equation adds exactly what m cycles from phi add --
    up to the inner cycles' binary32 rounding: each inner value carries a few units of 2^-24
    relative to the correction, so the bound is 2^-20 of the largest correction."""
    h = 1.0 / n[0]
    dlo, dhi = _dom(n)
    boxes = orc.chop(dlo, dhi, mb)
    rhs, phi0 = _vc_problem(n, periodic)
    ref = dense_ref.DenseVCycle(n, periodic, h)
    for k in (1, 2):
        phi, st, vc, _ = orc.solve(dlo, dhi, periodic, boxes, h, rhs, phi0=phi0, fixed_vcycles=k,
                                   mixed=True, inner_cycles=inner)
        d = ref.run(phi0, rhs, k * inner)
        assert st == 0 and vc == k
        assert np.abs(phi - d).max() <= 2.0 ** -20 * np.abs(d - phi0).max()


class _Mutant(dense_ref.DenseVCycle):
    """DenseVCycle with one planted schedule slip."""

    def __init__(self, slip, *a, **kw):
        super().__init__(*a, **kw)
        self.slip = slip

    def sweeps(self, l, phi, rhs, count):
        if self.slip == "black_first":
            for _ in range(count):
                phi = self.half_sweep(l, phi, rhs, 1)
                phi = self.half_sweep(l, phi, rhs, 0)
            return phi
        if self.slip == "one_sweep_less" and count > 0:
            count -= 1
        return super().sweeps(l, phi, rhs, count)

    def cycle(self, l, phi, rhs):
        if self.slip == "sum_restriction" and l < len(self.ext) - 1:
            phi = self.sweeps(l, phi, rhs, self.nu1)
            rc = 8.0 * (self.R[l] @ (rhs - self.A[l] @ phi))
            ec = self.cycle(l + 1, np.zeros_like(rc), rc)
            return self.sweeps(l, phi + 8.0 * (self.R[l].T @ ec), rhs, self.nu2)
        if self.slip == "no_coarse_correction" and l < len(self.ext) - 1:
            return self.sweeps(l, self.sweeps(l, phi, rhs, self.nu1), rhs, self.nu2)
        return super().cycle(l, phi, rhs)


@pytest.mark.parametrize("slip", ["black_first", "one_sweep_less", "sum_restriction",
                                  "no_coarse_correction"])
def test_vcycle_pin_detects_schedule_slips(orc, slip):
    n, mb, periodic = (8, 8, 8), (4, 4, 4), (0, 0, 0)
    h = 1.0 / n[0]
    dlo, dhi = _dom(n)
    rhs, phi0 = _vc_problem(n, periodic)
    phi, _, _, _ = orc.solve(dlo, dhi, periodic, orc.chop(dlo, dhi, mb), h, rhs, phi0=phi0,
                             fixed_vcycles=1)
    bad = _Mutant(slip, n, periodic, h).run(phi0, rhs, 1)
    assert np.abs(phi - bad).max() > 1e-3 * np.abs(phi).max()
