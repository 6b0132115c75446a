"""GPU parity: every kernel of the path, called through the C ABI, against the CPU oracle on
the same seeded inputs; then whole solves.  Ghost fill and box bookkeeping are compared
bit for bit; the FP64 stencil kernels are written so that each operation is one IEEE
rounding in the oracle's order, so they are compared bit for bit as well; whole solves
differ from the oracle only through the independently computed bottom matrix and are held
to 1e-12 relative."""
import numpy as np
import pytest
import torch

from paper_2403_12179_gb300 import inputs, mg
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

Z3 = (0, 0, 0)


@pytest.fixture(scope="module")
def gctx():
    import paper_2403_12179_gb300.build as b
    b.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()
    ctx = mg.mg_init(0)
    yield ctx
    mg.mg_finalize(ctx)


def _ba(ctx, dom, mb):
    ba = mg.mg_box_array_create(ctx, Z3, dom, mb)
    return ba, mg.mg_box_array_info(ctx, ba)[1]


FILL_CASES = [((11, 9, 7), (5, 4, 8), 2, 2), ((31, 31, 31), (16, 16, 16), 2, 4),
              ((15, 15, 15), (8, 8, 8), 1, 1), ((3, 3, 3), (4, 4, 4), 2, 1),
              ((23, 15, 7), (8, 8, 8), 1, 3)]


@pytest.mark.parametrize("dom,mb,ng,ncomp", FILL_CASES)
@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0), (1, 0, 1)])
@pytest.mark.parametrize("dt", [mg.MG_F64, mg.MG_F32])
def test_fill_boundary_bitwise(gctx, orc, dom, mb, ng, ncomp, periodic, dt):
    ba, boxes = _ba(gctx, dom, mb)
    npdt = np.float64 if dt == mg.MG_F64 else np.float32
    g = inputs.rng(31)
    fabs = [g.standard_normal(f.shape).astype(npdt) for f in orc.new_field(boxes, ng, ncomp)]
    ref = orc.fill_boundary(Z3, dom, periodic, boxes, fabs, ng)
    fab = gu.to_fab(gctx, ba, fabs, ng, dt)
    mg.mg_fill_boundary(gctx, fab, mg.make_bc(periodic))
    got = gu.from_fab(gctx, fab, len(boxes))
    for a, r in zip(got, ref):
        assert np.array_equal(a, r)
    mg.mg_fab_free(gctx, fab)


def test_fill_boundary_unfused_equals_fused(gctx, orc):
    dom, mb = (23, 15, 7), (8, 8, 8)
    ba, boxes = _ba(gctx, dom, mb)
    g = inputs.rng(30)
    fabs = [g.standard_normal(f.shape) for f in orc.new_field(boxes, 2, 3)]
    for periodic in [(1, 1, 1), (0, 1, 0)]:
        bc = mg.make_bc(periodic)
        a, b = gu.to_fab(gctx, ba, fabs, 2), gu.to_fab(gctx, ba, fabs, 2)
        mg.mg_fill_boundary(gctx, a, bc)
        mg.mg_fill_boundary_unfused(gctx, b, bc)
        for x, y in zip(gu.from_fab(gctx, a, len(boxes)), gu.from_fab(gctx, b, len(boxes))):
            assert np.array_equal(x, y)
        mg.mg_fab_free(gctx, a)
        mg.mg_fab_free(gctx, b)


def _level_inputs(orc, boxes, dom, periodic, ng_phi, ng_rhs, seed, dt=np.float64):
    g = inputs.rng(seed)
    phi = [g.standard_normal(f.shape).astype(dt) for f in orc.new_field(boxes, ng_phi)]
    rhs = [g.standard_normal(f.shape).astype(dt) for f in orc.new_field(boxes, ng_rhs)]
    phi = orc.fill_boundary(Z3, dom, periodic, boxes, phi, ng_phi)
    return phi, rhs


@pytest.mark.parametrize("color", [0, 1])
@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0), (0, 1, 0)])
@pytest.mark.parametrize("dt", [mg.MG_F64, mg.MG_F32])
def test_rbgs_half_sweep_bitwise(gctx, orc, color, periodic, dt):
    dom, mb, h = (19, 15, 11), (8, 8, 6), 1.0 / 20
    npdt = np.float64 if dt == mg.MG_F64 else np.float32
    ba, boxes = _ba(gctx, dom, mb)
    phi, rhs = _level_inputs(orc, boxes, dom, periodic, 1, 0, 32, npdt)
    ref = orc.rbgs(Z3, dom, boxes, h, phi, 1, rhs, 0, color)
    fp, fr = gu.to_fab(gctx, ba, phi, 1, dt), gu.to_fab(gctx, ba, rhs, 0, dt)
    mg.mg_smooth(gctx, fp, fr, mg.make_bc(periodic), h, color)
    got = gu.from_fab(gctx, fp, len(boxes))
    for a, r in zip(got, ref):
        assert np.array_equal(gu.valid(a, 1), gu.valid(r, 1))


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 1)])
def test_full_sweep_matches_fill_red_fill_black(gctx, orc, periodic):
    dom, mb, h = (15, 15, 15), (8, 8, 8), 1.0 / 16
    ba, boxes = _ba(gctx, dom, mb)
    phi, rhs = _level_inputs(orc, boxes, dom, periodic, 2, 1, 33)
    ref = phi
    for color in (0, 1):
        ref = orc.fill_boundary(Z3, dom, periodic, boxes, ref, 2)
        ref = orc.rbgs(Z3, dom, boxes, h, ref, 2, rhs, 1, color)
    fp, fr = gu.to_fab(gctx, ba, phi, 2), gu.to_fab(gctx, ba, rhs, 1)
    mg.mg_smooth(gctx, fp, fr, mg.make_bc(periodic), h, 2)
    got = gu.from_fab(gctx, fp, len(boxes))
    for a, r in zip(got, ref):
        assert np.array_equal(gu.valid(a, 2), gu.valid(r, 2))


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0)])
def test_residual_and_norm_bitwise(gctx, orc, periodic):
    dom, mb, h = (23, 15, 31), (8, 16, 12), 1.0 / 24
    ba, boxes = _ba(gctx, dom, mb)
    phi, rhs = _level_inputs(orc, boxes, dom, periodic, 1, 0, 34)
    r_ref, n_ref = orc.residual(Z3, dom, boxes, h, phi, 1, rhs, 0)
    fp, fr = gu.to_fab(gctx, ba, phi, 1), gu.to_fab(gctx, ba, rhs, 0)
    fo = mg.mg_fab_alloc(gctx, ba, 1, 0)
    nrm = mg.mg_residual(gctx, fp, fr, fo, h)
    got = gu.from_fab(gctx, fo, len(boxes))
    for a, r in zip(got, r_ref):
        assert np.array_equal(a, r)
    assert nrm == n_ref


@pytest.mark.parametrize("dom,mb", [((31, 31, 31), (16, 16, 16)), ((15, 15, 15), (4, 4, 4)),
                                    ((47, 23, 15), (32, 16, 8))])
def test_residual_restrict_bitwise(gctx, orc, dom, mb):
    h = 1.0 / (dom[0] + 1)
    periodic = (1, 0, 1)
    ba, boxes = _ba(gctx, dom, mb)
    levels = orc.hierarchy(Z3, dom, boxes)
    cba = mg.mg_hierarchy_level(gctx, ba, 1)
    cboxes = mg.mg_box_array_info(gctx, cba)[1]
    assert np.array_equal(np.array(cboxes), levels[1][2])
    phi, rhs = _level_inputs(orc, boxes, dom, periodic, 1, 0, 35)
    r, _ = orc.residual(Z3, dom, boxes, h, phi, 1, rhs, 0)
    c_ref = orc.restrict(levels[0], r, 0, levels[1], 0)
    fp, fr = gu.to_fab(gctx, ba, phi, 1), gu.to_fab(gctx, ba, rhs, 0)
    crhs = mg.mg_fab_alloc(gctx, cba, 1, 0)
    cphi = mg.mg_fab_alloc(gctx, cba, 1, 1)
    mg.mg_fab_set_val(gctx, cphi, 7.0)
    mg.mg_residual_restrict(gctx, fp, fr, crhs, cphi, h)
    got = gu.from_fab(gctx, crhs, len(cboxes))
    for a, c in zip(got, c_ref):
        assert np.array_equal(a, c)
    for a in gu.from_fab(gctx, cphi, len(cboxes)):
        assert not gu.valid(a, 1).any()


def test_restrict_and_prolong_bitwise(gctx, orc):
    dom, mb = (31, 15, 23), (8, 8, 8)
    ba, boxes = _ba(gctx, dom, mb)
    levels = orc.hierarchy(Z3, dom, boxes)
    cba = mg.mg_hierarchy_level(gctx, ba, 1)
    cboxes = mg.mg_box_array_info(gctx, cba)[1]
    g = inputs.rng(36)
    fine = [g.standard_normal(f.shape) for f in orc.new_field(boxes, 1)]
    coarse = [g.standard_normal(f.shape) for f in orc.new_field(cboxes, 1)]
    ff, fc = gu.to_fab(gctx, ba, fine, 1), gu.to_fab(gctx, cba, coarse, 1)
    mg.mg_restrict(gctx, ff, fc)
    c_ref = orc.restrict(levels[0], fine, 1, levels[1], 1)
    for a, c in zip(gu.from_fab(gctx, fc, len(cboxes)), c_ref):
        assert np.array_equal(gu.valid(a, 1), gu.valid(c, 1))
    fc2 = gu.to_fab(gctx, cba, coarse, 1)
    mg.mg_prolong_add(gctx, fc2, ff)
    p_ref = orc.prolong_add(levels[1], coarse, 1, levels[0], fine, 1)
    for a, p in zip(gu.from_fab(gctx, ff, len(boxes)), p_ref):
        assert np.array_equal(gu.valid(a, 1), gu.valid(p, 1))


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0), (1, 0, 1)])
def test_trilinear_prolong_bitwise(gctx, orc, periodic):
    """The trilinear prolongation entry point, on coarse ghosts filled by mg_fill_boundary,
    equals the oracle's (fill, then trilinear prolongation) bit for bit."""
    dom, mb = (31, 15, 23), (8, 8, 8)
    ba, boxes = _ba(gctx, dom, mb)
    levels = orc.hierarchy(Z3, dom, boxes)
    cba = mg.mg_hierarchy_level(gctx, ba, 1)
    cboxes = mg.mg_box_array_info(gctx, cba)[1]
    g = inputs.rng(37)
    fine = [g.standard_normal(f.shape) for f in orc.new_field(boxes, 1)]
    coarse = [g.standard_normal(f.shape) for f in orc.new_field(cboxes, 1)]
    ff, fc = gu.to_fab(gctx, ba, fine, 1), gu.to_fab(gctx, cba, coarse, 1)
    mg.mg_fill_boundary(gctx, fc, mg.make_bc(periodic))
    mg.mg_prolong_add_trilinear(gctx, fc, ff)
    cref = orc.fill_boundary(levels[1][0], levels[1][1], periodic, cboxes, coarse, 1)
    p_ref = orc.prolong_add(levels[1], cref, 1, levels[0], fine, 1, trilinear=True)
    for a, p in zip(gu.from_fab(gctx, ff, len(boxes)), p_ref):
        assert np.array_equal(gu.valid(a, 1), gu.valid(p, 1))
    with pytest.raises(mg.MgError):   # no coarse ghosts to read
        mg.mg_prolong_add_trilinear(gctx, gu.to_fab(gctx, cba, [c[:, 1:-1, 1:-1, 1:-1] for c in coarse], 0), ff)


@pytest.mark.parametrize("periodic,mb", [((1, 1, 1), (16, 16, 16)), ((0, 0, 0), (16, 8, 32)),
                                         ((0, 1, 0), (8, 16, 16))])
def test_trilinear_solve_matches_oracle(gctx, orc, periodic, mb):
    """Solves with the trilinear prolongation: FP64 iterates and the converged result equal
    the oracle's to the bottom-matrix rounding (1e-12), with the same V-cycle count; the mixed
    form reaches the tolerance within the a-priori bound of the oracle's mixed result."""
    n = 32
    rhs = inputs.rng(44).standard_normal((n, n, n))
    if all(periodic):
        rhs = inputs.remove_mean(rhs)
    dom = (n - 1,) * 3
    oboxes = orc.chop(Z3, dom, mb)
    tri = mg.MG_PROLONG_TRILINEAR
    for k in (1, 2):
        phi, res = _solve_pair(gctx, orc, n, mb, periodic, rhs, fixed=k, prolong=tri)
        o_phi, _, vc, _ = orc.solve(Z3, dom, periodic, oboxes, 1.0 / n, rhs, fixed_vcycles=k,
                                    trilinear=True)
        assert res.vcycles == k == vc
        assert np.abs(phi - o_phi).max() <= 1e-12 * np.abs(o_phi).max()
    phi, res = _solve_pair(gctx, orc, n, mb, periodic, rhs, prolong=tri)
    o_phi, st, vc, _ = orc.solve(Z3, dom, periodic, oboxes, 1.0 / n, rhs, trilinear=True)
    assert res.status == mg.MG_OK and st == 0 and res.vcycles == vc and res.rel_resid <= 1e-10
    assert np.abs(phi - o_phi).max() <= 1e-12 * np.abs(o_phi).max()
    pmx, rmx = _solve_pair(gctx, orc, n, mb, periodic, rhs, prolong=tri, precision=mg.MG_PREC_MIXED)
    o_mx, st, vc, _ = orc.solve(Z3, dom, periodic, oboxes, 1.0 / n, rhs, trilinear=True, mixed=True)
    assert rmx.status == mg.MG_OK and rmx.rel_resid <= 1e-10 and abs(rmx.vcycles - vc) <= 1
    d = pmx - o_mx
    if all(periodic):
        d -= d.mean()
    assert np.abs(d).max() <= 2 * 0.06 * 1e-10 * np.abs(rhs).max() * (10 if all(periodic) else 1)


@pytest.mark.parametrize("n,mb", [((2, 2, 2), (2, 2, 2)), ((3, 3, 3), (3, 3, 3)),
                                  ((4, 6, 2), (2, 3, 2)), ((8, 8, 8), (4, 8, 8))])
@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0), (0, 1, 0)])
def test_bottom_solve(gctx, orc, n, mb, periodic):
    dom = tuple(v - 1 for v in n)
    h = 0.25
    ba, boxes = _ba(gctx, dom, mb)
    g = inputs.rng(37)
    rhs = g.standard_normal((n[2], n[1], n[0]))
    M = orc.bottom_matrix(n, periodic, h)
    ref = (M @ rhs.ravel()).reshape(rhs.shape)
    fr = gu.dense_fab(gctx, ba, rhs, 0)
    fp = mg.mg_fab_alloc(gctx, ba, 1, 1)
    mg.mg_bottom_solve(gctx, fr, fp, mg.make_bc(periodic), h)
    got = gu.fab_dense(gctx, fp, rhs.shape)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_dense_roundtrip_and_set_val(gctx):
    dom = (20, 13, 9)
    ba, boxes = _ba(gctx, dom, (8, 8, 8))
    x = inputs.rng(38).standard_normal((3, 10, 14, 21))
    fab = mg.mg_fab_alloc(gctx, ba, 3, 2)
    t = torch.from_numpy(x).pin_memory()
    mg.mg_fab_copy_from_dense(gctx, fab, t.data_ptr(), True)
    out = torch.empty_like(t).pin_memory()
    mg.mg_fab_copy_to_dense(gctx, fab, out.data_ptr(), True)
    torch.cuda.synchronize()
    assert np.array_equal(out.numpy(), x)
    mg.mg_fab_set_val(gctx, fab, 2.5, include_ghosts=False)
    for a in gu.from_fab(gctx, fab, len(boxes)):
        assert np.all(gu.valid(a, 2) == 2.5)
        assert np.all(a[:, 0] == 0.0)


# ---- whole solves ----------------------------------------------------------------------

def _solve_pair(gctx, orc, n, mb, periodic, rhs, tol=1e-10, fixed=-1, precision=mg.MG_PREC_F64,
                use_graph=1, ng=(1, 0), prolong=mg.MG_PROLONG_CONSTANT):
    dom = (n - 1,) * 3
    h = 1.0 / n
    ba, boxes = _ba(gctx, dom, mb)
    fr = gu.dense_fab(gctx, ba, rhs, ng[1])
    fp = mg.mg_fab_alloc(gctx, ba, 1, ng[0])
    opt = mg.make_options(fixed_vcycles=fixed, precision=precision, use_graph=use_graph,
                          prolong=prolong)
    res = mg.mg_solve(gctx, fr, fp, mg.make_bc(periodic), tol, opt)
    phi = gu.fab_dense(gctx, fp, rhs.shape)
    mg.mg_fab_free(gctx, fr)
    mg.mg_fab_free(gctx, fp)
    return phi, res


def test_periodic_sine_64_matches_oracle(gctx, orc):
    n = 64
    rhs = inputs.periodic_sine(n, seed=1)
    phi, res = _solve_pair(gctx, orc, n, (32, 32, 32), (1, 1, 1), rhs)
    o_phi, st, vc, hist = orc.solve(Z3, (63,) * 3, (1, 1, 1), orc.chop(Z3, (63,) * 3, (32,) * 3),
                                    1.0 / n, rhs)
    assert res.status == mg.MG_OK and st == 0
    assert res.vcycles == vc
    assert res.rel_resid <= 1e-10 and abs(res.rel_resid - hist[-1]) <= 1e-3 * hist[-1]
    assert np.abs(phi - o_phi).max() <= 1e-12 * np.abs(o_phi).max()


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0)])
def test_iterates_match_oracle(gctx, orc, k, periodic):
    n = 32
    rhs = inputs.rng(40).standard_normal((n, n, n))
    if all(periodic):
        rhs = inputs.remove_mean(rhs)
    phi, res = _solve_pair(gctx, orc, n, (16, 16, 16), periodic, rhs, fixed=k)
    o_phi, _, vc, hist = orc.solve(Z3, (n - 1,) * 3, periodic, orc.chop(Z3, (n - 1,) * 3, (16,) * 3),
                                   1.0 / n, rhs, fixed_vcycles=k)
    assert res.vcycles == k == vc
    assert np.abs(phi - o_phi).max() <= 1e-12 * np.abs(o_phi).max()


def test_decomposition_invariance_bitwise(gctx, orc):
    n = 32
    rhs = inputs.rng(41).standard_normal((n, n, n))
    ref = None
    for mb in [(32, 32, 32), (16, 16, 16), (8, 8, 8), (16, 8, 32)]:
        phi, res = _solve_pair(gctx, orc, n, mb, (0, 0, 0), rhs, fixed=3)
        if ref is None:
            ref = phi
        assert np.array_equal(phi, ref)


def test_graph_replay_matches_eager(gctx, orc):
    n = 32
    rhs = inputs.rng(42).standard_normal((n, n, n))
    a, ra = _solve_pair(gctx, orc, n, (16, 16, 16), (0, 1, 0), rhs, use_graph=1)
    b, rb = _solve_pair(gctx, orc, n, (16, 16, 16), (0, 1, 0), rhs, use_graph=0)
    assert ra.vcycles == rb.vcycles and np.array_equal(a, b)


def test_edge_cases(gctx, orc):
    # zero rhs gives phi = 0 in zero V-cycles
    phi, res = _solve_pair(gctx, orc, 8, (4, 4, 4), (1, 1, 1), np.zeros((8, 8, 8)))
    assert res.status == mg.MG_OK and res.vcycles == 0 and not phi.any()
    # NaN in rhs is reported
    rhs = np.ones((8, 8, 8))
    rhs[1, 2, 3] = np.nan
    _, res = _solve_pair(gctx, orc, 8, (4, 4, 4), (0, 0, 0), rhs)
    assert res.status == mg.MG_ENAN
    # domain that is its own bottom level: exact in one cycle
    rhs = inputs.rng(43).standard_normal((2, 2, 2))
    phi, res = _solve_pair(gctx, orc, 2, (2, 2, 2), (0, 0, 0), rhs)
    o_phi, _, vc, _ = orc.solve(Z3, (1, 1, 1), (0, 0, 0), orc.chop(Z3, (1, 1, 1), (2, 2, 2)), 0.5, rhs)
    assert res.status == mg.MG_OK and res.vcycles == vc == 1
    assert np.abs(phi - o_phi).max() <= 1e-13 * np.abs(o_phi).max()
    # max_iter reached
    rhs = inputs.rng(44).standard_normal((16, 16, 16))
    dom = (15, 15, 15)
    ba, _ = _ba(gctx, dom, (8, 8, 8))
    fr, fp = gu.dense_fab(gctx, ba, rhs, 0), mg.mg_fab_alloc(gctx, ba, 1, 1)
    res = mg.mg_solve(gctx, fr, fp, mg.make_bc((0, 0, 0)), 1e-10, mg.make_options(max_iter=2))
    assert res.status == mg.MG_NOT_CONVERGED and res.vcycles == 2


def test_mixed_precision_solve(gctx, orc):
    n = 64
    rhs = inputs.gaussian_blobs(n, seed=5)
    tol = 1e-10
    p64, r64 = _solve_pair(gctx, orc, n, (32, 32, 32), (0, 0, 0), rhs, tol=tol)
    pmx, rmx = _solve_pair(gctx, orc, n, (32, 32, 32), (0, 0, 0), rhs, tol=tol,
                           precision=mg.MG_PREC_MIXED)
    assert r64.status == mg.MG_OK and rmx.status == mg.MG_OK and rmx.rel_resid <= tol
    assert np.abs(pmx - p64).max() <= 2 * 0.06 * tol * np.abs(rhs).max()
    o_phi, st, vc, _ = orc.solve(Z3, (n - 1,) * 3, (0, 0, 0), orc.chop(Z3, (n - 1,) * 3, (32,) * 3),
                                 1.0 / n, rhs, tol=tol, mixed=True)
    assert st == 0 and abs(rmx.vcycles - vc) <= 1
    assert np.abs(pmx - o_phi).max() <= 2 * 0.06 * tol * np.abs(rhs).max()


def test_full_size_dirichlet_256(gctx, orc):
    """The benchmarked workload: 256^3 Dirichlet, 64 boxes of 64^3, Jacobi-smoothed N(0,1)."""
    n = 256
    rhs = inputs.dirichlet_jacobi(n, seed=2)
    phi, res = _solve_pair(gctx, orc, n, (64, 64, 64), (0, 0, 0), rhs, ng=(2, 1))
    assert res.status == mg.MG_OK and res.rel_resid <= 1e-10 and res.vcycles <= 30
    r = gu.residual_numpy(phi, rhs, (0, 0, 0), 1.0 / n)
    assert np.abs(r).max() <= 1.01e-10 * np.abs(rhs).max()
    o_phi, st, vc, hist = orc.solve(Z3, (n - 1,) * 3, (0, 0, 0), orc.chop(Z3, (n - 1,) * 3, (64,) * 3),
                                    1.0 / n, rhs)
    assert st == 0 and res.vcycles == vc
    assert np.abs(phi - o_phi).max() <= 1e-12 * np.abs(o_phi).max()


def test_full_size_mixed_512(gctx):
    """The mixed-precision configuration at full size: 512^3 Dirichlet, 64 boxes of 128^3,
    Gaussian blobs.  The answer meets 1e-10 (checked with an independent numpy residual) and
    differs from the plain FP64 GPU answer by at most the bound two converged answers obey."""
    n, tol = 512, 1e-10
    rhs = inputs.gaussian_blobs(n, seed=5)
    dom = (n - 1,) * 3
    ba, _ = _ba(gctx, dom, (128, 128, 128))
    fr = gu.dense_fab(gctx, ba, rhs, 1)
    out = []
    for prec in (mg.MG_PREC_MIXED, mg.MG_PREC_F64):
        fp = mg.mg_fab_alloc(gctx, ba, 1, 2)
        res = mg.mg_solve(gctx, fr, fp, mg.make_bc((0, 0, 0)), tol, mg.make_options(precision=prec))
        assert res.status == mg.MG_OK and res.rel_resid <= tol
        out.append(gu.fab_dense(gctx, fp, rhs.shape))
        mg.mg_fab_free(gctx, fp)
    mg.mg_fab_free(gctx, fr)
    r = gu.residual_numpy(out[0], rhs, (0, 0, 0), 1.0 / n)
    assert np.abs(r).max() <= 1.01 * tol * np.abs(rhs).max()
    assert np.abs(out[0] - out[1]).max() <= 2 * 0.06 * tol * np.abs(rhs).max()


def test_degenerate_domains(gctx, orc):
    """One-cell domains (bottom only: the Dirichlet inverse, the periodic pseudo-inverse), a
    domain with negative low corner, and flat boxes, all against the oracle."""
    for per in [(0, 0, 0), (1, 1, 1), (1, 0, 1)]:
        rhs = np.full((1, 1, 1), 0.0 if all(per) else 2.5)
        phi, res = _solve_pair(gctx, orc, 1, (1, 1, 1), per, rhs)
        o_phi, st, vc, _ = orc.solve(Z3, Z3, per, orc.chop(Z3, Z3, (1, 1, 1)), 1.0, rhs)
        assert res.status == mg.MG_OK and res.vcycles == vc
        assert np.array_equal(phi, o_phi) or np.abs(phi - o_phi).max() <= 1e-14
    g = inputs.rng(50)
    lo, hi = (-8, -16, 4), (7, 15, 19)
    shape = tuple(h - l + 1 for l, h in zip(reversed(lo), reversed(hi)))
    rhs = g.standard_normal(shape)
    for mb in [(8, 8, 8), (16, 4, 16)]:
        ba = mg.mg_box_array_create(gctx, lo, hi, mb)
        fr, fp = gu.dense_fab(gctx, ba, rhs, 0), mg.mg_fab_alloc(gctx, ba, 1, 1)
        res = mg.mg_solve(gctx, fr, fp, mg.make_bc((0, 1, 0)), 1e-10,
                          mg.make_options(fixed_vcycles=3, h=1.0 / 16))
        phi = gu.fab_dense(gctx, fp, rhs.shape)
        o_phi, _, vc, _ = orc.solve(lo, hi, (0, 1, 0), orc.chop(lo, hi, mb), 1.0 / 16, rhs,
                                    fixed_vcycles=3)
        assert res.vcycles == vc == 3
        assert np.abs(phi - o_phi).max() <= 1e-12 * np.abs(o_phi).max()
        mg.mg_fab_free(gctx, fr)
        mg.mg_fab_free(gctx, fp)


# ---- fused red + black sweep (TMA-staged z-slabs) ---------------------------------------

FUSED_CASES = [((63, 63, 63), (64, 64, 64)), ((47, 37, 21), (24, 19, 11)), ((15, 15, 15), (4, 4, 4)),
               ((31, 31, 31), (16, 16, 16)), ((7, 9, 5), (3, 5, 6)), ((15, 15, 39), (8, 16, 40)),
               ((19, 7, 47), (20, 8, 33))]


@pytest.mark.parametrize("dom,mb", FUSED_CASES)
@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0), (1, 0, 0), (0, 1, 1)])
@pytest.mark.parametrize("dt", [mg.MG_F64, mg.MG_F32])
@pytest.mark.parametrize("gp,gr", [(2, 1), (4, 3)])
def test_fused_sweep_bitwise(gctx, orc, dom, mb, periodic, dt, gp, gr):
    """Ghost widths: phi 2 / rhs 1 (the minimum) and wider ones (the sweep reads two / one)."""
    npdt = np.float64 if dt == mg.MG_F64 else np.float32
    h = 1.0 / (dom[0] + 1)
    ba, boxes = _ba(gctx, dom, mb)
    g = inputs.rng(45)
    phi = [g.standard_normal(f.shape).astype(npdt) for f in orc.new_field(boxes, gp)]
    rhs = [g.standard_normal(f.shape).astype(npdt) for f in orc.new_field(boxes, gr)]
    ref = phi
    for color in (0, 1):
        ref = orc.fill_boundary(Z3, dom, periodic, boxes, ref, gp)
        ref = orc.rbgs(Z3, dom, boxes, h, ref, gp, rhs, gr, color)
    bc = mg.make_bc(periodic)
    fa, fr = gu.to_fab(gctx, ba, phi, gp, dt), gu.to_fab(gctx, ba, rhs, gr, dt)
    fb = mg.mg_fab_alloc(gctx, ba, 1, gp, dt)
    mg.mg_fill_boundary(gctx, fa, bc)
    mg.mg_fill_boundary(gctx, fr, bc)
    mg.mg_smooth_fused(gctx, fa, fr, fb, bc, h)
    got = gu.from_fab(gctx, fb, len(boxes))
    for a, r in zip(got, ref):
        assert np.array_equal(gu.valid(a, gp), gu.valid(r, gp))
    for f in (fa, fr, fb):
        mg.mg_fab_free(gctx, f)


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0)])
def test_fused_solver_equals_half_sweep_solver(gctx, orc, periodic):
    n = 64
    rhs = inputs.rng(46).standard_normal((n, n, n))
    if all(periodic):
        rhs = inputs.remove_mean(rhs)
    dom = (n - 1,) * 3
    out = []
    for sm in (mg.MG_SMOOTH_FUSED, mg.MG_SMOOTH_HALF):
        ba, _ = _ba(gctx, dom, (32, 32, 32))
        fr = gu.dense_fab(gctx, ba, rhs, 1)
        fp = mg.mg_fab_alloc(gctx, ba, 1, 2)
        res = mg.mg_solve(gctx, fr, fp, mg.make_bc(periodic), 1e-10, mg.make_options(smoother=sm))
        out.append((gu.fab_dense(gctx, fp, rhs.shape), res.vcycles, res.status))
    assert out[0][2] == out[1][2] == mg.MG_OK and out[0][1] == out[1][1]
    assert np.array_equal(out[0][0], out[1][0])


# ---- the coarse end of the cycle as one launch -----------------------------------------

COARSE_CASES = [
    # domain extents, max box, periodic, precision, coarse_cells
    ((32, 32, 32), (16, 16, 16), (1, 1, 1), mg.MG_PREC_F64, 0),
    ((32, 32, 32), (8, 8, 8), (0, 0, 0), mg.MG_PREC_F64, 4096),
    ((64, 32, 16), (16, 16, 16), (1, 0, 1), mg.MG_PREC_F64, 0),
    ((24, 24, 24), (8, 8, 8), (0, 1, 0), mg.MG_PREC_MIXED, 0),
    ((48, 48, 48), (16, 16, 16), (0, 0, 0), mg.MG_PREC_MIXED, 0),
    ((16, 16, 16), (8, 8, 8), (0, 0, 0), mg.MG_PREC_F64, 4096),    # whole cycle in one launch
    ((16, 16, 16), (16, 16, 16), (1, 1, 1), mg.MG_PREC_MIXED, 0),  # ... in mixed precision
]


def _solve_with(gctx, ext, mb, periodic, rhs, phi0, opt):
    dom = tuple(e - 1 for e in ext)
    ba, _ = _ba(gctx, dom, mb)
    fr = gu.dense_fab(gctx, ba, rhs, 0)
    fp = gu.dense_fab(gctx, ba, phi0, 1)
    before = mg.mg_kernel_launches()
    res = mg.mg_solve(gctx, fr, fp, mg.make_bc(periodic), 1e-10, opt)
    launches = mg.mg_kernel_launches() - before
    phi = gu.fab_dense(gctx, fp, rhs.shape)
    mg.mg_fab_free(gctx, fr)
    mg.mg_fab_free(gctx, fp)
    return phi, res, launches


@pytest.mark.parametrize("ext,mb,periodic,precision,cells", COARSE_CASES)
def test_coarse_cycle_kernel_bitwise(gctx, orc, ext, mb, periodic, precision, cells):
    """The one-launch coarse cycle gives bit for bit the iterates of the stage-by-stage cycle
    (with a non-zero initial guess, which the whole-cycle cases read), in fewer launches."""
    g = inputs.rng(47)
    shape = tuple(reversed(ext))
    rhs = g.standard_normal(shape)
    if all(periodic):
        rhs = inputs.remove_mean(rhs)
    phi0 = 0.1 * g.standard_normal(shape)
    out = []
    for c in (cells, -1):
        opt = mg.make_options(precision=precision, coarse_cells=c)
        _solve_with(gctx, ext, mb, periodic, rhs, phi0, opt)  # one-time tuning not counted
        out.append(_solve_with(gctx, ext, mb, periodic, rhs, phi0, opt))
    (a, ra, la), (b, rb, lb) = out
    assert ra.status == rb.status == mg.MG_OK
    assert ra.vcycles == rb.vcycles and ra.rel_resid == rb.rel_resid
    assert np.array_equal(a, b)
    assert la < lb
    # and against the oracle on a fixed number of cycles (FP64 path)
    if precision == mg.MG_PREC_F64:
        opt = mg.make_options(coarse_cells=cells, fixed_vcycles=2)
        c, _, _ = _solve_with(gctx, ext, mb, periodic, rhs, np.zeros(shape), opt)
        dom = tuple(e - 1 for e in ext)
        o_phi, _, vc, _ = orc.solve(Z3, dom, periodic, orc.chop(Z3, dom, mb), 1.0 / ext[0], rhs,
                                    fixed_vcycles=2)
        assert vc == 2
        assert np.abs(c - o_phi).max() <= 1e-12 * np.abs(o_phi).max()


# ---- stencils reading neighbouring boxes directly -----------------------------------------

DIRECT_CASES = [
    ((32, 32, 32), (16, 16, 16), (0, 0, 0), mg.MG_PREC_F64),
    ((32, 32, 32), (8, 8, 8), (1, 1, 1), mg.MG_PREC_F64),
    ((64, 32, 16), (16, 16, 16), (1, 0, 1), mg.MG_PREC_F64),
    ((32, 32, 32), (32, 32, 32), (0, 1, 0), mg.MG_PREC_F64),     # one box: self images
    ((32, 32, 32), (16, 32, 32), (1, 0, 0), mg.MG_PREC_F64),     # two boxes along x
    ((48, 48, 48), (32, 32, 32), (0, 0, 0), mg.MG_PREC_F64),     # uneven boxes: fills
    ((32, 32, 32), (16, 16, 16), (1, 0, 1), mg.MG_PREC_MIXED),
]


@pytest.mark.parametrize("ext,mb,periodic,precision", DIRECT_CASES)
def test_direct_reads_equal_filled_ghosts(gctx, orc, ext, mb, periodic, precision):
    """Solves whose stencils read neighbouring boxes (or periodic images, or the negated
    boundary cell across Dirichlet faces) directly equal, bit for bit, solves that fill the
    ghost layer first, with a non-zero initial guess."""
    g = inputs.rng(49)
    shape = tuple(reversed(ext))
    rhs = g.standard_normal(shape)
    if all(periodic):
        rhs = inputs.remove_mean(rhs)
    phi0 = 0.1 * g.standard_normal(shape)
    # first use of a shape autotunes the fused FP32 sweep (extra launches): warm it up
    _solve_with(gctx, ext, mb, periodic, rhs, phi0, mg.make_options(precision=precision))
    out = []
    for direct in (1, 0):
        opt = mg.make_options(precision=precision, direct_reads=direct, coarse_cells=-1)
        out.append(_solve_with(gctx, ext, mb, periodic, rhs, phi0, opt))
    (a, ra, la), (b, rb, lb) = out
    assert ra.status == rb.status == mg.MG_OK
    assert ra.vcycles == rb.vcycles and ra.rel_resid == rb.rel_resid
    assert np.array_equal(a, b)
    if mb != (32, 32, 32) or ext != (48, 48, 48):
        assert la < lb          # the fills are gone


@pytest.mark.parametrize("periodic,direct", [((0, 0, 0), 1), ((1, 0, 1), 1), ((0, 0, 0), 0)])
def test_solve_norm_equals_full_residual_norm(gctx, periodic, direct):
    """The norm a solve reports after each V-cycle -- its last black half-sweep takes the
    black cells' residuals, a second pass the red ones -- equals the max-norm of a full
    residual pass over the final iterate."""
    n, mb = 32, (16, 16, 16)
    rhs = inputs.rng(51).standard_normal((n, n, n))
    ba, _ = _ba(gctx, (n - 1,) * 3, mb)
    fr, fp = gu.dense_fab(gctx, ba, rhs, 0), mg.mg_fab_alloc(gctx, ba, 1, 1)
    bc = mg.make_bc(periodic)
    for k in (1, 3):
        mg.mg_fab_set_val(gctx, fp, 0.0, True)
        res = mg.mg_solve(gctx, fr, fp, bc, 1e-10,
                          mg.make_options(fixed_vcycles=k, direct_reads=direct, coarse_cells=-1))
        mg.mg_fill_boundary(gctx, fp, bc)
        full = mg.mg_residual(gctx, fp, fr, 0, 1.0 / n)
        assert res.vcycles == k and res.rel_resid == full / float(np.abs(rhs).max())
    mg.mg_fab_free(gctx, fr)
    mg.mg_fab_free(gctx, fp)


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0), (0, 1, 1)])
def test_smooth_direct_reads_equals_filled(gctx, periodic):
    """mg_smooth with MG_SMOOTH_DIRECT_READS (neighbour boxes read directly, ghost cells
    untouched) equals fill + half-sweep, bit for bit, for both colours."""
    dom, mb, n = (31, 31, 31), (16, 16, 16), 32
    g = inputs.rng(52)
    ba, _ = _ba(gctx, dom, mb)
    phi, rhs = g.standard_normal((n, n, n)), g.standard_normal((n, n, n))
    bc = mg.make_bc(periodic)
    a, b = gu.dense_fab(gctx, ba, phi, 1), gu.dense_fab(gctx, ba, phi, 1)
    fr = gu.dense_fab(gctx, ba, rhs, 0)
    for color in (0, 1, 0):
        mg.mg_fill_boundary(gctx, a, bc)
        mg.mg_smooth(gctx, a, fr, bc, 1.0 / n, color)
        mg.mg_smooth(gctx, b, fr, bc, 1.0 / n, color | mg.MG_SMOOTH_DIRECT_READS)
        assert np.array_equal(gu.fab_dense(gctx, a, phi.shape), gu.fab_dense(gctx, b, phi.shape))
    uneven, _ = _ba(gctx, (47, 47, 47), (32, 32, 32))
    c, d = gu.dense_fab(gctx, uneven, np.zeros((48,) * 3), 1), gu.dense_fab(gctx, uneven, np.zeros((48,) * 3), 0)
    with pytest.raises(mg.MgError):
        mg.mg_smooth(gctx, c, d, bc, 1.0 / 48, mg.MG_SMOOTH_DIRECT_READS)
    for f in (a, b, fr, c, d):
        mg.mg_fab_free(gctx, f)


def test_sweep_timing_inside_solves(gctx):
    n = 64
    rhs = inputs.dirichlet_jacobi(n, seed=2)
    ba, _ = _ba(gctx, (n - 1,) * 3, (32, 32, 32))
    fr, fp = gu.dense_fab(gctx, ba, rhs, 1), mg.mg_fab_alloc(gctx, ba, 1, 2)
    mg.mg_sweep_timing(gctx, True)
    res = mg.mg_solve(gctx, fr, fp, mg.make_bc((0, 0, 0)), 1e-10)
    ms, cnt = mg.mg_sweep_timing(gctx, False)
    assert res.status == mg.MG_OK and cnt == res.vcycles and ms > 0
    mg.mg_fab_set_val(gctx, fp, 0.0, True)
    res2 = mg.mg_solve(gctx, fr, fp, mg.make_bc((0, 0, 0)), 1e-10)
    assert mg.mg_sweep_timing(gctx, False) == (0.0, 0) and res2.vcycles == res.vcycles
    mg.mg_fab_free(gctx, fr)
    mg.mg_fab_free(gctx, fp)


@pytest.mark.parametrize("rhs_smem,ty,depth", [(1, 4, 2), (0, 4, 2), (1, 6, 3), (1, 14, 4),
                                                (0, 22, 4)])
@pytest.mark.parametrize("dt", [mg.MG_F64, mg.MG_F32])
def test_fused_sweep_rhs_staging_forced(orc, tmp_path, monkeypatch, rhs_smem, ty, depth, dt):
    """Both ways the fused sweep reads rhs (staged through shared memory by TMA, or from global
    memory), tile heights that leave a ragged last tile and each prefetch depth, forced
    through the tuning file, equal the oracle's fill-red-fill-black."""
    import paper_2403_12179_gb300.build as b
    b.build()
    dom, mb = (31, 47, 15), (16, 24, 16)
    es = 8 if dt == mg.MG_F64 else 4
    align = 16 // es
    pitch = lambda n, g: (n + 2 * g + align - 1) // align * align
    key = f"v2_dt{dt}_b16x24x16_n4_p{pitch(16, 2)}_{pitch(16, 1)}_g2_1"
    tune = tmp_path / "tune.txt"
    tune.write_text(f"{key} {ty} 8 {depth} {rhs_smem}\n")
    monkeypatch.setenv("GBMG_TUNE_FILE", str(tune))
    ctx = mg.mg_init(0)
    try:
        npdt = np.float64 if dt == mg.MG_F64 else np.float32
        ba, boxes = _ba(ctx, dom, mb)
        assert len(boxes) == 4
        g = inputs.rng(53)
        phi = [g.standard_normal(f.shape).astype(npdt) for f in orc.new_field(boxes, 2)]
        rhs = [g.standard_normal(f.shape).astype(npdt) for f in orc.new_field(boxes, 1)]
        ref = phi
        for color in (0, 1):
            ref = orc.fill_boundary(Z3, dom, (0, 1, 0), boxes, ref, 2)
            ref = orc.rbgs(Z3, dom, boxes, 1.0 / 32, ref, 2, rhs, 1, color)
        bc = mg.make_bc((0, 1, 0))
        fa, fr = gu.to_fab(ctx, ba, phi, 2, dt), gu.to_fab(ctx, ba, rhs, 1, dt)
        fb = mg.mg_fab_alloc(ctx, ba, 1, 2, dt)
        mg.mg_fill_boundary(ctx, fa, bc)
        mg.mg_fill_boundary(ctx, fr, bc)
        mg.mg_smooth_fused(ctx, fa, fr, fb, bc, 1.0 / 32)
        for a, r in zip(gu.from_fab(ctx, fb, len(boxes)), ref):
            assert np.array_equal(gu.valid(a, 2), gu.valid(r, 2))
    finally:
        mg.mg_finalize(ctx)


# ---- the mixed-precision form against the oracle's mixed form, iterate by iterate -------
#
# After k outer iterations (FP64 residual, exact power-of-two scaling into FP32, one FP32
# V-cycle, FP64 correction) the GPU iterate equals the oracle's bit for bit: every FP32 and
# FP64 stencil kernel rounds as the oracle does, the scaling and the correction are exact
# operations or single roundings on both sides, and the bottom solve sums in FP64 before one
# rounding to FP32.  The one source of difference is the bottom matrix, which the two sides
# build independently (entries equal to about 1e-16 relative): a bottom value could round to
# the neighbouring binary32 number, an event of probability ~1e-9 per value, so these seeded
# cases are expected to be exact.  Cases: half-sweeps throughout (the default for levels
# below 256^3), the fused sweep on every level but the bottom, and the fused sweep with the
# one-launch coarse cycle switched off (fused sweeps down to 4^3).

MIXED_ITER_CASES = [(mg.MG_SMOOTH_AUTO, 0, 0), (mg.MG_SMOOTH_FUSED, 0, 0),
                    (mg.MG_SMOOTH_FUSED, -1, 0), (mg.MG_SMOOTH_AUTO, 0, 1),
                    (mg.MG_SMOOTH_FUSED, 0, 3)]


@pytest.mark.parametrize("smoother,coarse,inner", MIXED_ITER_CASES)
@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0), (0, 1, 1)])
def test_mixed_iterates_match_oracle_bitwise(gctx, orc, smoother, coarse, inner, periodic):
    """Mixed-form iterates (FP32 inner cycles, inner = 0: the default two) equal the
    oracle's bit for bit after 1, 2 and 3 outer iterations."""
    n, mb = 32, (16, 16, 16)
    dom = (n - 1,) * 3
    rhs = inputs.rng(46).standard_normal((n, n, n))
    if all(periodic):
        rhs = inputs.remove_mean(rhs)
    ba, _ = _ba(gctx, dom, mb)
    fr = gu.dense_fab(gctx, ba, rhs, 1)
    boxes = orc.chop(Z3, dom, mb)
    for k in (1, 2, 3):
        fp = mg.mg_fab_alloc(gctx, ba, 1, 2)
        opt = mg.make_options(precision=mg.MG_PREC_MIXED, fixed_vcycles=k, smoother=smoother,
                              coarse_cells=coarse, inner_cycles=inner)
        res = mg.mg_solve(gctx, fr, fp, mg.make_bc(periodic), 1e-10, opt)
        phi = gu.fab_dense(gctx, fp, rhs.shape)
        mg.mg_fab_free(gctx, fp)
        o_phi, st, vc, _ = orc.solve(Z3, dom, periodic, boxes, 1.0 / n, rhs, fixed_vcycles=k,
                                     mixed=True, inner_cycles=inner or 2)
        assert res.status == mg.MG_OK and res.vcycles == vc == k
        assert np.array_equal(phi, o_phi), (k, np.abs(phi - o_phi).max())
    mg.mg_fab_free(gctx, fr)


def test_mixed_iterates_match_oracle_at_64(gctx, orc):
    """The mixed form at 64^3 (Gaussian blobs, Dirichlet, 8 boxes): three outer iterations
    equal the oracle's bit for bit, and the converged answer meets 1e-10."""
    n, mb = 64, (32, 32, 32)
    dom = (n - 1,) * 3
    rhs = inputs.gaussian_blobs(n, seed=5)
    ba, _ = _ba(gctx, dom, mb)
    fr = gu.dense_fab(gctx, ba, rhs, 1)
    fp = mg.mg_fab_alloc(gctx, ba, 1, 2)
    res = mg.mg_solve(gctx, fr, fp, mg.make_bc((0, 0, 0)), 1e-10,
                      mg.make_options(precision=mg.MG_PREC_MIXED, fixed_vcycles=3))
    phi = gu.fab_dense(gctx, fp, rhs.shape)
    mg.mg_fab_free(gctx, fp)
    mg.mg_fab_free(gctx, fr)
    o_phi, st, vc, _ = orc.solve(Z3, dom, (0, 0, 0), orc.chop(Z3, dom, mb), 1.0 / n, rhs,
                                 fixed_vcycles=3, mixed=True)
    assert res.vcycles == vc == 3
    assert np.array_equal(phi, o_phi), np.abs(phi - o_phi).max()


# ---- binary32 half-sweeps on wide rows (17 to 128 cells) -------------------------------

ROWS_CASES = [((79, 23, 11), (40, 12, 6)), ((63, 31, 15), (64, 16, 8)),
              ((99, 19, 9), (100, 10, 5)), ((63, 63, 31), (32, 32, 32)),
              ((33, 16, 7), (17, 17, 8))]


@pytest.mark.parametrize("dom,mb", ROWS_CASES)
@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0), (1, 0, 1)])
@pytest.mark.parametrize("direct", [False, True])
def test_rbgs_half_wide_rows_bitwise(gctx, orc, dom, mb, periodic, direct):
    """Binary32 half-sweeps on rows of 17 to 128 cells (one, two and four lane steps per
    row, ragged widths), both colours, reading ghost cells or (regular box grids) the
    neighbouring boxes directly -- with every ghost cell NaN, so a stray ghost read would
    show -- equal the oracle bit for bit."""
    h = 1.0 / (dom[0] + 1)
    ba, boxes = _ba(gctx, dom, mb)
    regular = all((dom[d] + 1) % mb[d] == 0 for d in range(3))
    odd_periodic = any(periodic[d] and (dom[d] + 1) % 2 for d in range(3))
    phi, rhs = _level_inputs(orc, boxes, dom, periodic, 1, 0, 34, np.float32)
    bc = mg.make_bc(periodic)
    if direct and (not regular or odd_periodic):
        # direct reads need a regular box grid and even periodic extents (an odd one would
        # make a boundary cell's periodic image a cell of its own colour): refused
        fp, fr = gu.to_fab(gctx, ba, phi, 1, mg.MG_F32), gu.to_fab(gctx, ba, rhs, 0, mg.MG_F32)
        with pytest.raises(mg.MgError) as e:
            mg.mg_smooth(gctx, fp, fr, bc, h, mg.MG_SMOOTH_DIRECT_READS)
        assert e.value.code == mg.MG_EINVAL
        mg.mg_fab_free(gctx, fp)
        mg.mg_fab_free(gctx, fr)
        return
    src = phi
    if direct:
        src = [a.copy() for a in phi]
        for a in src:
            v = a[:, 1:-1, 1:-1, 1:-1].copy()
            a[...] = np.nan
            a[:, 1:-1, 1:-1, 1:-1] = v
    fp, fr = gu.to_fab(gctx, ba, src, 1, mg.MG_F32), gu.to_fab(gctx, ba, rhs, 0, mg.MG_F32)
    ref = phi
    for color in (0, 1, 0):
        ref = orc.fill_boundary(Z3, dom, periodic, boxes, ref, 1)
        ref = orc.rbgs(Z3, dom, boxes, h, ref, 1, rhs, 0, color)
        if not direct:
            mg.mg_fill_boundary(gctx, fp, bc)
        mg.mg_smooth(gctx, fp, fr, bc, h, color | (mg.MG_SMOOTH_DIRECT_READS if direct else 0))
        got = gu.from_fab(gctx, fp, len(boxes))
        for a, r in zip(got, ref):
            assert np.array_equal(gu.valid(a, 1), gu.valid(r, 1))
    mg.mg_fab_free(gctx, fp)
    mg.mg_fab_free(gctx, fr)
