"""Host-side checks of libgbmg.so (no GPU): exported symbols, box arrays, hierarchy, copy
tags and the closed-form bottom matrix, each against the CPU oracle or numpy."""
import ctypes

import numpy as np
import pytest

from paper_2403_12179_gb300 import inputs
from tests import dense_ref

mg = pytest.importorskip("paper_2403_12179_gb300.mg")


@pytest.fixture(scope="module")
def hctx():
    import paper_2403_12179_gb300.build as b
    b.build()
    ctx = mg.mg_init(-1)
    yield ctx
    mg.mg_finalize(ctx)


def test_library_exports_every_declared_symbol(hctx):
    L = mg.lib()
    syms = mg.declared_symbols()
    assert len(syms) >= 30
    missing = [s for s in syms if not hasattr(L, s)]
    assert not missing, missing
    assert mg.mg_version() >= 1


def test_chop_matches_oracle(hctx, orc):
    for dom, mb in [((47, 47, 47), (32, 32, 32)), ((11, 9, 7), (5, 4, 8)), ((255, 255, 255), (64, 64, 64))]:
        ba = mg.mg_box_array_create(hctx, (0, 0, 0), dom, mb)
        _, boxes = mg.mg_box_array_info(hctx, ba)
        assert np.array_equal(np.array(boxes), orc.chop((0, 0, 0), dom, mb))


@pytest.mark.parametrize("dom,mb", [((31, 31, 31), (32, 32, 32)), ((47, 47, 47), (32, 32, 32)),
                                    ((63, 63, 63), (16, 16, 16)), ((31, 31, 31), (12, 20, 32)),
                                    ((95, 47, 23), (32, 16, 8)), ((255, 255, 255), (64, 64, 64))])
def test_hierarchy_matches_oracle(hctx, orc, dom, mb):
    ba = mg.mg_box_array_create(hctx, (0, 0, 0), dom, mb)
    ref = orc.hierarchy((0, 0, 0), dom, orc.chop((0, 0, 0), dom, mb))
    assert mg.mg_hierarchy_levels(hctx, ba) == len(ref)
    for l, (lo, hi, boxes) in enumerate(ref):
        lb = mg.mg_hierarchy_level(hctx, ba, l)
        (dlo, dhi), got = mg.mg_box_array_info(hctx, lb)
        assert tuple(dlo) == tuple(lo) and tuple(dhi) == tuple(hi)
        assert np.array_equal(np.array(got), boxes)
        mg.mg_box_array_free(hctx, lb)


def _apply_tags(tags, boxes, fabs, ng):
    out = [f.copy() for f in fabs]
    written = [np.zeros(f.shape[1:], np.int32) for f in fabs]
    for t in tags:
        sb, db = t[0], t[1]
        sf, dl, dr, ex, sign = np.array(t[2:5]), np.array(t[5:8]), np.array(t[8:11]), t[11:14], t[14]
        k, j, i = np.meshgrid(np.arange(ex[2]), np.arange(ex[1]), np.arange(ex[0]), indexing="ij")
        dlo = np.array(boxes[db][:3])
        dx, dy, dz = dl[0] + i - dlo[0] + ng, dl[1] + j - dlo[1] + ng, dl[2] + k - dlo[2] + ng
        written[db][dz, dy, dx] += 1
        if sign == 0:
            out[db][:, dz, dy, dx] = 0.0
            continue
        slo = np.array(boxes[sb][:3])
        sx = sf[0] + dr[0] * i - slo[0] + ng
        sy = sf[1] + dr[1] * j - slo[1] + ng
        sz = sf[2] + dr[2] * k - slo[2] + ng
        out[db][:, dz, dy, dx] = sign * fabs[sb][:, sz, sy, sx]
    return out, written


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0), (0, 1, 0), (1, 0, 1)])
@pytest.mark.parametrize("dom,mb,ng", [((11, 9, 7), (5, 4, 8), 2), ((15, 15, 15), (8, 8, 8), 1),
                                       ((3, 3, 3), (4, 4, 4), 2), ((1, 2, 1), (2, 3, 2), 1),
                                       ((23, 15, 7), (8, 8, 8), 2), ((11, 9, 7), (5, 4, 8), 4),
                                       ((15, 15, 15), (4, 4, 4), 4)])
def test_copy_tags_reproduce_oracle_fill_bitwise(hctx, orc, periodic, dom, mb, ng):
    if not all(periodic) and any(ng > d + 1 for d, p in zip(dom, periodic) if not p):
        pytest.skip("ghost wider than a Dirichlet extent")
    ba = mg.mg_box_array_create(hctx, (0, 0, 0), dom, mb)
    _, boxes = mg.mg_box_array_info(hctx, ba)
    g = inputs.rng(21)
    fabs = [g.standard_normal(f.shape) for f in orc.new_field(boxes, ng, 2)]
    ref = orc.fill_boundary((0, 0, 0), dom, periodic, boxes, fabs, ng)
    tags = mg.mg_copy_tags(hctx, ba, mg.make_bc(periodic), ng)
    got, written = _apply_tags(tags, boxes, fabs, ng)
    for f, r, w in zip(got, ref, written):
        valid = np.zeros(w.shape, bool)
        valid[ng:w.shape[0] - ng, ng:w.shape[1] - ng, ng:w.shape[2] - ng] = True
        assert np.all(w[valid] == 0) and np.all(w[~valid] == 1)   # each ghost written once
        assert np.array_equal(f, r)


@pytest.mark.parametrize("n", [(2, 2, 2), (3, 3, 3), (2, 3, 4), (4, 4, 4), (10, 10, 10)])
@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0), (0, 1, 1)])
def test_bottom_matrix_matches_oracle_and_numpy(hctx, orc, n, periodic):
    h = 1.0 / 8
    M = mg.mg_bottom_matrix(n, periodic, h)
    R = orc.bottom_matrix(n, periodic, h)
    assert np.abs(M - R).max() <= 1e-12 * np.abs(R).max()
    if np.prod(n) <= 64:
        A = dense_ref.assemble(n, periodic, h)
        ref = np.linalg.pinv(A, rcond=1e-10) if all(periodic) else np.linalg.inv(A)
        assert np.abs(M - ref).max() <= 1e-12 * np.abs(ref).max()


def test_errors_are_reported(hctx):
    with pytest.raises(mg.MgError) as e:
        mg.mg_box_array_from_list(hctx, (0, 0, 0), (7, 7, 7), [(0, 0, 0, 7, 7, 3), (0, 0, 3, 7, 7, 7)])
    assert e.value.code == mg.MG_EINVAL and "overlap" in str(e.value)
    with pytest.raises(mg.MgError):
        mg.mg_box_array_from_list(hctx, (0, 0, 0), (7, 7, 7), [(0, 0, 0, 7, 7, 3)])
    ba = mg.mg_box_array_create(hctx, (0, 0, 0), (87, 87, 87), (32, 32, 32))
    with pytest.raises(mg.MgError) as e:
        mg.mg_hierarchy_levels(hctx, ba)          # 88 -> 11^3 bottom > 1024 cells
    assert "bottom" in str(e.value)
    with pytest.raises(mg.MgError) as e:
        mg.mg_fab_alloc(hctx, ba, 1, 1)
    assert "host-only" in str(e.value)
    bad = mg.mg_bc()
    bad.kind[0][0], bad.kind[0][1] = mg.MG_BC_PERIODIC, mg.MG_BC_DIRICHLET0
    with pytest.raises(mg.MgError):
        mg.mg_copy_tags(hctx, ba, bad, 1)
    assert mg.lib().mg_box_array_info(hctx, ctypes.c_int64(999999), None, None, None) == mg.MG_EINVAL


def test_layout_rows_16_byte_aligned(hctx):
    ba = mg.mg_box_array_create(hctx, (0, 0, 0), (47, 47, 47), (32, 32, 32))
    for dt, es in ((mg.MG_F64, 8), (mg.MG_F32, 4)):
        for g in (0, 1, 2):
            nbytes = mg.mg_fab_layout(hctx, ba, 1, g, dt)
            assert nbytes % 256 == 0
            assert nbytes >= sum((32 + 2 * g) ** 3 for _ in range(1)) * es
