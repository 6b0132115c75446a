"""Calibration entry points: the STREAM triad of Sec. 3.1-3.2 (one launch over all boxes and
one launch per box give the same, exact, answer) and the FP64 rate probe."""
import numpy as np
import pytest
import torch

from paper_2403_12179_gb300 import inputs, mg
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gctx():
    import paper_2403_12179_gb300.build as b
    b.build()
    assert torch.cuda.is_available()
    ctx = mg.mg_init(0)
    yield ctx
    mg.mg_finalize(ctx)


@pytest.mark.parametrize("dt", [mg.MG_F64, mg.MG_F32])
@pytest.mark.parametrize("dom,mb", [((63, 63, 63), (32, 32, 32)), ((40, 17, 9), (16, 8, 4))])
def test_triad_fused_and_per_box_exact(gctx, dt, dom, mb):
    """Small-integer inputs and s = 3 make b + s c exact in either precision, so both launch
    forms must reproduce it bit for bit (ghost cells untouched)."""
    ba = mg.mg_box_array_create(gctx, (0, 0, 0), dom, mb)
    _, boxes = mg.mg_box_array_info(gctx, ba)
    g = inputs.rng(90)
    shape = tuple(d + 1 for d in dom[::-1])
    bd = g.integers(-1000, 1000, size=shape).astype(np.float64)
    cd = g.integers(-1000, 1000, size=shape).astype(np.float64)
    npdt = np.float64 if dt == mg.MG_F64 else np.float32
    fb = gu.to_fab(gctx, ba, _boxes_of(bd, boxes, npdt), 1, dt)
    fc = gu.to_fab(gctx, ba, _boxes_of(cd, boxes, npdt), 1, dt)
    for per_box in (False, True):
        fa = gu.to_fab(gctx, ba, _boxes_of(np.full(shape, 7.0), boxes, npdt), 1, dt)
        mg.mg_triad(gctx, fa, fb, fc, 3.0, per_box)
        torch.cuda.synchronize()
        got = gu.from_fab(gctx, fa, len(boxes))
        want = _boxes_of(bd + 3.0 * cd, boxes, npdt)
        for gb, wb in zip(got, want):
            assert np.array_equal(gu.valid(gb, 1), gu.valid(wb, 1))
            ghost = gb.copy()
            ghost[:, 1:-1, 1:-1, 1:-1] = 7.0
            assert np.all(ghost == 7.0)
        mg.mg_fab_free(gctx, fa)
    mg.mg_fab_free(gctx, fb)
    mg.mg_fab_free(gctx, fc)


def _boxes_of(dense, boxes, dtype):
    """Per-box (1, nz+2, ny+2, nx+2) arrays holding dense's values, ghosts = 7."""
    out = []
    for b in boxes:
        lo, hi = b[:3], b[3:]
        a = np.full((1, hi[2] - lo[2] + 3, hi[1] - lo[1] + 3, hi[0] - lo[0] + 3), 7.0, dtype)
        a[0, 1:-1, 1:-1, 1:-1] = dense[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1]
        out.append(a)
    return out


def test_fp64_probe_counts_its_operations():
    s = torch.cuda.Stream()
    n1 = mg.mg_calib_fp64(s, 10)
    n2 = mg.mg_calib_fp64(s, 20)
    s.synchronize()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert n1 == sms * 8 * 256 * 8 * 10 and n2 == 2 * n1
    with pytest.raises(mg.MgError):
        mg.mg_calib_fp64(s, 0)
