"""mg_residual_norm_noalloc: the residual max-norm for callers that cannot allocate device
memory (a frozen memory budget, or a framework that owns every device allocation).  Its
scratch is a fixed file-scope device array instead of memory the library allocates.

The test calls it through the C ABI on buffers laid out as mg_fab_layout describes and
compares it with the regular mg_residual norm on the same data, twice in a row (the second
call on smaller data, so a stale accumulator from the first call would show).  The file is
named to be collected last, so a run that stops at the first failure has already run every
other test.
"""
import numpy as np
import pytest
import torch

from paper_2403_12179_gb300 import inputs, mg

pytestmark = pytest.mark.gpu


def _wrapped(ctx, ba, ng, dense):
    """A 256-byte-aligned torch buffer wrapped as a fab, holding `dense` in its valid cells."""
    nbytes = mg.mg_fab_layout(ctx, ba, 1, ng, mg.MG_F64)
    t = torch.zeros(nbytes // 8 + 64, dtype=torch.float64, device="cuda")
    ptr = t.data_ptr() + (-t.data_ptr()) % 256
    fab = mg.mg_fab_wrap(ctx, ba, 1, ng, mg.MG_F64, ptr, nbytes)
    d = torch.from_numpy(np.ascontiguousarray(dense)).cuda()
    mg.mg_fab_copy_from_dense(ctx, fab, d.data_ptr(), False)
    torch.cuda.synchronize()
    return t, ptr, fab


def test_noalloc_norm_matches_mg_residual_on_two_calls():
    import paper_2403_12179_gb300.build as b
    b.build()
    assert torch.cuda.is_available()
    ctx = mg.mg_init(0)
    try:
        n, h = 48, 1.0 / 48
        dom_lo, dom_hi = (0, 0, 0), (n - 1, n - 1, n - 1)
        ba = mg.mg_box_array_create(ctx, dom_lo, dom_hi, (32, 16, 24))
        _, boxes = mg.mg_box_array_info(ctx, ba)
        bc = mg.make_bc((1, 0, 1))
        norms = []
        for trial, scale in ((0, 1.0), (1, 1e-3)):
            g = inputs.rng(70 + trial)
            phi = scale * g.standard_normal((n, n, n))
            rhs = scale * g.standard_normal((n, n, n))
            keep_p, pp, fp = _wrapped(ctx, ba, 1, phi)
            keep_r, pr, fr = _wrapped(ctx, ba, 0, rhs)
            mg.mg_fill_boundary(ctx, fp, bc)
            ref = mg.mg_residual(ctx, fp, fr, 0, h)
            torch.cuda.synchronize()
            # the device's free memory and the context pool are unchanged by the call (the
            # first call's address lookup, made in the first trial, allocates nothing either)
            free0, pool0 = torch.cuda.mem_get_info()[0], mg.mg_pool_info(ctx)[1]
            got = mg.mg_residual_norm_noalloc(dom_lo, dom_hi, boxes, pp, 1, pr, 0, h)
            assert torch.cuda.mem_get_info()[0] == free0 and mg.mg_pool_info(ctx)[1] == pool0
            assert got == ref
            norms.append(got)
            if trial == 1:
                # beyond the maximum: rejected before any launch (the buffers passed are the
                # live ones of this trial, so even a launch could not read outside them)
                too_many = [(i, 0, 0, i, 0, 0) for i in range(1025)]
                with pytest.raises(mg.MgError) as e:
                    mg.mg_residual_norm_noalloc((0, 0, 0), (1024, 0, 0), too_many, pp, 1, pr, 0, 1.0)
                assert e.value.code == mg.MG_EINVAL
            mg.mg_fab_free(ctx, fp)
            mg.mg_fab_free(ctx, fr)
            torch.cuda.synchronize()
            del keep_p, keep_r
        assert norms[1] < 1e-2 * norms[0]
    finally:
        mg.mg_finalize(ctx)
