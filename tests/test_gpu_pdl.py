"""Programmatic dependent launch changes no result: solves (FP64 with the speculative norm
check and stored residuals, mixed, batched) give the same bits in a process that launches
every kernel plainly (GBMG_NO_PDL=1) as in this one, which launches them with the
attribute."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2403_12179_gb300 import inputs, mg
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (cells per edge, box edge, periodic faces, precision)
CASES = [(64, 16, (0, 0, 0), "f64"), (48, 16, (1, 1, 1), "f64"), (64, 32, (1, 0, 1), "mixed"),
         (32, 8, (0, 1, 0), "f64")]

SCRIPT = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from tests.test_gpu_pdl import run_all
out = run_all()
np.savez(sys.argv[2], **{k: v for k, v in out.items()})
"""


def run_all():
    """Every case solved alone, then all cases as one batch (FP64); dense results by name."""
    ctx = mg.mg_init(0)
    out = {}
    fabs = []
    for i, (n, box, per, prec) in enumerate(CASES):
        r = inputs.rng(300 + i).standard_normal((n, n, n))
        if all(per):
            r = inputs.remove_mean(r)
        ba = mg.mg_box_array_create(ctx, (0, 0, 0), (n - 1,) * 3, (box,) * 3)
        fr = gu.dense_fab(ctx, ba, r, 0)
        fp = mg.mg_fab_alloc(ctx, ba, 1, 1)
        p = mg.MG_PREC_MIXED if prec == "mixed" else mg.MG_PREC_F64
        res = mg.mg_solve(ctx, fr, fp, mg.make_bc(per), 1e-10, mg.make_options(precision=p))
        out[f"alone{i}"] = gu.fab_dense(ctx, fp, (n, n, n))
        out[f"alone{i}_vc"] = np.array([res.vcycles, res.rel_resid])
        mg.mg_fab_set_val(ctx, fp, 0.0, True)
        fabs.append((fr, fp, per, n))
    res = mg.mg_solve_batch(ctx, [f[0] for f in fabs], [f[1] for f in fabs],
                            [mg.make_bc(f[2]) for f in fabs], 1e-10, mg.make_options())
    for i, (fr, fp, per, n) in enumerate(fabs):
        out[f"batch{i}"] = gu.fab_dense(ctx, fp, (n, n, n))
        out[f"batch{i}_vc"] = np.array([res[i].vcycles, res[i].rel_resid])
        mg.mg_fab_free(ctx, fr)
        mg.mg_fab_free(ctx, fp)
    mg.mg_finalize(ctx)
    return out


def test_plain_launches_give_the_same_bits(tmp_path):
    import paper_2403_12179_gb300.build as b
    b.build()
    assert torch.cuda.is_available()
    here = run_all()
    dst = str(tmp_path / "plain.npz")
    env = dict(os.environ, GBMG_NO_PDL="1")
    subprocess.run([sys.executable, "-c", SCRIPT, ROOT, dst], env=env, check=True, cwd=ROOT,
                   timeout=600)
    plain = np.load(dst)
    assert set(plain.files) == set(here)
    for k, v in here.items():
        assert np.array_equal(plain[k], v), k
