"""The multi-rank host logic of bench.py on CPU: two gloo ranks (world size 2) initialise the
process group from torchrun-style environment variables, meet at the barriers, take the
maximum of their timed regions over ranks and turn it into the whole-job rate; the reference
arm does no work on ranks other than 0.  (The solve itself is replicated per GPU, never
sharded, so these are the only steps that involve more than one rank.)"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_PROGRAM = r"""
import os, sys, json
sys.path.insert(0, sys.argv[1])
import bench
rank, world, local = bench.dist_init(None, backend="gloo")
assert (rank, world) == (int(os.environ["RANK"]), 2)
bench.barrier(world)
# each rank's timed region: rank r took 100 * (r + 1) ms for 5 units
mx = bench.max_over_ranks(100.0 * (rank + 1), world)
rate = bench.whole_job_rate(world, 5, mx)
bench.barrier(world)
# the reference arm: only rank 0 works (the others return at once, before any oracle work)
class A: steps = 1; warmup = 0
if rank != 0:
    assert bench.run_reference(A(), "dirichlet256") is None
import torch.distributed as dist
dist.destroy_process_group()
print(json.dumps({"rank": rank, "max_ms": mx, "rate": rate}))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_max_and_rate(tmp_path):
    pytest.importorskip("torch.distributed")
    prog = tmp_path / "rank.py"
    prog.write_text(RANK_PROGRAM)
    port = str(_free_port())
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=port, CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, str(prog), ROOT], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=240)
        assert p.returncode == 0, err[-2000:]
        outs.append(out.strip().splitlines()[-1])
    import json
    res = sorted((json.loads(o) for o in outs), key=lambda d: d["rank"])
    for d in res:
        assert d["max_ms"] == 200.0                 # the slower rank's time, on both ranks
        assert abs(d["rate"] - 2 * 5 / 0.2) < 1e-9  # all ranks' units over that time
