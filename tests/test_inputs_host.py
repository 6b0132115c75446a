"""The seeded input generators: the in-place form the serving benchmark uses (drawing a
request's rhs straight into pinned host memory) gives the same values, bit for bit, as the
reference form that the oracle tests read."""
import numpy as np

from paper_2403_12179_gb300 import inputs


def test_request_rhs_into_equals_rhs():
    reqs = inputs.serving_requests(40, seed=6)
    seen = set()
    for rq in reqs:
        if rq.n > 64 or (rq.n, rq.periodic) in seen:
            continue
        seen.add((rq.n, rq.periodic))
        out = np.empty((rq.n,) * 3)
        rq.rhs_into(out)
        assert np.array_equal(out, rq.rhs())
    assert {p for _, p in seen} == {True, False}


def test_serving_mix_follows_the_recipe():
    reqs = inputs.serving_requests(5000, seed=6)
    t = np.array([r.t_arrive for r in reqs])
    assert np.all(np.diff(t) > 0) and abs(len(t) / t[-1] - 200.0) < 10.0
    ns = np.array([r.n for r in reqs])
    for n, p in zip((32, 64, 128, 256), (0.4, 0.3, 0.2, 0.1)):
        assert abs(np.mean(ns == n) - p) < 0.03
    assert abs(np.mean([r.periodic for r in reqs]) - 0.5) < 0.03
    assert set(r.box for r in reqs) <= {32, 64}
