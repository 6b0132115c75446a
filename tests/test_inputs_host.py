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


def test_amr_sine_closed_form():
    """The two-level manufactured problem: u = prod sin(pi x_d) at each level's cell
    centres (level 1 over the refined region, half the cell size) and f = -3 pi^2 u."""
    n0, A, B = 8, (2, 1, 3), (6, 5, 7)
    f0, f1, u0, u1 = inputs.amr_sine(n0, A, B)
    assert u0.shape == (8, 8, 8) and u1.shape == (8, 8, 8)
    h0 = 1.0 / n0
    i, j, k = 3, 5, 6
    assert np.isclose(u0[k, j, i], np.sin(np.pi * (i + .5) * h0) * np.sin(np.pi * (j + .5) * h0) *
                      np.sin(np.pi * (k + .5) * h0), rtol=0, atol=1e-15)
    x = [A[d] * h0 + (v + .5) * h0 / 2 for d, v in enumerate((i, j, k))]
    assert np.isclose(u1[k, j, i], np.prod(np.sin(np.pi * np.array(x))), rtol=0, atol=1e-15)
    assert np.allclose(f1, -3 * np.pi ** 2 * u1, rtol=1e-15, atol=0)
    assert np.allclose(f0, -3 * np.pi ** 2 * u0, rtol=1e-15, atol=0)
