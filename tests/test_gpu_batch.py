"""Batched solves (one launch per V-cycle stage for many solves) and the serving loop
(continuous batching via mg_submit / mg_poll): every result must equal, bit for bit, the
same problem solved alone with mg_solve, whatever company it had."""
import time

import numpy as np
import pytest
import torch

from paper_2403_12179_gb300 import inputs, mg
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

PROBLEMS = [(32, 16, (1, 1, 1)), (24, 8, (0, 0, 0)), (16, 16, (1, 0, 1)), (48, 16, (0, 0, 0)),
            (8, 8, (1, 1, 1)), (32, 32, (0, 1, 0)), (2, 2, (0, 0, 0))]


@pytest.fixture(scope="module")
def gctx():
    import paper_2403_12179_gb300.build as b
    b.build()
    assert torch.cuda.is_available()
    ctx = mg.mg_init(0)
    yield ctx
    mg.mg_finalize(ctx)


def _rhs(n, periodic, seed):
    r = inputs.rng(seed).standard_normal((n, n, n))
    return inputs.remove_mean(r) if all(periodic) else r


def _make(ctx, n, box, periodic, seed, ng=(2, 1)):
    ba = mg.mg_box_array_create(ctx, (0, 0, 0), (n - 1,) * 3, (box,) * 3)
    rhs = _rhs(n, periodic, seed)
    fr = gu.dense_fab(ctx, ba, rhs, ng[1])
    fp = mg.mg_fab_alloc(ctx, ba, 1, ng[0])
    return rhs, fr, fp


def _alone(ctx, n, box, periodic, seed, precision, smoother=mg.MG_SMOOTH_AUTO,
           prolong=mg.MG_PROLONG_CONSTANT, **opts):
    rhs, fr, fp = _make(ctx, n, box, periodic, seed)
    res = mg.mg_solve(ctx, fr, fp, mg.make_bc(periodic), 1e-10,
                      mg.make_options(precision=precision, smoother=smoother, prolong=prolong,
                                      **opts))
    phi = gu.fab_dense(ctx, fp, rhs.shape)
    mg.mg_fab_free(ctx, fr)
    mg.mg_fab_free(ctx, fp)
    return phi, res


TRI = mg.MG_PROLONG_TRILINEAR


@pytest.mark.parametrize("precision,smoother,prolong",
                         [(mg.MG_PREC_F64, mg.MG_SMOOTH_AUTO, 0), (mg.MG_PREC_MIXED, mg.MG_SMOOTH_AUTO, 0),
                          (mg.MG_PREC_F64, mg.MG_SMOOTH_FUSED, 0), (mg.MG_PREC_MIXED, mg.MG_SMOOTH_FUSED, 0),
                          (mg.MG_PREC_F64, mg.MG_SMOOTH_AUTO, TRI), (mg.MG_PREC_MIXED, mg.MG_SMOOTH_FUSED, TRI)])
def test_batch_equals_alone_bitwise(gctx, precision, smoother, prolong):
    alone = [_alone(gctx, n, b, p, 100 + i, precision, smoother, prolong)
             for i, (n, b, p) in enumerate(PROBLEMS)]
    made = [_make(gctx, n, b, p, 100 + i) for i, (n, b, p) in enumerate(PROBLEMS)]
    res = mg.mg_solve_batch(gctx, [m[1] for m in made], [m[2] for m in made],
                            [mg.make_bc(p) for (_, _, p) in PROBLEMS], 1e-10,
                            mg.make_options(precision=precision, smoother=smoother, prolong=prolong))
    for (rhs, fr, fp), r, (phi_a, res_a) in zip(made, res, alone):
        assert r.status == mg.MG_OK and res_a.status == mg.MG_OK
        assert r.vcycles == res_a.vcycles and r.rel_resid <= 1e-10
        assert np.array_equal(gu.fab_dense(gctx, fp, rhs.shape), phi_a)
    for _, fr, fp in made:
        mg.mg_fab_free(gctx, fr)
        mg.mg_fab_free(gctx, fp)


def test_batch_reports_each_status(gctx):
    made = [_make(gctx, 16, 8, (0, 0, 0), 120), _make(gctx, 16, 8, (0, 0, 0), 121)]
    rhs_bad = made[1][0].copy()
    rhs_bad[3, 4, 5] = np.nan
    t = torch.from_numpy(rhs_bad).cuda()
    mg.mg_fab_copy_from_dense(gctx, made[1][1], t.data_ptr(), False)
    torch.cuda.synchronize()
    res = mg.mg_solve_batch(gctx, [m[1] for m in made], [m[2] for m in made],
                            [mg.make_bc((0, 0, 0))] * 2, 1e-10)
    assert res[0].status == mg.MG_OK and res[1].status == mg.MG_ENAN


def _serve(ctx, specs, precision, timeout_ms=-1):
    made, tickets = [], []
    for i, (n, b, p) in enumerate(specs):
        m = _make(ctx, n, b, p, 200 + i)
        made.append(m)
        tickets.append(mg.mg_submit(ctx, m[1], m[2], mg.make_bc(p), 1e-10,
                                    mg.make_options(precision=precision)))
    out = []
    for t in tickets:
        rc, r = mg.mg_poll(ctx, t, timeout_ms)
        assert rc == mg.MG_OK
        out.append(r)
    return made, out


@pytest.mark.parametrize("precision", [mg.MG_PREC_F64, mg.MG_PREC_MIXED])
def test_serving_results_equal_alone(precision):
    ctx = mg.mg_init(0)
    actx = mg.mg_init(0)
    try:
        specs = PROBLEMS * 2
        made, res = _serve(ctx, specs, precision)
        for i, ((n, b, p), (rhs, fr, fp), r) in enumerate(zip(specs, made, res)):
            assert r.status == mg.MG_OK and r.rel_resid <= 1e-10
            assert r.t_end >= r.t_admit >= r.t_start and r.seconds > 0
            phi = gu.fab_dense(ctx, fp, rhs.shape)
            phi_a, res_a = _alone(actx, n, b, p, 200 + i, precision)
            assert res_a.vcycles == r.vcycles
            assert np.array_equal(phi, phi_a)
    finally:
        mg.mg_finalize(ctx)
        mg.mg_finalize(actx)


def test_serving_many_members_both_precisions_equal_alone():
    """More members than the initial norm slots hold (the arrays grow while members run),
    FP64 and mixed-precision members (half-sweep and fused smoothers, injection and trilinear
    prolongation, one to three inner cycles, V(2,2) and V(1,1) -- members that step in
    separate groups) at once, later requests joining running ones: every result and V-cycle
    count equals the solve alone."""
    ctx = mg.mg_init(0)
    actx = mg.mg_init(0)
    try:
        count = 84
        specs = [PROBLEMS[i % len(PROBLEMS)] for i in range(count)]
        precs = [mg.MG_PREC_F64 if i % 3 == 0 else mg.MG_PREC_MIXED for i in range(count)]
        smooth = [mg.MG_SMOOTH_FUSED if i % 3 == 2 else mg.MG_SMOOTH_AUTO for i in range(count)]
        prol = [mg.MG_PROLONG_TRILINEAR if i % 4 == 3 else mg.MG_PROLONG_CONSTANT for i in range(count)]
        extra = [dict(inner_cycles=(i // 2) % 4, nu1=1 + (i % 5 == 4), nu2=1 + (i % 5 == 4))
                 if i % 2 else {} for i in range(count)]
        made, tickets = [], []
        for i, ((n, b, p), pr) in enumerate(zip(specs, precs)):
            m = _make(ctx, n, b, p, 400 + i)
            made.append(m)
            tickets.append(mg.mg_submit(ctx, m[1], m[2], mg.make_bc(p), 1e-10,
                                        mg.make_options(precision=pr, smoother=smooth[i],
                                                        prolong=prol[i], **extra[i])))
            if i % 12 == 11:
                time.sleep(0.02)
        res = [mg.mg_poll(ctx, t, -1)[1] for t in tickets]
        stats = mg.mg_server_stats_get(ctx)
        assert stats["completed"] == count
        for i, ((n, b, p), pr, (rhs, fr, fp), r) in enumerate(zip(specs, precs, made, res)):
            phi = gu.fab_dense(ctx, fp, rhs.shape)
            phi_a, res_a = _alone(actx, n, b, p, 400 + i, pr, smooth[i], prol[i], **extra[i])
            # (V(1,1) with injection does not reach 1e-10 in 50 cycles on some of these
            # problems: the served solve must then stop the same way)
            assert r.status == res_a.status, (i, n, b, p, pr, extra[i])
            assert r.status != mg.MG_OK or r.rel_resid <= 1e-10
            assert res_a.vcycles == r.vcycles, (i, n, b, p, pr)
            assert np.array_equal(phi, phi_a)
    finally:
        mg.mg_finalize(ctx)
        mg.mg_finalize(actx)


def _wrapped_problem(ctx, n, box, per, seed, keep):
    ba = mg.mg_box_array_create(ctx, (0, 0, 0), (n - 1,) * 3, (box,) * 3)
    rhs = _rhs(n, per, seed)
    out = []
    for ng in (1, 2):
        nb = mg.mg_fab_layout(ctx, ba, 1, ng, mg.MG_F64)
        t = torch.zeros(nb // 8 + 64, dtype=torch.float64, device="cuda")
        ptr = t.data_ptr() + (-t.data_ptr()) % 256
        keep.append(t)
        out.append(mg.mg_fab_wrap(ctx, ba, 1, ng, mg.MG_F64, ptr, nb))
    fr, fp = out
    t = torch.from_numpy(rhs).cuda()
    mg.mg_fab_copy_from_dense(ctx, fr, t.data_ptr(), False)
    torch.cuda.synchronize()
    return rhs, fr, fp


def test_serving_admission_under_small_pool():
    """The pool holds the coarse levels of about two solves at a time: later requests wait
    for running solves to retire, and every result equals the solve alone."""
    n, box, per = 64, 32, (0, 0, 0)
    keep = []
    # bytes one solve's hierarchy takes from the pool
    probe = mg.mg_init(0)
    try:
        rhs, fr, fp = _wrapped_problem(probe, n, box, per, 299, keep)
        _, before = mg.mg_pool_info(probe)
        mg.mg_solve(probe, fr, fp, mg.make_bc(per), 1e-10)
        _, after = mg.mg_pool_info(probe)
    finally:
        mg.mg_finalize(probe)
    per_solve = after - before
    assert per_solve > 0
    ctx = mg.mg_init(0)
    _, base = mg.mg_pool_info(ctx)
    mg.mg_finalize(ctx)
    ctx = mg.mg_init(0, base + int(2.5 * per_solve) + (1 << 20))
    actx = mg.mg_init(0)
    try:
        made = [_wrapped_problem(ctx, n, box, per, 300 + i, keep) for i in range(8)]
        tickets = [mg.mg_submit(ctx, fr, fp, mg.make_bc(per), 1e-10) for (_, fr, fp) in made]
        res = [mg.mg_poll(ctx, t, -1)[1] for t in tickets]
        assert all(r.status == mg.MG_OK for r in res)
        first_end = min(r.t_end for r in res)
        assert sum(r.t_admit >= first_end for r in res) >= 4   # admitted only after retirements
        for i, ((rhs, fr, fp), r) in enumerate(zip(made, res)):
            phi = gu.fab_dense(ctx, fp, rhs.shape)
            phi_a, res_a = _alone(actx, n, box, per, 300 + i, mg.MG_PREC_F64)
            assert np.array_equal(phi, phi_a) and res_a.vcycles == r.vcycles
    finally:
        mg.mg_finalize(ctx)
        mg.mg_finalize(actx)


def test_poll_paths():
    ctx = mg.mg_init(0)
    try:
        with pytest.raises(mg.MgError):
            mg.mg_poll(ctx, 12345, 0)
        rhs, fr, fp = _make(ctx, 128, 64, (0, 0, 0), 400)
        t = mg.mg_submit(ctx, fr, fp, mg.make_bc((0, 0, 0)), 1e-10)
        rc, _ = mg.mg_poll(ctx, t, 0)
        assert rc in (mg.MG_PENDING, mg.MG_OK)
        if rc == mg.MG_PENDING:
            rc, r = mg.mg_poll(ctx, t, -1)
            assert rc == mg.MG_OK and r.status == mg.MG_OK
        with pytest.raises(mg.MgError):
            mg.mg_poll(ctx, t, 0)            # a ticket is released once reported
    finally:
        mg.mg_finalize(ctx)


@pytest.mark.parametrize("precision", [mg.MG_PREC_F64, mg.MG_PREC_MIXED])
def test_batch_coarse_cycle_kernel_bitwise(gctx, precision):
    """Batched solves whose coarse levels run as one launch (one CTA per member, members of
    several depths) equal the batch run stage by stage."""
    out = []
    for cells in (0, -1):
        made = [_make(gctx, n, b, p, 500 + i) for i, (n, b, p) in enumerate(PROBLEMS)]
        res = mg.mg_solve_batch(gctx, [m[1] for m in made], [m[2] for m in made],
                                [mg.make_bc(p) for (_, _, p) in PROBLEMS], 1e-10,
                                mg.make_options(precision=precision, coarse_cells=cells))
        out.append(([gu.fab_dense(gctx, m[2], m[0].shape) for m in made],
                    [(r.status, r.vcycles) for r in res]))
        for _, fr, fp in made:
            mg.mg_fab_free(gctx, fr)
            mg.mg_fab_free(gctx, fp)
    assert out[0][1] == out[1][1] and all(s == mg.MG_OK for s, _ in out[0][1])
    for a, b in zip(out[0][0], out[1][0]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [mg.MG_PREC_F64, mg.MG_PREC_MIXED])
def test_batch_direct_reads_bitwise(gctx, precision):
    """Batched members reading neighbouring boxes directly (regular grids) or through filled
    ghosts (uneven boxes) equal the batch that fills every level."""
    out = []
    for direct in (1, 0):
        made = [_make(gctx, n, b, p, 600 + i) for i, (n, b, p) in enumerate(PROBLEMS)]
        res = mg.mg_solve_batch(gctx, [m[1] for m in made], [m[2] for m in made],
                                [mg.make_bc(p) for (_, _, p) in PROBLEMS], 1e-10,
                                mg.make_options(precision=precision, direct_reads=direct))
        out.append(([gu.fab_dense(gctx, m[2], m[0].shape) for m in made],
                    [(r.status, r.vcycles) for r in res]))
        for _, fr, fp in made:
            mg.mg_fab_free(gctx, fr)
            mg.mg_fab_free(gctx, fp)
    assert out[0][1] == out[1][1] and all(s == mg.MG_OK for s, _ in out[0][1])
    for a, b in zip(out[0][0], out[1][0]):
        assert np.array_equal(a, b)


def test_full_size_batched_512(gctx):
    """The batched configuration at full size: 512 periodic problems, edges drawn from
    {32, 48, 64, 96, 128}, 32^3 boxes, mixed precision in one batch.  Every member converges,
    and sampled members equal the same problem solved alone, bit for bit."""
    probs = inputs.batched_periodic(512, seed=4)
    fr, fp = [], []
    for pb in probs:
        ba = mg.mg_box_array_create(gctx, (0, 0, 0), (pb.n - 1,) * 3, (pb.box,) * 3)
        fr.append(gu.dense_fab(gctx, ba, pb.rhs(), 1))
        fp.append(mg.mg_fab_alloc(gctx, ba, 1, 2))
    opt = mg.make_options(precision=mg.MG_PREC_MIXED)
    res = mg.mg_solve_batch(gctx, fr, fp, [mg.make_bc((1, 1, 1))] * len(probs), 1e-10, opt)
    assert all(r.status == mg.MG_OK and r.rel_resid <= 1e-10 for r in res)
    actx = mg.mg_init(0)
    try:
        for i in (0, 17, 256, 511):
            pb = probs[i]
            ba = mg.mg_box_array_create(actx, (0, 0, 0), (pb.n - 1,) * 3, (pb.box,) * 3)
            a, b = gu.dense_fab(actx, ba, pb.rhs(), 1), mg.mg_fab_alloc(actx, ba, 1, 2)
            r = mg.mg_solve(actx, a, b, mg.make_bc((1, 1, 1)), 1e-10, opt)
            assert r.vcycles == res[i].vcycles
            assert np.array_equal(gu.fab_dense(actx, b, (pb.n,) * 3),
                                  gu.fab_dense(gctx, fp[i], (pb.n,) * 3))
    finally:
        mg.mg_finalize(actx)
    for a, b in zip(fr, fp):
        mg.mg_fab_free(gctx, a)
        mg.mg_fab_free(gctx, b)


# ---- serving from host memory (mg_submit_host) ------------------------------------------

def _pinned(a):
    t = torch.from_numpy(np.ascontiguousarray(a, np.float64)).pin_memory()
    return t


def _serve_host(ctx, specs, precision, seed0):
    """Submit every spec as a host-memory request (pinned rhs and phi); returns the rhs, the
    pinned phi tensors and the results."""
    rhs, phis, tickets = [], [], []
    for i, (n, b, p) in enumerate(specs):
        r = _pinned(_rhs(n, p, seed0 + i))
        ph = torch.zeros((n, n, n), dtype=torch.float64).pin_memory()
        rhs.append(r)
        phis.append(ph)
        tickets.append(mg.mg_submit_host(ctx, (0, 0, 0), (n - 1,) * 3, (b,) * 3, mg.make_bc(p),
                                         r.data_ptr(), ph.data_ptr(), False, 1e-10,
                                         mg.make_options(precision=precision)))
    res = [mg.mg_poll(ctx, t, -1)[1] for t in tickets]
    return rhs, phis, res


@pytest.mark.parametrize("precision", [mg.MG_PREC_F64, mg.MG_PREC_MIXED])
def test_serving_from_host_equals_alone(precision):
    """Requests whose rhs and phi live in (pinned) host memory: the scheduler allocates their
    fine levels from the pool, copies rhs in and phi out; each answer equals the solve alone,
    bit for bit, and the pool returns to its starting level once all have completed."""
    ctx = mg.mg_init(0)
    actx = mg.mg_init(0)
    try:
        _, pool0 = mg.mg_pool_info(ctx)
        specs = PROBLEMS * 2
        rhs, phis, res = _serve_host(ctx, specs, precision, 600)
        for i, ((n, b, p), r, ph) in enumerate(zip(specs, res, phis)):
            assert r.status == mg.MG_OK and r.rel_resid <= 1e-10
            assert r.t_end >= r.t_admit >= r.t_start and r.seconds > 0
            phi_a, res_a = _alone(actx, n, b, p, 600 + i, precision)
            assert res_a.vcycles == r.vcycles
            assert np.array_equal(ph.numpy(), phi_a)
        assert mg.mg_server_stats_get(ctx)["completed"] == len(specs)
        # the workspaces stay resident: the same requests again reuse them (the pool does
        # not grow, and the answers are the same); mg_server_trim releases them
        _, held = mg.mg_pool_info(ctx)
        assert held > pool0
        _, phis2, res2 = _serve_host(ctx, specs, precision, 600)
        assert mg.mg_pool_info(ctx)[1] <= held + (1 << 20)
        for a, b, r in zip(phis, phis2, res2):
            assert r.status == mg.MG_OK and torch.equal(a, b)
        mg.mg_server_trim(ctx)
        assert mg.mg_pool_info(ctx)[1] <= pool0 + (1 << 20)   # fine levels released too
    finally:
        mg.mg_finalize(ctx)
        mg.mg_finalize(actx)


def test_serving_from_host_admission_by_pool_room():
    """A pool with room for about two whole host-memory requests (fine level, copies and
    coarse levels): later ones wait in the queue until running ones retire; a request larger
    than the empty pool completes with MG_ENOMEM; every other answer equals the solve alone."""
    n, box, per = 64, 32, (0, 0, 0)
    probe = mg.mg_init(0)
    try:
        ba = mg.mg_box_array_create(probe, (0, 0, 0), (n - 1,) * 3, (box,) * 3)
        fine = mg.mg_fab_layout(probe, ba, 1, 1, mg.MG_F64) + mg.mg_fab_layout(probe, ba, 1, 2, mg.MG_F64)
        rhs, fr, fp = _make(probe, n, box, per, 299)
        _, before = mg.mg_pool_info(probe)
        mg.mg_solve(probe, fr, fp, mg.make_bc(per), 1e-10)
        _, after = mg.mg_pool_info(probe)
    finally:
        mg.mg_finalize(probe)
    one = fine + (after - before) + 2 * n ** 3 * 8
    ctx = mg.mg_init(0)
    _, base = mg.mg_pool_info(ctx)
    mg.mg_finalize(ctx)
    ctx = mg.mg_init(0, base + int(2.5 * one) + (1 << 20))
    actx = mg.mg_init(0)
    try:
        specs = [(n, box, per)] * 8
        rhs, phis, res = _serve_host(ctx, specs, mg.MG_PREC_F64, 700)
        assert all(r.status == mg.MG_OK for r in res)
        first_end = min(r.t_end for r in res)
        assert sum(r.t_admit >= first_end for r in res) >= 4
        for i, (r, ph) in enumerate(zip(res, phis)):
            phi_a, res_a = _alone(actx, n, box, per, 700 + i, mg.MG_PREC_F64)
            assert np.array_equal(ph.numpy(), phi_a) and res_a.vcycles == r.vcycles
        big = 256
        rb = _pinned(_rhs(big, per, 799))
        pb = torch.zeros((big,) * 3, dtype=torch.float64).pin_memory()
        t = mg.mg_submit_host(ctx, (0, 0, 0), (big - 1,) * 3, (64,) * 3, mg.make_bc(per),
                              rb.data_ptr(), pb.data_ptr(), False, 1e-10)
        rc, r = mg.mg_poll(ctx, t, -1)
        assert rc == mg.MG_OK and r.status == mg.MG_ENOMEM
    finally:
        mg.mg_finalize(ctx)
        mg.mg_finalize(actx)


def test_serving_from_host_with_initial_guess():
    """phi_is_guess = 1 starts from the caller's phi: a converged answer submitted as its own
    guess needs no V-cycle and comes back unchanged."""
    ctx = mg.mg_init(0)
    try:
        n, b, p = 32, 16, (0, 0, 0)
        rhs, phis, res = _serve_host(ctx, [(n, b, p)], mg.MG_PREC_F64, 800)
        assert res[0].status == mg.MG_OK and res[0].vcycles > 0
        guess = phis[0].clone().pin_memory()
        t = mg.mg_submit_host(ctx, (0, 0, 0), (n - 1,) * 3, (b,) * 3, mg.make_bc(p),
                              rhs[0].data_ptr(), guess.data_ptr(), True, 1e-10)
        rc, r = mg.mg_poll(ctx, t, -1)
        assert rc == mg.MG_OK and r.status == mg.MG_OK and r.vcycles == 0
        assert torch.equal(guess, phis[0])
    finally:
        mg.mg_finalize(ctx)
