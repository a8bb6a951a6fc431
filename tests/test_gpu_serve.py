"""GPU tests of the serving entry points (fe_serve_*): every served request is
solved to the same bar as a single solve (true FP64 residual <= 1e-8 with the
oracle's matrix, field within 1e-6 of the oracle's direct solve, node ids
bit-exact), a request gives bitwise the same field alone and among others
(continuous batching does not change its arithmetic), a request that arrives
while a long solve runs starts beside it and finishes first, and errors and
the memory budget are reported per request."""
import numpy as np
import pytest

from oracle import fem
from paper_0704_2344_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PEC = 255


def _mixed_requests():
    """Small problems of several sizes and tile widths (1, 2, 4, 8 after
    padding), with PEC boxes and a lossy dielectric."""
    rng = np.random.default_rng(11)
    reqs = []
    for i, nrhs in enumerate((1, 3, 2, 5, 1, 4, 7)):
        prob = W.random_small_grid(100 + i, n_max=7, n_pec_boxes=1)
        reqs.append((prob, W.random_waves(nrhs, rng)))
    box = W.pec_box_problem(9, 2.5e9, np.random.default_rng(5), name="pecbox9")
    reqs.append((box, W.random_waves(2, rng)))
    return reqs


def _check_against_oracle(res, prob, waves):
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps)
    B = fem.rhs(prob, waves, maps=maps)
    xref = fem.solve_direct(A, B)
    assert res["status"] == 0, res["message"]
    assert res["n_dof"] == maps.n_dof and res["nrhs"] == B.shape[1]
    np.testing.assert_array_equal(res["node_id"], np.flatnonzero(maps.node_active))
    x = res["x"]
    assert fem.true_relative_residual(A, x, B).max() <= 1e-8
    for c in range(B.shape[1]):
        assert np.linalg.norm(x[:, c] - xref[:, c]) <= 1e-6 * np.linalg.norm(xref[:, c])
    assert all(r["status"] == 0 for r in res["reports"])


@pytest.mark.parametrize("precision", ["FP64", "MIXED", "DF"])
def test_served_requests_match_oracle(fe, ctx, precision):
    reqs = _mixed_requests()
    srv = fe.fe_serve_create(ctx, fe.serve_opts(precision=getattr(fe, f"FE_PREC_{precision}")))
    try:
        tickets = [fe.fe_serve_submit(srv, p, w) for p, w in reqs]
        results = [fe.fe_serve_wait(srv, t, timeout_s=120.0) for t in tickets]
        assert all(r is not None for r in results)
        for (p, w), r in zip(reqs, results):
            _check_against_oracle(r, p, w)
            assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
            assert r["batch_jobs"] >= 1 and r["batch_ctas"] >= 1
        info = fe.fe_serve_info(srv)
        assert info["submitted"] == info["completed"] == len(reqs) and info["failed"] == 0
        assert info["jobs_launched"] >= len(reqs)   # each request runs in one or more segments
        # requests that were ready together shared segments
        assert max(r["batch_jobs"] for r in results) >= 2
        for t in tickets:
            assert fe.fe_serve_release(srv, t) == fe.FE_OK
    finally:
        fe.fe_serve_destroy(srv)


def test_served_equals_single_solve(fe, ctx):
    prob = W.random_small_grid(31, n_max=7, n_pec_boxes=1)
    waves = W.random_waves(3, np.random.default_rng(3))
    mesh = fe.fe_mesh_create_from(ctx, prob)
    system = fe.fe_assemble(ctx, mesh, prob.freq_hz, fe.FE_PREC_FP64)
    try:
        n_dof = fe.fe_mesh_info(mesh)["n_dof"]
        _, x1, _ = fe.fe_solve_batch(ctx, system, waves, n_dof, fe.solve_opts(precision=fe.FE_PREC_FP64))
    finally:
        fe.fe_system_destroy(system)
        fe.fe_mesh_destroy(mesh)
    srv = fe.fe_serve_create(ctx)
    try:
        r = fe.fe_serve_wait(srv, fe.fe_serve_submit(srv, prob, waves), timeout_s=60.0)
    finally:
        fe.fe_serve_destroy(srv)
    assert r["status"] == 0
    assert np.linalg.norm(r["x"] - x1) <= 1e-7 * np.linalg.norm(x1)


def test_serve_request_errors(fe, ctx):
    good = W.random_small_grid(7, n_max=5, n_pec_boxes=1)
    bad = W.empty_box(4)
    bad.material[0, 1, 1] = PEC  # PEC on the outer box
    waves = W.normal_incidence()
    srv = fe.fe_serve_create(ctx)
    try:
        tb = fe.fe_serve_submit(srv, bad, waves)
        tg = fe.fe_serve_submit(srv, good, waves)
        rb = fe.fe_serve_wait(srv, tb, timeout_s=60.0)
        rg = fe.fe_serve_wait(srv, tg, timeout_s=60.0)
        assert rb["status"] == fe.FE_ERR_MESH and rb["x"] is None and rb["message"]
        _check_against_oracle(rg, good, waves)
        with pytest.raises(fe.FeError) as e:
            fe.fe_serve_submit(srv, good, W.random_waves(33, np.random.default_rng(0)))
        assert e.value.status == fe.FE_ERR_INVALID_ARG
        assert fe.fe_serve_release(srv, tb) == fe.FE_OK
        with pytest.raises(fe.FeError) as e:
            fe.fe_serve_poll(srv, tb)
        assert e.value.status == fe.FE_ERR_INVALID_ARG
        info = fe.fe_serve_info(srv)
        assert info["failed"] == 1 and info["completed"] == 2
    finally:
        fe.fe_serve_destroy(srv)


def test_serve_memory_budget(fe, ctx):
    """With a budget that holds about one request at a time every request is
    still served (one after another) and the admitted total never exceeds the
    budget; a request larger than the whole budget fails with FE_ERR_OOM."""
    rng = np.random.default_rng(21)
    reqs = [(W.pec_box_problem(8, 3e9, rng, name=f"b{i}"), W.random_waves(2, rng)) for i in range(4)]
    budget = 12 << 20  # each request's estimate is about 8.2 MiB in the FP32-pair mode
    srv = fe.fe_serve_create(ctx, fe.serve_opts(precision=fe.FE_PREC_DF, hbm_budget=budget))
    try:
        tickets = [fe.fe_serve_submit(srv, p, w) for p, w in reqs]
        big = W.empty_box(60, name="big")
        tbig = fe.fe_serve_submit(srv, big, W.normal_incidence())
        for (p, w), t in zip(reqs, tickets):
            _check_against_oracle(fe.fe_serve_wait(srv, t, timeout_s=120.0), p, w)
        rbig = fe.fe_serve_wait(srv, tbig, timeout_s=60.0)
        assert rbig["status"] == fe.FE_ERR_OOM and "budget" in rbig["message"]
        info = fe.fe_serve_info(srv)
        assert info["budget_bytes"] == budget
        assert 0 < info["peak_admitted_bytes"] <= budget
    finally:
        fe.fe_serve_destroy(srv)


def test_serve_destroy_with_pending_requests(fe, ctx):
    """Destroying a server with queued requests stops cleanly."""
    rng = np.random.default_rng(4)
    srv = fe.fe_serve_create(ctx)
    for i in range(6):
        fe.fe_serve_submit(srv, W.random_small_grid(200 + i, n_max=6, n_pec_boxes=1), W.random_waves(2, rng))
    fe.fe_serve_destroy(srv)


def test_request_alone_and_in_a_mix_is_bitwise_the_same(fe, ctx):
    """Request Q served alone, then the same Q third in a stream of eight
    requests of other sizes and tile widths: its CTA count depends on its own
    size only, and a segment boundary saves and restores its Krylov state
    exactly, so the two fields are bitwise equal; both meet the oracle."""
    rng = np.random.default_rng(17)
    q_prob = W.pec_box_problem(12, 3.2e9, np.random.default_rng(8), name="q")
    q_waves = W.random_waves(3, rng)
    others = [(W.random_small_grid(300 + i, n_max=8, n_pec_boxes=1), W.random_waves(int(k), rng))
              for i, k in enumerate((1, 5, 2, 9, 1, 4, 16))]
    srv = fe.fe_serve_create(ctx, fe.serve_opts(precision=fe.FE_PREC_DF, seg_iters=16))
    try:
        alone = fe.fe_serve_wait(srv, fe.fe_serve_submit(srv, q_prob, q_waves), timeout_s=120.0)
        tickets = [fe.fe_serve_submit(srv, p, w) for p, w in others[:2]]
        tq = fe.fe_serve_submit(srv, q_prob, q_waves)
        tickets += [fe.fe_serve_submit(srv, p, w) for p, w in others[2:]]
        mixed = fe.fe_serve_wait(srv, tq, timeout_s=120.0)
        rest = [fe.fe_serve_wait(srv, t, timeout_s=120.0) for t in tickets]
    finally:
        fe.fe_serve_destroy(srv)
    _check_against_oracle(alone, q_prob, q_waves)
    _check_against_oracle(mixed, q_prob, q_waves)
    assert mixed["batch_jobs"] >= 2           # it really shared segments
    assert alone["reports"][0]["iterations"] > 16   # and ran over several segments
    np.testing.assert_array_equal(mixed["x"], alone["x"])
    assert [r["iterations"] for r in mixed["reports"]] == [r["iterations"] for r in alone["reports"]]
    for (p, w), r in zip(others, rest):
        _check_against_oracle(r, p, w)


def test_request_arriving_mid_solve_finishes_first(fe, ctx):
    """A small request submitted while a long solve is on the device is
    admitted at the next segment, runs beside it and finishes before it."""
    import time

    long_prob = W.pec_box_problem(44, 3e9, np.random.default_rng(3), name="long")
    long_waves = W.random_waves(16, np.random.default_rng(4))
    small = W.random_small_grid(41, n_max=6, n_pec_boxes=1)
    small_waves = W.random_waves(2, np.random.default_rng(5))
    srv = fe.fe_serve_create(ctx, fe.serve_opts(precision=fe.FE_PREC_DF))
    try:
        tl = fe.fe_serve_submit(srv, long_prob, long_waves)
        # wait until the long request is admitted and its first segments run
        t0 = time.time()
        while fe.fe_serve_info(srv)["jobs_launched"] < 1 and time.time() - t0 < 60:
            time.sleep(0.002)
        ts = fe.fe_serve_submit(srv, small, small_waves)
        rs = fe.fe_serve_wait(srv, ts, timeout_s=120.0)
        rl = fe.fe_serve_wait(srv, tl, timeout_s=300.0)
    finally:
        fe.fe_serve_destroy(srv)
    assert rl["status"] == 0 and rs["status"] == 0
    assert rs["t_submit"] > rl["t_admit"]       # it arrived while the long one was in flight
    assert rs["t_done"] < rl["t_done"]          # and did not wait for it
    _check_against_oracle(rs, small, small_waves)
