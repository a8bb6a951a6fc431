"""GPU parity at full size on the batched and large-scatterer workloads.

* The 3-wavelength cube with its 64 sphere waves (32 directions x two
  polarisations), solved in FP32-pair mode through fe_solve_batch with the
  library's tile autotuner: every column reaches a true FP64 residual of
  1e-8 (recomputed on the CPU with the oracle's matrix), and the columns the
  oracle solved directly (tests/golden/config3_x.npz, two of each 32-column
  launch) match to 1e-6 in full, and all 64 columns match to 1e-6 on a seeded
  sample of 4 096 unknowns.
* The 40^3 voxel aircraft (206 k unknowns, the half-size stand-in for the
  paper's PEC airplane), one wave: residual 1e-8 and field error 1e-6 against
  the oracle's solution (tests/golden/aircraft40_x.npz, COCG to 1e-12).
* The autotuner keeps its choice per system shape: a second solve of the same
  shape takes it from the cache.
* On the aircraft the expanded form of p^T A p shortens the FP32-pair solve's
  residual plateau."""
from pathlib import Path

import numpy as np
import pytest

from oracle import fem
from paper_0704_2344_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = Path(__file__).with_name("golden")


def _solve(fe, ctx, prob, waves, precision, **kw):
    mesh = fe.fe_mesh_create_from(ctx, prob)
    try:
        system = fe.fe_assemble(ctx, mesh, prob.freq_hz, precision)
        try:
            n_dof = fe.fe_mesh_info(mesh)["n_dof"]
            st, x, rep = fe.fe_solve_batch(ctx, system, waves, n_dof, fe.solve_opts(precision=precision, **kw),
                                           raise_on_fail=False)
            stats = fe.fe_last_solve_stats(ctx)
        finally:
            fe.fe_system_destroy(system)
    finally:
        fe.fe_mesh_destroy(mesh)
    return st, x, rep, stats


def test_config3_64_waves_match_the_direct_solve(fe, ctx):
    prob, waves = W.config3()
    ref = np.load(GOLDEN / "config3_x.npz")
    st, x, rep, stats = _solve(fe, ctx, prob, waves, fe.FE_PREC_DF)
    assert st == fe.FE_OK and all(r["status"] == fe.FE_OK for r in rep)
    assert stats["tuned"] in (1, 2) and stats["tile_width"] in (8, 16, 32)
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps)
    B = fem.rhs(prob, waves, maps=maps)
    assert fem.true_relative_residual(A, x, B).max() <= 1e-8
    for k, c in enumerate(ref["columns"]):
        xr = ref["x"][:, k].astype(np.complex128)
        assert np.linalg.norm(x[:, c] - xr) <= 1e-6 * np.linalg.norm(xr), c
    # every column against the direct solution on the stored sample of unknowns
    rows, xs = ref["sample_rows"], ref["x_sample"].astype(np.complex128)
    err = np.linalg.norm(x[rows, :] - xs, axis=0) / np.linalg.norm(xs, axis=0)
    assert err.max() <= 1e-6, (err.argmax(), err.max())


def test_autotuner_keeps_its_choice(fe, ctx):
    prob = W.random_small_grid(61, n_max=8, n_pec_boxes=1)
    waves = W.random_waves(12, np.random.default_rng(61))
    st1, x1, _, s1 = _solve(fe, ctx, prob, waves, fe.FE_PREC_DF)
    st2, x2, _, s2 = _solve(fe, ctx, prob, waves, fe.FE_PREC_DF)
    assert st1 == st2 == fe.FE_OK
    assert s1["tuned"] == 1 and s1["tune_ms"] > 0.0     # timed in the first call
    assert s2["tuned"] == 2 and s2["tune_ms"] == 0.0    # cached for the second
    assert (s1["tile_width"], s1["grid_ctas"]) == (s2["tile_width"], s2["grid_ctas"])
    assert s1["tile_width"] in (8, 16)                  # at most the column count rounded up
    np.testing.assert_array_equal(x1, x2)               # same partition: the same arithmetic


def test_aircraft40_matches_the_oracle(fe, ctx):
    prob = W.aircraft_mesh(40, 4)
    waves = W.config4()[1].column(0)
    ref = np.load(GOLDEN / "aircraft40_x.npz")
    st, x, rep, _ = _solve(fe, ctx, prob, waves, fe.FE_PREC_DF)
    assert st == fe.FE_OK and rep[0]["status"] == fe.FE_OK
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps)
    B = fem.rhs(prob, waves, maps=maps)
    assert fem.true_relative_residual(A, x, B).max() <= 1e-8
    xr = ref["x"].astype(np.complex128)
    assert np.linalg.norm(x[:, 0] - xr) <= 1e-6 * np.linalg.norm(xr)


def test_aircraft40_expanded_recurrence_shortens_the_plateau(fe, ctx):
    """On the aircraft, whose residual plateaus for thousands of iterations,
    the FP32-pair solve with p^T A p from its three inner products needs far
    fewer iterations than with the Chronopoulos-Gear recurrence (measured
    10 645 against 19 385), and meets the same bars."""
    prob = W.aircraft_mesh(40, 4)
    waves = W.config4()[1].column(0)
    ref = np.load(GOLDEN / "aircraft40_x.npz")
    _, _, rep_cg, _ = _solve(fe, ctx, prob, waves, fe.FE_PREC_DF)
    st, x, rep, _ = _solve(fe, ctx, prob, waves, fe.FE_PREC_DF, recurrence=fe.FE_RECURRENCE_EXPANDED)
    assert st == fe.FE_OK and rep[0]["status"] == fe.FE_OK
    assert rep[0]["iterations"] <= 0.8 * rep_cg[0]["iterations"], (rep, rep_cg)
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps)
    B = fem.rhs(prob, waves, maps=maps)
    assert fem.true_relative_residual(A, x, B).max() <= 1e-8
    xr = ref["x"].astype(np.complex128)
    assert np.linalg.norm(x[:, 0] - xr) <= 1e-6 * np.linalg.norm(xr)
