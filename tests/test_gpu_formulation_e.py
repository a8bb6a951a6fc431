"""GPU parity of the E-field formulation (a context with
FE_FORMULATION_E): assembled values (material roles exchanged, tangential E
held on PEC surfaces), right-hand sides and solves against the oracle's E
formulation, and the PEC standing wave."""
import numpy as np
import pytest

from oracle import fem
from paper_0704_2344_gb300 import workloads as W
from test_gpu_parity import _check_values
from test_oracle_formulation_e import _column

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ectx(fe):
    import torch
    c = fe.fe_ctx_create(0, formulation=fe.FE_FORMULATION_E)
    yield c
    fe.fe_ctx_synchronize(c)
    fe.fe_ctx_destroy(c)
    torch.cuda.synchronize()


def _solve(fe, ctx, prob, waves, precision):
    m = fe.fe_mesh_create_from(ctx, prob)
    try:
        s = fe.fe_assemble(ctx, m, prob.freq_hz, precision)
        try:
            n_dof = fe.fe_mesh_info(m)["n_dof"]
            b = fe.fe_rhs(ctx, s, waves, n_dof)
            _, x, rep = fe.fe_solve_batch(ctx, s, waves, n_dof, fe.solve_opts(precision=precision))
        finally:
            fe.fe_system_destroy(s)
    finally:
        fe.fe_mesh_destroy(m)
    return b, x, rep


@pytest.mark.parametrize("seed", [2, 5, 9])
def test_e_values(fe, ectx, seed):
    prob = W.random_small_grid(seed, n_max=7, n_pec_boxes=2)
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps, formulation="E")
    assert fem.held_dofs(prob, maps, "E").any() or not (np.asarray(prob.material) == 255).any()
    _check_values(fe, ectx, prob, A=A, maps=maps)


@pytest.mark.parametrize("precision", ["DF", "FP64", "MIXED"])
@pytest.mark.parametrize("seed", [2, 9])
def test_e_solve_matches_oracle(fe, ectx, seed, precision):
    prob = W.random_small_grid(seed, n_max=7, n_pec_boxes=2)
    waves = W.random_waves(3, np.random.default_rng(seed))
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps, formulation="E")
    B = fem.rhs(prob, waves, maps=maps, formulation="E")
    b, x, rep = _solve(fe, ectx, prob, waves, getattr(fe, f"FE_PREC_{precision}"))
    assert np.abs(b - B).max() <= 1e-11 * np.abs(B).max()
    assert all(r["status"] == 0 for r in rep)
    assert fem.true_relative_residual(A, x, B).max() <= 1e-8
    xref = fem.solve_direct(A, B)
    assert np.linalg.norm(x - xref) <= 1e-6 * np.linalg.norm(xref)
    assert np.all(x[fem.held_dofs(prob, maps, "E")] == 0)


def test_e_pec_standing_wave(fe, ectx):
    prob, waves = _column(40, "E")
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps, formulation="E")
    B = fem.rhs(prob, waves, maps=maps, formulation="E")
    _, x, rep = _solve(fe, ectx, prob, waves, fe.FE_PREC_DF)
    xref = fem.solve_direct(A, B)
    assert rep[0]["status"] == 0
    assert np.linalg.norm(x - xref) <= 1e-6 * np.linalg.norm(xref)
    k0 = fem.wavenumber(prob.freq_hz)
    z = fem.node_positions(prob, maps)[:, 2]
    exact = np.exp(1j * k0 * z) - np.exp(1j * k0 * (2 * prob.h[2] - z))
    assert np.linalg.norm(x.reshape(-1, 3)[:, 0] - exact) <= 0.01 * np.linalg.norm(exact)
