"""Edge cases through the C ABI: the smallest mesh (one element, 24
unknowns), a right-hand-side count that is not a tile width (padded with
zero columns), and a mesh without any active element."""
import numpy as np
import pytest

from oracle import fem
from paper_0704_2344_gb300 import workloads as W
from test_gpu_parity import _solve

pytestmark = pytest.mark.gpu

PEC = 255


@pytest.mark.parametrize("precision", ["FP64", "MIXED", "DF"])
def test_one_element(fe, ctx, precision):
    prob = W.empty_box(1, name="one")
    waves = W.random_waves(2, np.random.default_rng(3))
    maps = fem.mesh_maps(prob)
    assert maps.n_dof == 24
    A = fem.assemble(prob, maps=maps)
    B = fem.rhs(prob, waves, maps=maps)
    x, rep = _solve(fe, ctx, prob, waves, getattr(fe, f"FE_PREC_{precision}"))
    assert all(r["status"] == 0 for r in rep)
    xref = fem.solve_direct(A, B)
    assert np.linalg.norm(x - xref) <= 1e-6 * np.linalg.norm(xref)


def test_five_waves_padded_to_a_tile_of_eight(fe, ctx):
    prob = W.random_small_grid(41, n_max=7, n_pec_boxes=1)
    waves = W.random_waves(5, np.random.default_rng(8))
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps)
    B = fem.rhs(prob, waves, maps=maps)
    x, rep = _solve(fe, ctx, prob, waves, fe.FE_PREC_DF)
    assert len(rep) == 5 and all(r["status"] == 0 for r in rep)
    assert fe.fe_last_solve_stats(ctx)["tile_width"] == 8
    assert fem.true_relative_residual(A, x, B).max() <= 1e-8
    xref = fem.solve_direct(A, B)
    assert np.linalg.norm(x - xref) <= 1e-6 * np.linalg.norm(xref)


def test_no_active_element(fe, ctx):
    prob = W.empty_box(3, name="all_pec")
    prob.material[:] = PEC
    prob.boundary = (1, 1, 2, 2, 1, 1)       # planes only, so PEC may touch every face
    with pytest.raises(ValueError):
        fem.validate(prob)
    with pytest.raises(fe.FeError) as e:
        fe.fe_mesh_create_from(ctx, prob)
    assert e.value.status == fe.FE_ERR_MESH
