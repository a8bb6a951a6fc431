"""GPU parity of the symmetry planes (Section 3.1.3, Eqs. 6a/6b), through the
C ABI: the maps with plane faces (no outer face on a plane), the assembled
values with the held unknowns as identity rows, the right-hand side, solves
against the oracle's direct solution, and the quarter of the full-size
3-wavelength cube against the stored solution of the whole cube."""
from pathlib import Path

import numpy as np
import pytest

from oracle import fem
from paper_0704_2344_gb300 import workloads as W
from test_gpu_parity import _check_maps, _check_values, _solve

pytestmark = pytest.mark.gpu

PEC = 255


def _symmetric_box():
    prob = W.empty_box((10, 10, 8), name="sym_full")
    prob.material[3:5, 4:6, 4:6] = PEC
    prob.material[1:3, 2:8, 2:8] = 1                      # a lossy dielectric layer, also centred
    prob.eps_r = np.array([1.0 + 0j, 2.2 - 0.3j])
    prob.mu_r = np.array([1.0 + 0j, 1.0 + 0j])
    return prob


PARTS = {"x_anti": (2, 0), "y_sym": (0, 1), "quarter": (2, 1)}


@pytest.mark.parametrize("part", list(PARTS))
def test_maps_and_values_with_planes(fe, ctx, part):
    prob = W.mirror_part(_symmetric_box(), *PARTS[part])
    _check_maps(fe, ctx, prob)
    _check_values(fe, ctx, prob)


@pytest.mark.parametrize("precision", ["DF", "FP64"])
@pytest.mark.parametrize("part", list(PARTS))
def test_solve_with_planes_matches_oracle(fe, ctx, part, precision):
    prob = W.mirror_part(_symmetric_box(), *PARTS[part])
    waves = W.normal_incidence()
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps)
    B = fem.rhs(prob, waves, maps=maps)
    m = fe.fe_mesh_create_from(ctx, prob)
    try:
        s = fe.fe_assemble(ctx, m, prob.freq_hz, getattr(fe, f"FE_PREC_{precision}"))
        try:
            b_gpu = fe.fe_rhs(ctx, s, waves, maps.n_dof)
        finally:
            fe.fe_system_destroy(s)
    finally:
        fe.fe_mesh_destroy(m)
    assert np.abs(b_gpu - B).max() <= 1e-11 * np.abs(B).max()
    assert np.all(b_gpu[maps.fixed] == 0)
    x, rep = _solve(fe, ctx, prob, waves, getattr(fe, f"FE_PREC_{precision}"))
    assert rep[0]["status"] == 0
    assert fem.true_relative_residual(A, x, B).max() <= 1e-8
    xref = fem.solve_direct(A, B)
    assert np.linalg.norm(x - xref) <= 1e-6 * np.linalg.norm(xref)
    assert np.all(x[maps.fixed] == 0)


def test_plane_faces_accept_pec_and_absorbing_faces_do_not(fe, ctx):
    part = W.mirror_part(_symmetric_box(), 2, 0)
    assert np.any(np.asarray(part.material)[:, :, 0] == PEC)
    m = fe.fe_mesh_create_from(ctx, part)
    fe.fe_mesh_destroy(m)
    part.boundary = (0,) * 6
    with pytest.raises(fe.FeError) as e:
        fe.fe_mesh_create_from(ctx, part)
    assert e.value.status == fe.FE_ERR_MESH
    part.boundary = (3, 0, 0, 0, 0, 0)
    with pytest.raises(fe.FeError) as e:
        fe.fe_mesh_create_from(ctx, part)
    assert e.value.status == fe.FE_ERR_INVALID_ARG


def test_config2_quarter_matches_the_whole_cube(fe, ctx):
    """The +x, +y quarter of the 3-wavelength cube (x = mid an antisymmetry,
    y = mid a symmetry plane) in the FP32-pair mode: its field equals the
    stored SuperLU solution of the whole cube on the quarter's nodes to 1e-6,
    with a quarter of the unknowns."""
    full, waves = W.config2()
    quarter, _ = W.config2_quarter()
    fmaps = fem.mesh_maps(full)
    qmaps = fem.mesh_maps(quarter)
    ref = np.load(Path(__file__).with_name("golden") / "config2_x.npz")["x"].astype(np.complex128)[:, 0]
    ids = np.flatnonzero(qmaps.node_active)
    i = ids % (quarter.nx + 1)
    j = (ids // (quarter.nx + 1)) % (quarter.ny + 1)
    k = ids // ((quarter.nx + 1) * (quarter.ny + 1))
    fid = (i + full.nx // 2) + (full.nx + 1) * ((j + full.ny // 2) + (full.ny + 1) * k)
    xref = ref.reshape(-1, 3)[fmaps.node_rank[fid]].reshape(-1)
    x, rep = _solve(fe, ctx, quarter, waves, fe.FE_PREC_DF)
    assert rep[0]["status"] == 0
    assert qmaps.n_dof < 0.3 * fmaps.n_dof
    A = fem.assemble(quarter, maps=qmaps)
    B = fem.rhs(quarter, waves, maps=qmaps)
    assert fem.true_relative_residual(A, x, B).max() <= 1e-8
    assert np.linalg.norm(x[:, 0] - xref) <= 1e-6 * np.linalg.norm(xref)
