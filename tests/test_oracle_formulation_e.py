"""Pins of the E-field formulation (Section 2: the steps of the H formulation
applied to E; Section 3.1.3: n x E = 0 held on conductors) and of the PEC
treatment of both formulations.

The one-dimensional standing wave: a column one element wide with symmetry
planes on its four sides (so the field depends on z only), a PEC floor at
z0, the absorbing face on top, and a wave falling along -z.  The continuous
total fields are E_x = e^{j k0 z} - e^{j k0 (2 z0 - z)} (tangential E vanishes
on the conductor) and H_y = e^{j k0 z} + e^{j k0 (2 z0 - z)} (tangential H
doubles there).  Both discrete solutions converge to them at second order."""
import numpy as np
import pytest

from oracle import fem
from paper_0704_2344_gb300 import workloads as W

PEC = 255


def _column(per, formulation):
    """1 x 1 x (per + 1) elements of lambda / per, the bottom layer PEC."""
    p = W.empty_box((1, 1, per + 1), 3e9, per, name=f"col{per}")
    p.material[0] = PEC
    # field along x (E) or y (H): the faces normal to the field hold the
    # tangential components (n x F = 0), the others the normal one (n . F = 0)
    p.boundary = (2, 2, 1, 1, 1, 0) if formulation == "E" else (1, 1, 2, 2, 1, 0)
    waves = W.PlaneWaves(np.array([[0.0, 0.0, -1.0]]),
                         np.array([[1.0, 0.0, 0.0]]) if formulation == "E" else np.array([[0.0, 1.0, 0.0]]))
    return p, waves


def _standing_wave_error(per, formulation):
    p, waves = _column(per, formulation)
    m = fem.mesh_maps(p)
    A = fem.assemble(p, maps=m, formulation=formulation)
    B = fem.rhs(p, waves, maps=m, formulation=formulation)
    x = fem.solve_direct(A, B)[:, 0].reshape(-1, 3)
    k0 = fem.wavenumber(p.freq_hz)
    z = fem.node_positions(p, m)[:, 2]
    z0 = p.h[2]
    sign = -1.0 if formulation == "E" else 1.0
    exact = np.exp(1j * k0 * z) + sign * np.exp(1j * k0 * (2 * z0 - z))
    comp = 0 if formulation == "E" else 1
    held = fem.held_dofs(p, m, formulation).reshape(-1, 3)
    assert held[:, [c for c in range(3) if c != comp]].all()   # the other components are held everywhere
    if formulation == "E":
        assert np.all(x[np.isclose(z, z0), comp] == 0)        # n x E = 0 on the conductor, exactly
    return np.linalg.norm(x[:, comp] - exact) / np.linalg.norm(exact)


@pytest.mark.parametrize("formulation", ["E", "H"])
def test_pec_standing_wave_converges_second_order(formulation):
    errs = [_standing_wave_error(per, formulation) for per in (10, 20, 40)]
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 0.01, errs
    assert np.all(np.abs(slopes - 2.0) <= 0.25), (errs, slopes)


def test_e_plane_wave_in_an_empty_box_converges_second_order():
    k = np.array([np.sin(0.5) * np.cos(0.3), np.sin(0.5) * np.sin(0.3), np.cos(0.5)])
    t = np.array([np.cos(0.5) * np.cos(0.3), np.cos(0.5) * np.sin(0.3), -np.sin(0.5)])
    errs = []
    for per in (10, 20, 40):
        n_t = max(2, int(round(0.2 * per)))
        p = W.empty_box((n_t, n_t, per), 3e9, per)
        wv = W.PlaneWaves(np.array([k]), np.array([t]))
        m = fem.mesh_maps(p)
        A = fem.assemble(p, maps=m, formulation="E")
        x = fem.solve_direct(A, fem.rhs(p, wv, maps=m, formulation="E"))
        ex = fem.plane_wave_at_nodes(p, m, wv)
        errs.append(np.linalg.norm(x - ex) / np.linalg.norm(ex))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert abs(slopes[-1] - 2.0) <= 0.25, (errs, slopes)


def test_without_conductors_e_is_h_with_the_materials_exchanged():
    p = W.random_small_grid(3, n_max=5, n_pec_boxes=0)
    q = W.random_small_grid(3, n_max=5, n_pec_boxes=0)
    q.eps_r, q.mu_r = p.mu_r.copy(), p.eps_r.copy()
    a_e = fem.assemble(p, formulation="E")
    a_h = fem.assemble(q)
    assert abs(a_e - a_h).max() == 0.0


def test_e_holds_tangential_components_on_conductor_surfaces_only():
    p = W.empty_box((6, 6, 6), name="box")
    p.material[2:4, 2:4, 2:4] = PEC
    m = fem.mesh_maps(p)
    held = fem.held_dofs(p, m, "E").reshape(-1, 3)
    assert not fem.held_dofs(p, m, "H").any()
    ids = np.flatnonzero(m.node_active)
    i, j, k = ids % 7, (ids // 7) % 7, ids // 49
    on = (i >= 2) & (i <= 4) & (j >= 2) & (j <= 4) & (k >= 2) & (k <= 4)   # nodes of the PEC block's surface
    assert not held[~on].any()
    face_x = on & (i == 2) & (j == 3) & (k == 3)                           # centre of the -x face
    assert list(held[face_x][0]) == [False, True, True]
    corner = on & (i == 2) & (j == 2) & (k == 2)
    assert held[corner].all()
