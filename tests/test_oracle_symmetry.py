"""Pins of the symmetry planes (Section 3.1.3, Eqs. 6a and 6b) in the oracle.

A box that is mirror-symmetric about its mid planes, lit at normal
incidence (k = z, H along x), has a total field whose x component is even
and whose y, z components are odd across x = mid (so n x H = 0 there, an
antisymmetry plane) and whose y component is odd across y = mid (n . H = 0,
a symmetry plane).  Solving only the half or the quarter with those face
kinds must reproduce the full solution on the shared nodes to rounding: the
discrete problems coincide.  A wrong kind must not."""
import numpy as np
import pytest

from oracle import fem
from paper_0704_2344_gb300 import workloads as W

PEC = 255


def _full():
    prob = W.empty_box((10, 10, 8), name="sym_full")
    prob.material[3:5, 4:6, 4:6] = PEC          # centred in x and y: nodes 4..6 around node 5
    return prob, W.normal_incidence()


def _solve(prob, waves):
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps)
    B = fem.rhs(prob, waves, maps=maps)
    return maps, fem.solve_direct(A, B)[:, 0], A, B


def _on_part(full, fmaps, xfull, part, pmaps, x0, y0):
    """The full solution at the part's active nodes, in the part's rank order."""
    ids = np.flatnonzero(pmaps.node_active)
    i = ids % (part.nx + 1)
    j = (ids // (part.nx + 1)) % (part.ny + 1)
    k = ids // ((part.nx + 1) * (part.ny + 1))
    fid = (i + x0) + (full.nx + 1) * ((j + y0) + (full.ny + 1) * k)
    r = fmaps.node_rank[fid]
    assert np.all(r >= 0)
    return xfull.reshape(-1, 3)[r].reshape(-1)


@pytest.mark.parametrize("x_kind,y_kind", [(2, 0), (0, 1), (2, 1)])
def test_planes_reproduce_the_full_solution(x_kind, y_kind):
    full, waves = _full()
    fmaps, xf, _, _ = _solve(full, waves)
    part = W.mirror_part(full, x_kind=x_kind, y_kind=y_kind)
    pmaps, xp, A, B = _solve(part, waves)
    assert fem.true_relative_residual(A, xp[:, None], B).max() <= 1e-12
    ref = _on_part(full, fmaps, xf, part, pmaps, full.nx // 2 if x_kind else 0, full.ny // 2 if y_kind else 0)
    scale = np.abs(xf).max()
    # the constrained components vanish in the full solution too (mirror symmetry)
    assert np.abs(ref[pmaps.fixed]).max() <= 1e-10 * scale
    assert np.abs(xp - ref).max() <= 1e-10 * scale


def test_a_wrong_plane_kind_does_not_match():
    full, waves = _full()
    fmaps, xf, _, _ = _solve(full, waves)
    part = W.mirror_part(full, x_kind=1)     # x = mid is an antisymmetry plane for this incidence
    pmaps, xp, _, _ = _solve(part, waves)
    ref = _on_part(full, fmaps, xf, part, pmaps, full.nx // 2, 0)
    assert np.abs(xp - ref).max() > 1e-2 * np.abs(xf).max()


def test_plane_faces_carry_no_surface_terms_and_may_cut_the_scatterer():
    full, _ = _full()
    part = W.mirror_part(full, x_kind=2, y_kind=1)
    maps = fem.mesh_maps(part)
    faces = maps.faces_ext
    f = faces % 6
    e = faces // 6
    i = e % part.nx
    j = (e // part.nx) % part.ny
    # no outer face on the two plane sides (-x, -y); the PEC block touches them
    assert not np.any((f == 0) & (i == 0)) and not np.any((f == 2) & (j == 0))
    assert np.any(np.asarray(part.material)[:, :, 0] == PEC)
    fem.validate(part)   # accepted although PEC touches the plane faces
    bad = W.mirror_part(full, x_kind=2)
    bad.boundary = (0,) * 6       # the same cut as an absorbing face: PEC on the outer box
    with pytest.raises(ValueError):
        fem.validate(bad)


def test_a_mesh_without_active_elements_is_rejected():
    prob = W.empty_box(3, name="all_pec")
    prob.material[:] = PEC
    prob.boundary = (1, 1, 2, 2, 1, 1)
    with pytest.raises(ValueError):
        fem.validate(prob)
