"""Pins of the oracle's assembled system, right-hand side and solvers (CPU).

* integer maps against a pure-Python brute force on tiny grids;
* the assembled interior stencil against its closed form (the Q1 27-point
  Laplacian-Helmholtz stencil; cross-component blocks vanish at interior nodes
  because d_a u d_b v - d_b u d_a v integrates to a boundary term);
* the empty-box plane wave: the incident wave solves the continuous weak
  problem of Eq. 4 exactly at any incidence (the scattered field is zero and
  G(W, H) cancels G(W, H_i)), so the nodal error must fall as O(h^2);
* brute force: dense LAPACK vs sparse LU vs the CPU COCG on tiny systems;
* mirror symmetry of the field for a mirror-symmetric scatterer.
"""
import numpy as np
import pytest

from oracle import fem, krylov
from paper_0704_2344_gb300 import workloads as W


def brute_maps(prob):
    nx, ny, nz = prob.nx, prob.ny, prob.nz
    mat = prob.material.reshape(nz, ny, nx)

    def active(i, j, k):
        return 0 <= i < nx and 0 <= j < ny and 0 <= k < nz and mat[k, j, i] != fem.PEC

    rank = {}
    order = []
    for k in range(nz + 1):
        for j in range(ny + 1):
            for i in range(nx + 1):
                if any(active(i - 1 + a, j - 1 + b, k - 1 + c) for a in (0, 1) for b in (0, 1) for c in (0, 1)):
                    rank[(i, j, k)] = len(order)
                    order.append((i, j, k))
    rows = []
    for (i, j, k) in order:
        nb = set()
        for (ei, ej, ek) in [(i - 1 + a, j - 1 + b, k - 1 + c) for a in (0, 1) for b in (0, 1) for c in (0, 1)]:
            if active(ei, ej, ek):
                for a in range(8):
                    nb.add(rank[(ei + (a & 1), ej + ((a >> 1) & 1), ek + ((a >> 2) & 1))])
        rows.append(sorted(nb))
    row_ptr = np.cumsum([0] + [len(r) for r in rows])
    col_idx = np.concatenate(rows)
    node_rank = np.full((nx + 1) * (ny + 1) * (nz + 1), -1)
    for (i, j, k), r in rank.items():
        node_rank[i + (nx + 1) * (j + (ny + 1) * k)] = r
    slot = np.full((nx * ny * nz, 8, 8), -1)
    ext, pec = [], []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                e = i + nx * (j + ny * k)
                if not active(i, j, k):
                    continue
                nodes = [(i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1)) for a in range(8)]
                for a in range(8):
                    ra = rank[nodes[a]]
                    for b in range(8):
                        slot[e, a, b] = row_ptr[ra] + rows[ra].index(rank[nodes[b]])
                c = (i, j, k)
                dims = (nx, ny, nz)
                for f in range(6):
                    ax, side = f // 2, f % 2
                    n = list(c)
                    n[ax] += 1 if side else -1
                    if n[ax] < 0 or n[ax] >= dims[ax]:
                        ext.append(6 * e + f)
                    elif mat[n[2], n[1], n[0]] == fem.PEC:
                        pec.append(6 * e + f)
    return node_rank, row_ptr, col_idx, slot, np.array(sorted(ext)), np.array(sorted(pec))


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5, 6])
def test_maps_match_brute_force(seed):
    prob = W.random_small_grid(seed, n_max=5, n_pec_boxes=2)
    m = fem.mesh_maps(prob)
    nr, rp, ci, sl, ext, pec = brute_maps(prob)
    assert np.array_equal(m.node_rank, nr)
    assert np.array_equal(m.row_ptr, rp)
    assert np.array_equal(m.col_idx, ci)
    assert np.array_equal(m.elem_slot, sl)
    assert np.array_equal(m.faces_ext, ext)
    assert np.array_equal(m.faces_pec, pec)


def test_config_counts():
    # 30^3 elements with a 6^3 PEC cube: 26 784 active elements, 29 666 active
    # nodes (the 5^3 nodes inside the cube drop out), 5 400 outer and 216 PEC faces.
    prob, _ = W.config2()
    m = fem.mesh_maps(prob)
    assert int(m.elem_active.sum()) == 26784
    assert m.n_act == 29666
    assert m.faces_ext.size == 5400 and m.faces_pec.size == 216
    assert m.nnzb == 748658
    # constant bandwidth of the node-numbered matrix (Section 3.1.2)
    rows = np.repeat(np.arange(m.n_act), np.diff(m.row_ptr))
    assert np.diff(m.row_ptr).max() == 27
    ids = np.flatnonzero(m.node_active)
    assert np.abs(ids[m.col_idx] - ids[rows]).max() == 31 * 31 + 31 + 1


def test_interior_stencil_closed_form():
    p = W.empty_box(4)
    m = fem.mesh_maps(p)
    vals = fem.to_bsr_values(fem.assemble(p, maps=m), m)
    h = p.h[0]
    kh2 = (fem.wavenumber(p.freq_hz) * h) ** 2
    expect = {0: 8 / 3 - kh2 * 8 / 27, 1: -kh2 * 2 / 27, 2: -1 / 6 - kh2 / 54, 3: -1 / 12 - kh2 / 216}
    nid = 2 + 5 * (2 + 5 * 2)
    r = m.node_rank[nid]
    ids = np.flatnonzero(m.node_active)
    assert m.row_ptr[r + 1] - m.row_ptr[r] == 27
    for s in range(m.row_ptr[r], m.row_ptr[r + 1]):
        c = ids[m.col_idx[s]]
        dist = abs(c % 5 - 2) + abs((c // 5) % 5 - 2) + abs(c // 25 - 2)
        blk = vals[s] / h
        assert np.abs(blk - expect[dist] * np.eye(3)).max() <= 1e-13
    assert 8 / 3 - kh2 * 8 / 27 == pytest.approx(2.5496935774685703, rel=1e-15)


def _empty_box_error(per, k_hat, p_hat, trans=0.2):
    n_t = max(2, int(round(trans * per)))
    p = W.empty_box((n_t, n_t, per), 3e9, per)
    wv = W.PlaneWaves(np.array([k_hat]), np.array([p_hat]))
    m = fem.mesh_maps(p)
    A = fem.assemble(p, maps=m)
    X = fem.solve_direct(A, fem.rhs(p, wv, maps=m))
    ex = fem.plane_wave_at_nodes(p, m, wv)
    return np.linalg.norm(X - ex) / np.linalg.norm(ex)


@pytest.mark.slow
@pytest.mark.parametrize("theta,phi", [(0.0, 0.0), (0.5, 0.3), (1.0, 2.0)])
def test_empty_box_plane_wave_converges_second_order(theta, phi):
    k = np.array([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)])
    t = np.array([np.cos(theta) * np.cos(phi), np.cos(theta) * np.sin(phi), -np.sin(theta)])
    errs = [_empty_box_error(per, k, t) for per in (10, 20, 40)]
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 0.01
    assert abs(slopes[-1] - 2.0) <= 0.2, (errs, slopes)
    assert abs(slopes[0] - 2.0) <= 0.35, (errs, slopes)


def test_brute_force_2x2x2_dense_sparse_cocg():
    p = W.empty_box(2)  # every element touches the outer box, so all are vacuum
    wv = W.oblique_wave(0.7, 0.4)
    m = fem.mesh_maps(p)
    assert m.n_act == 27 and m.n_dof == 81 and m.nnzb == 343
    A = fem.assemble(p, maps=m)
    B = fem.rhs(p, wv, maps=m)
    xd = np.linalg.solve(A.toarray(), B)
    import scipy.sparse.linalg as spla
    xs = spla.splu(A.tocsc()).solve(B)
    assert np.linalg.norm(xd - xs) <= 1e-12 * np.linalg.norm(xd)
    xc, it, _ = krylov.cocg(A, B[:, 0], tol=1e-13)
    assert np.linalg.norm(xc - xd[:, 0]) <= 1e-10 * np.linalg.norm(xd)
    assert np.abs(A - A.T).max() <= 1e-15 * np.abs(A).max()


def test_variants_literal_and_symmetrised():
    prob = W.random_small_grid(3, n_max=4)
    AL = fem.assemble(prob, variant="L")
    AP = fem.assemble(prob, variant="P")
    AS = fem.assemble(prob, variant="S")
    assert np.abs((AP - AP.T)).max() <= 1e-15 * np.abs(AP).max()
    assert np.abs((AS - AS.T)).max() <= 1e-15 * np.abs(AS).max()
    assert np.abs((AL - AL.T)).max() > 1e-3 * np.abs(AL).max()  # literal Eq. 4 is not symmetric
    assert np.abs(AP - 0.5 * (AL + AL.T)).max() <= 1e-15 * np.abs(AL).max()


def test_mirror_symmetry_of_the_field():
    # centred PEC cube, k_hat = z, H_i = x: H(x,y,z) = P_y H(x,-y,z) (Hx, Hz even,
    # Hy odd in y) and H = -P_x H(-x,y,z) (Hx even, Hy, Hz odd in x).
    p = W.empty_box(8)
    p.material[3:5, 3:5, 3:5] = fem.PEC
    wv = W.normal_incidence()
    m = fem.mesh_maps(p)
    X = fem.solve_direct(fem.assemble(p, maps=m), fem.rhs(p, wv, maps=m))[:, 0].reshape(-1, 3)
    n = 9
    full = np.zeros((n, n, n, 3), complex)
    ids = np.flatnonzero(m.node_active)
    full.reshape(-1, 3)[ids] = X
    scale = np.abs(X).max()
    fy = full[:, ::-1, :, :]
    assert np.abs(full[..., 0] - fy[..., 0]).max() <= 1e-10 * scale
    assert np.abs(full[..., 1] + fy[..., 1]).max() <= 1e-10 * scale
    assert np.abs(full[..., 2] - fy[..., 2]).max() <= 1e-10 * scale
    fx = full[:, :, ::-1, :]
    assert np.abs(full[..., 0] - fx[..., 0]).max() <= 1e-10 * scale
    assert np.abs(full[..., 1] + fx[..., 1]).max() <= 1e-10 * scale
    assert np.abs(full[..., 2] + fx[..., 2]).max() <= 1e-10 * scale


def test_mesh_rules():
    p = W.empty_box(4)
    p.material[0, 1, 1] = fem.PEC
    with pytest.raises(ValueError):
        fem.assemble(p)
    p = W.empty_box(4)
    p.eps_r = np.array([1.0 + 0j, 2.0 + 0j])
    p.mu_r = np.array([1.0 + 0j, 1.0 + 0j])
    p.material[0, 0, 0] = 1
    with pytest.raises(ValueError):
        fem.assemble(p)


def _centred_quarter(c, margin, kind):
    """A cube of c elements (eps_r = 4 dielectric or PEC) centred in a box of
    c + 2 margin elements at lambda/10, the box centred on the origin, reduced
    to its +x, +y quarter by the mirror planes of normal incidence (H along x:
    x = 0 is an antisymmetry plane, y = 0 a symmetry plane)."""
    n = c + 2 * margin
    prob = W.empty_box(n, 3e9, 10.0, name=f"{kind}{c}_m{margin}")
    h = prob.h[0]
    prob.origin = (-n / 2 * h, -n / 2 * h, -n / 2 * h)
    if kind == "pec":
        prob.material[margin:margin + c, margin:margin + c, margin:margin + c] = W.PEC
    else:
        prob.material[margin:margin + c, margin:margin + c, margin:margin + c] = 1
        prob.eps_r = np.array([1.0 + 0j, 4.0 + 0j])
        prob.mu_r = np.array([1.0 + 0j, 1.0 + 0j])
    return W.mirror_part(prob, x_kind=2, y_kind=1)


def _box_size_difference(c, m_small, m_big, sigma, kind, rim):
    """Relative difference of the fields of two box sizes on the small box's
    nodes at least `rim` elements inside its absorbing faces (Eq. 3 with
    transverse-term sign sigma)."""
    waves = W.normal_incidence()
    out = []
    for m in (m_small, m_big):
        prob = _centred_quarter(c, m, kind)
        maps = fem.mesh_maps(prob)
        A = fem.assemble(prob, maps=maps, sigma=sigma)
        B = fem.rhs(prob, waves, maps=maps, sigma=sigma)
        x = fem.solve_direct(A, B)[:, 0].reshape(-1, 3)
        pos = np.round(fem.node_positions(prob, maps) / prob.h[0]).astype(np.int64)
        out.append((pos, x))
    (ps, xs), (pb, xb) = out
    index = {tuple(p): i for i, p in enumerate(pb)}
    xb = xb[[index[tuple(p)] for p in ps]]
    lim = (c + 2 * m_small) / 2 - rim
    inner = np.all(np.abs(ps) <= lim, axis=1)
    return np.linalg.norm(xs[inner] - xb[inner]) / np.linalg.norm(xb[inner])


@pytest.mark.slow
def test_box_size_accuracy_orders_the_abc_terms():
    """The box-size accuracy study of the absorbing condition (Eq. 3), on the
    oracle: an eps_r = 4 cube of 0.4 wavelength, boxes with 0.4 and 1.2
    wavelengths of margin.  Close to the scatterer the field at the outer
    faces has strong evanescent content: the first-order condition (sigma = 0)
    differs least from the larger box, the transverse term as printed (sigma
    = +1, which damps evanescent modes a little more) a little more, and the
    opposite sign (sigma = -1, whose boundary amplifies evanescent modes with
    tangential wavenumbers above sqrt(2) k0) most.  A sign error in the
    oracle's transverse term would swap the last two."""
    d = {s: _box_size_difference(4, 4, 12, s, "diel", 3) for s in (-1.0, 0.0, 1.0)}
    assert d[0.0] < d[1.0] < d[-1.0]
    assert d[-1.0] < 0.3 and d[1.0] < 1.2 * d[0.0]
