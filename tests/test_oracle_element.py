"""Pins of the oracle's element and face matrices (CPU only).

The oracle integrates Eq. 1 + Eq. 2 and the face forms of Eqs. 3-4 by Gauss
quadrature with explicit curls and divergences.  These tests pin it to facts
that do not come from the oracle itself: symmetry, null spaces, an
independently written Kronecker-product closed form, textbook Q1 values on a
unit cube (tests/golden/unit_cube_q1.txt) and passivity."""
import numpy as np
import pytest

from oracle import fem

H = (0.011, 0.009, 0.013)
K0 = fem.wavenumber(3e9)


def _local(a):
    return (a & 1, (a >> 1) & 1, (a >> 2) & 1)


def kron_closed_form(h, eps, mu, k0, s):
    """Second derivation: 1-D matrices M1 = h/6[[2,1],[1,2]], K1 = 1/h[[1,-1],[-1,1]],
    D1[p][q] = int phi_p' phi_q = [[-1/2,-1/2],[1/2,1/2]]; C^{gd}_ab =
    int d_g N_a d_d N_b is a product of one factor per axis."""
    M1 = [np.array([[2, 1], [1, 2]]) * hh / 6 for hh in h]
    K1 = [np.array([[1, -1], [-1, 1]]) / hh for hh in h]
    D1 = np.array([[-0.5, -0.5], [0.5, 0.5]])

    def C(g, d, a, b):
        la, lb = _local(a), _local(b)
        v = 1.0
        for t in range(3):
            if g == d == t:
                v *= K1[t][la[t], lb[t]]
            elif t == g:
                v *= D1[la[t], lb[t]]
            elif t == d:
                v *= D1[lb[t], la[t]]
            else:
                v *= M1[t][la[t], lb[t]]
        return v

    A = np.zeros((24, 24), complex)
    for a in range(8):
        for b in range(8):
            G = sum(C(g, g, a, b) for g in range(3))
            M = np.prod([M1[t][_local(a)[t], _local(b)[t]] for t in range(3)])
            for al in range(3):
                for be in range(3):
                    v = (1 / eps) * ((al == be) * G - C(be, al, a, b)) + s * C(al, be, a, b)
                    if al == be:
                        v -= k0 ** 2 * mu * M
                    A[3 * a + al, 3 * b + be] = v
    return A


def test_element_matrix_is_symmetric():
    A = fem.element_matrix(H, 2.5 - 0.3j, 1.2 - 0.1j, K0, 1.0)
    assert np.abs(A - A.T).max() <= 1e-15 * np.abs(A).max()


def test_element_matrix_matches_kronecker_closed_form():
    for eps, mu, s in [(1.0, 1.0, 1.0), (4.0, 1.0, 1.0), (2.5 - 0.3j, 1.2 - 0.1j, 0.7)]:
        A = fem.element_matrix(H, eps, mu, K0, s)
        B = kron_closed_form(H, eps, mu, K0, s)
        assert np.abs(A - B).max() <= 1e-14 * np.abs(B).max()


def test_stiffness_null_space_constant_and_harmonic_fields():
    # k0 = 0 leaves curl-curl + grad-div; a constant field and the harmonic
    # linear field H = (x, -y, 0) (curl = 0, div = 0) carry zero energy.
    A = fem.element_matrix(H, 1.0, 1.0, 0.0, 1.0).real
    pts = np.array([np.array(_local(a)) * H for a in range(8)])
    fields = [np.tile(c, 8) for c in np.eye(3)]
    fields.append(np.stack([pts[:, 0], -pts[:, 1], np.zeros(8)], axis=1).ravel())
    fields.append(np.stack([pts[:, 1], pts[:, 0], np.zeros(8)], axis=1).ravel())  # grad(xy)
    for u in fields:
        assert np.abs(A @ u).max() <= 1e-12 * np.abs(A).max() * np.abs(u).max()
    # a field with curl (H = (y, 0, 0)) has positive energy
    u = np.stack([pts[:, 1], np.zeros(8), np.zeros(8)], axis=1).ravel()
    assert u @ A @ u > 1e-3 * np.abs(A).max() * np.abs(u).max() ** 2


def test_unit_cube_textbook_values(tmp_path):
    """Q1 mass and Laplacian entries of the unit cube (golden file)."""
    from pathlib import Path
    gold = {}
    for line in Path(__file__).with_name("golden").joinpath("unit_cube_q1.txt").read_text().splitlines():
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            num, den = v.strip().split("/")
            gold[k.strip()] = float(num) / float(den)
    h = (1.0, 1.0, 1.0)
    M = -fem.element_matrix(h, 1.0, 1.0, 1.0, 0.0).real + fem.element_matrix(h, 1.0, 1.0, 0.0, 0.0).real
    K = fem.element_matrix(h, 1.0, 1.0, 0.0, 1.0).real  # vector Laplacian weak form (s = 1, eps = 1)
    pairs = {"self": (0, 0), "edge": (0, 1), "face_diag": (0, 3), "body_diag": (0, 7)}
    for name, (a, b) in pairs.items():
        assert M[3 * a, 3 * b] == pytest.approx(gold[f"mass_{name}"], rel=1e-14)
        assert M[3 * a, 3 * b + 1] == 0.0
    # x-x entry of curl-curl + grad-div with eps = 1, s = 1 is the Q1 Laplacian
    for name, (a, b) in pairs.items():
        assert K[3 * a, 3 * b] == pytest.approx(gold[f"laplace_{name}"], rel=1e-13, abs=1e-15)


def test_face_matrices():
    for f in range(6):
        G = fem.face_abc_matrix(H, f, K0, -1.0)
        assert np.abs(G - G.T).max() <= 1e-15 * np.abs(G).max()
        axis, side = f // 2, f % 2
        for a in range(8):
            for al in range(3):
                row = G[3 * a + al]
                if _local(a)[axis] != side or al == axis:
                    assert np.all(row == 0)  # only tangential components of face nodes
        # the j k0 part integrates W_t . H_t over the face: total = k0 * area per component
        area = np.prod([H[t] for t in range(3) if t != axis])
        G0 = fem.face_abc_matrix(H, f, K0, 0.0)
        tang = [t for t in range(3) if t != axis]
        ones = np.zeros(24)
        ones[[3 * a + tang[0] for a in range(8)]] = 1.0
        assert (ones @ G0 @ ones).imag == pytest.approx(K0 * area, rel=1e-14)
        # penalty term: -s int (W.n)(div H); for H = (x, 0, 0) (div = 1) and W = e_axis const
        Lp = fem.face_penalty_matrix(H, f, 1.0)
        pts = np.array([np.array(_local(a)) * H for a in range(8)])
        u = np.stack([pts[:, 0], np.zeros(8), np.zeros(8)], axis=1).ravel()
        w = np.zeros(24)
        w[[3 * a + axis for a in range(8)]] = 1.0
        expect = -(1.0 if side else -1.0) * area
        assert w @ Lp @ u == pytest.approx(expect, rel=1e-13)


def test_passivity_of_absorbing_boundary_and_losses():
    # e^{j omega t}: lossy eps'' > 0 is eps = eps' - j eps''; the first-order
    # ABC j k0 H_t radiates: Im(x^H A x) >= 0 for every x.
    from paper_0704_2344_gb300 import workloads as W
    prob = W.random_small_grid(11, n_max=4)
    A = fem.assemble(prob, sigma=0.0).toarray()
    rng = np.random.default_rng(5)
    for _ in range(20):
        x = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
        assert (x.conj() @ A @ x).imag >= -1e-12 * np.abs(A).max() * (np.abs(x) ** 2).sum()
