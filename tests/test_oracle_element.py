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


# ---------------------------------------------------------------------------
# The transverse term of the absorbing condition (Eq. 3).  Its weak form on a
# face with normal axis nu and tangential axes t1, t2 is
#     sigma (j / 2k0) int sum_g grad_t (W_t)_g . grad_t (H_t)_g ds,
# which for W = N_a e_alpha, H = N_b e_beta is zero unless alpha = beta is
# tangential and both nodes lie on the face, and then equals the 2-D Q1
# stiffness of the face, K1(t1) x M1(t2) + M1(t1) x K1(t2).  The pins below
# build that matrix from the 1-D matrices alone and check exact integrals of
# Q1 fields, so a dropped factor, a flipped sign or a projector that lets the
# normal derivative in fails one of them.
# ---------------------------------------------------------------------------
def _transverse_closed_form(h, face):
    axis, side = face // 2, face % 2
    tang = [t for t in range(3) if t != axis]
    M1 = {t: np.array([[2.0, 1.0], [1.0, 2.0]]) * h[t] / 6.0 for t in tang}
    K1 = {t: np.array([[1.0, -1.0], [-1.0, 1.0]]) / h[t] for t in tang}
    t1, t2 = tang
    T = np.zeros((24, 24))
    for a in range(8):
        la = _local(a)
        if la[axis] != side:
            continue
        for b in range(8):
            lb = _local(b)
            if lb[axis] != side:
                continue
            v = (K1[t1][la[t1], lb[t1]] * M1[t2][la[t2], lb[t2]]
                 + M1[t1][la[t1], lb[t1]] * K1[t2][la[t2], lb[t2]])
            for al in tang:
                T[3 * a + al, 3 * b + al] = v
    return T


def _mass_closed_form(h, face):
    axis, side = face // 2, face % 2
    tang = [t for t in range(3) if t != axis]
    M1 = {t: np.array([[2.0, 1.0], [1.0, 2.0]]) * h[t] / 6.0 for t in tang}
    T = np.zeros((24, 24))
    for a in range(8):
        la = _local(a)
        for b in range(8):
            lb = _local(b)
            if la[axis] != side or lb[axis] != side:
                continue
            for al in tang:
                T[3 * a + al, 3 * b + al] = M1[tang[0]][la[tang[0]], lb[tang[0]]] * M1[tang[1]][la[tang[1]], lb[tang[1]]]
    return T


@pytest.mark.parametrize("h", [H, (0.004, 0.017, 0.010), (0.02, 0.02, 0.005)])
def test_abc_transverse_term_closed_form(h):
    """Every entry of the face form G = j k0 int W_t.H_t + sigma (j/2k0) int
    grad_t W : grad_t H against the Kronecker form built from the 1-D
    matrices, on all six faces, anisotropic bricks, three values of sigma."""
    for f in range(6):
        T = _transverse_closed_form(h, f)
        Mt = _mass_closed_form(h, f)
        for sigma in (1.0, -1.0, 0.5):
            G = fem.face_abc_matrix(h, f, K0, sigma)
            expect = 1j * K0 * Mt + sigma * (1j / (2.0 * K0)) * T
            assert np.abs(G - expect).max() <= 1e-13 * np.abs(expect).max()
        # the transverse part alone: the difference of two sigmas
        D = (fem.face_abc_matrix(h, f, K0, 1.0) - fem.face_abc_matrix(h, f, K0, 0.0)) * (2.0 * K0 / 1j)
        assert np.abs(D - T).max() <= 1e-12 * np.abs(T).max()


def _nodal(h, fn):
    """Nodal values [24] of the vector field fn(x) (-> 3-vector) on the brick."""
    u = np.zeros(24)
    for a in range(8):
        x = np.array(_local(a), dtype=float) * np.asarray(h)
        u[3 * a:3 * a + 3] = fn(x)
    return u


@pytest.mark.parametrize("h", [(0.004, 0.017, 0.010), (0.011, 0.009, 0.013)])
def test_abc_transverse_term_exact_integrals(h):
    """u^T T v = int grad_t u_g . grad_t v_g ds for Q1 fields whose integrals
    are known exactly: linear, bilinear and normal-only fields."""
    for f in range(6):
        axis, side = f // 2, f % 2
        t1, t2 = [t for t in range(3) if t != axis]
        T = (fem.face_abc_matrix(h, f, K0, 1.0) - fem.face_abc_matrix(h, f, K0, 0.0)).imag * (2.0 * K0)
        area = h[t1] * h[t2]
        e = np.eye(3)
        # component t1 linear in t1: |grad_t|^2 = 1 over the face
        u = _nodal(h, lambda x: x[t1] * e[t1])
        assert u @ T @ u == pytest.approx(area, rel=1e-13)
        # component t2 = 3 x_t1 - 2 x_t2 against component t2 = x_t2: grad . grad = -2
        u = _nodal(h, lambda x: (3.0 * x[t1] - 2.0 * x[t2]) * e[t2])
        v = _nodal(h, lambda x: x[t2] * e[t2])
        assert u @ T @ v == pytest.approx(-2.0 * area, rel=1e-13)
        # bilinear x_t1 x_t2 in component t1: int (x_t2^2 + x_t1^2) = area (h2^2 + h1^2) / 3
        u = _nodal(h, lambda x: x[t1] * x[t2] * e[t1])
        assert u @ T @ u == pytest.approx(area * (h[t1] ** 2 + h[t2] ** 2) / 3.0, rel=1e-13)
        # a field varying only along the normal is constant on the face: no transverse energy
        u = _nodal(h, lambda x: (x[axis] + 0.3) * (e[t1] + e[t2]))
        assert abs(T @ u).max() <= 1e-12 * np.abs(T).max() * np.abs(u).max()
        # the normal component never enters
        u = _nodal(h, lambda x: (x[t1] * x[t2] + x[axis]) * e[axis])
        assert np.all(T @ u == 0.0)


def _hat_exp_integrals(a, h):
    """Exact 1-D integrals over [0, h] of the two hats phi0 = 1 - t/h,
    phi1 = t/h and of their derivatives against exp(a t) (a complex, a h != 0):
    returns (int phi_p e, int phi_p' e) for p = 0, 1."""
    ea = np.exp(a * h)
    j0 = (ea - 1.0) / a                      # int e^{at}
    j1 = h * ea / a - (ea - 1.0) / a ** 2    # int t e^{at}
    val = np.array([j0 - j1 / h, j1 / h])
    der = np.array([-j0 / h, j0 / h])
    return val, der


def test_abc_transverse_rhs_term_against_exact_integral():
    """The transverse part of the right-hand side G(W, H_i) on every face,
    (j/2k0) int grad_t N_a . grad_t (H_i)_alpha ds with grad_t H_i =
    -j k0 k_t H_i, against the exact integral of the plane wave (products of
    closed-form 1-D integrals).  The oracle uses 2x2 Gauss points, whose error
    at k0 h = 2 pi / 40 is below 1e-5 of the largest entry."""
    lam = fem.C0 / 3e9
    h = (lam / 40.0, lam / 33.0, lam / 45.0)
    k_hat = np.array([0.48, -0.6, 0.64])
    k_hat /= np.linalg.norm(k_hat)
    p_hat = np.cross(k_hat, [0.0, 0.0, 1.0])
    p_hat /= np.linalg.norm(p_hat)
    amp = 0.7 - 0.2j
    corner = np.array([[0.013, -0.021, 0.007]])
    for f in range(6):
        axis, side = f // 2, f % 2
        tang = [t for t in range(3) if t != axis]
        got = (fem.face_rhs(h, f, corner, K0, k_hat, p_hat, amp, 1.0)
               - fem.face_rhs(h, f, corner, K0, k_hat, p_hat, amp, 0.0))[0, :, 0]
        a = -1j * K0 * k_hat  # H_i = p amp exp(a . x)
        x_face = corner[0, axis] + side * h[axis]
        base = amp * np.exp(a[axis] * x_face + sum(a[t] * corner[0, t] for t in tang))
        ints = {t: _hat_exp_integrals(a[t], h[t]) for t in tang}
        expect = np.zeros(24, complex)
        for b in range(8):
            lb = _local(b)
            if lb[axis] != side:
                continue
            # int grad_t N_b . grad_t exp(a.x) = sum_t a_t int d_t N_b exp(a.x)
            s = 0.0
            for t in tang:
                o = [u for u in tang if u != t][0]
                s += a[t] * ints[t][1][lb[t]] * ints[o][0][lb[o]]
            for al in tang:
                expect[3 * b + al] = (1j / (2.0 * K0)) * base * p_hat[al] * s
        assert np.abs(got - expect).max() <= 1e-5 * np.abs(expect).max()
        # normal components and off-face nodes get nothing
        assert np.all(got[[3 * b + axis for b in range(8)]] == 0.0)
        assert np.all(got[[3 * b + al for b in range(8) if _local(b)[axis] != side for al in range(3)]] == 0.0)
