"""Pins of the oracle's block incomplete Cholesky preconditioner (Section
3.1.5.2, Eq. 5; Section 3.1.5.3; Eq. 6) against facts fixed by the
mathematics rather than by the code:

* the defining property of an incomplete Cholesky factor: L L^T equals A on
  the factor's pattern (unconjugated), and L has no entry outside it;
* on a pattern with no fill (one element: every node couples to every
  other) the factor is the exact Cholesky factor, equal to LAPACK's for a
  real SPD matrix, and M^{-1} = A^{-1};
* one node per band: M^{-1} is the 3x3 block-Jacobi inverse;
* preconditioned COCG reaches the direct solution.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem, krylov, precond
from paper_0704_2344_gb300 import workloads as W

PEC = 255


def _scatterer(shape=(5, 4, 4)):
    prob = W.empty_box(shape, name="bicp_small")     # material is indexed [z, y, x]
    prob.material[1, 1:3, 2] = PEC
    prob.material[2, 1:3, 1:4] = 1
    prob.eps_r = np.array([1.0 + 0j, 3.0 - 0.5j])
    prob.mu_r = np.array([1.0 + 0j, 1.2 + 0j])
    return prob


def _pattern_mask(maps, n_sub):
    """Scalar (i, j), i >= j, of the factor's pattern as a boolean matrix."""
    n = 3 * maps.n_act
    sub = precond.node_subdomain(maps.n_act, n_sub)
    M = np.zeros((n, n), dtype=bool)
    for I in range(maps.n_act):
        for J in maps.col_idx[maps.row_ptr[I]:maps.row_ptr[I + 1]]:
            if J <= I and sub[J] == sub[I]:
                M[3 * I:3 * I + 3, 3 * J:3 * J + 3] = True
    return np.tril(M)


def test_subdomain_bounds():
    assert precond.subdomain_bounds(10, 4).tolist() == [0, 2, 5, 7, 10]
    assert precond.node_subdomain(10, 4).tolist() == [0, 0, 1, 1, 1, 2, 2, 3, 3, 3]
    assert precond.subdomain_bounds(3, 5).tolist() == [0, 0, 1, 1, 2, 3]
    assert precond.node_subdomain(3, 5).tolist() == [1, 3, 4]
    assert precond.node_subdomain(7, 1).tolist() == [0] * 7


@pytest.mark.parametrize("n_sub", [1, 3, 7])
def test_factor_reproduces_A_on_its_pattern(n_sub):
    prob = _scatterer()
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps)
    L = precond.ic0(A, maps, n_sub).toarray()
    mask = _pattern_mask(maps, n_sub)
    assert np.all(L[~mask] == 0)
    assert np.all(np.diag(L) != 0) and np.all(np.diag(L).real > 0)   # principal square roots
    Ad = A.toarray()
    LLt = L @ L.T
    scale = np.abs(Ad).max()
    assert np.abs((LLt - Ad)[mask]).max() <= 1e-13 * scale
    # the factor is incomplete: off the pattern L L^T differs from A (the dropped fill)
    if n_sub == 1:
        assert np.abs(np.tril(LLt - Ad)[~mask]).max() > 1e-6 * scale
    # the conjugated product does not reproduce A: the factor is the complex symmetric one
    assert np.abs((L @ L.conj().T - Ad)[mask]).max() > 1e-6 * scale


def test_no_fill_pattern_gives_lapack_cholesky():
    """One element: all 8 nodes share it, the pattern is dense, IC(0) is the
    exact factorisation.  With a real SPD matrix on that pattern the factor
    equals LAPACK's Cholesky factor."""
    prob = W.empty_box((1, 1, 1), name="one_element")
    maps = fem.mesh_maps(prob)
    assert maps.n_act == 8 and maps.nnzb == 64
    rng = np.random.default_rng(7)
    G = rng.standard_normal((24, 24))
    S = G @ G.T + 24 * np.eye(24)
    L = precond.ic0(sp.csr_matrix(S.astype(complex)), maps, 1).toarray()
    assert np.abs(L.imag).max() == 0
    np.testing.assert_allclose(L.real, np.linalg.cholesky(S), rtol=0, atol=1e-12 * np.abs(S).max())
    # and for the complex symmetric FE matrix of that element, M^{-1} = A^{-1}
    A = fem.assemble(prob, maps=maps)
    Lc = precond.ic0(A, maps, 1)
    r = rng.standard_normal(24) + 1j * rng.standard_normal(24)
    z = precond.apply(Lc, r)
    np.testing.assert_allclose(z, np.linalg.solve(A.toarray(), r), rtol=1e-10)


def test_one_node_per_band_is_block_jacobi():
    prob = W.empty_box((3, 3, 3), name="bicp_tiny")
    prob.material[1, 1, 1] = PEC
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps)
    L = precond.ic0(A, maps, maps.n_act)
    rng = np.random.default_rng(3)
    r = rng.standard_normal((A.shape[0], 2)) + 1j * rng.standard_normal((A.shape[0], 2))
    Dinv = krylov.block_jacobi_inverse(A)
    for c in range(2):
        np.testing.assert_allclose(precond.apply(L, r[:, c]), krylov.apply_block(Dinv, r[:, c]), rtol=1e-11)


def test_apply_is_forward_then_back_substitution():
    """Eq. 6 on a random lower triangular matrix: L y = r and L^T z = y."""
    rng = np.random.default_rng(11)
    n = 30
    L = np.tril(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)), -1) * 0.2
    L[np.arange(n), np.arange(n)] = 2.0 + rng.standard_normal(n) * 0.1 + 0.3j
    r = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    z = precond.apply(sp.csr_matrix(L), r)
    np.testing.assert_allclose(L @ (L.T @ z), r, rtol=0, atol=1e-12)


@pytest.mark.parametrize("n_sub", [1, 4])
def test_bicp_cocg_reaches_the_direct_solution(n_sub):
    prob = _scatterer()
    maps = fem.mesh_maps(prob)
    A = fem.assemble(prob, maps=maps)
    b = np.asarray(fem.rhs(prob, W.normal_incidence(), maps=maps))[:, 0]
    M, _ = precond.preconditioner(A, maps, n_sub)
    x, it, _ = krylov.cocg(A, b, tol=1e-10, M=M)
    xref = fem.solve_direct(A, b)
    assert np.linalg.norm(x - xref) <= 1e-7 * np.linalg.norm(xref)
    assert 0 < it < 400


def test_held_unknowns_stay_unit_rows_and_columns():
    """Symmetry planes hold unknowns as identity rows and columns of A
    (Eqs. 6a/6b).  Eq. 5 then gives L_ii = 1 and no coupling to or from a
    held unknown, exactly, and L L^T = A still holds on the pattern."""
    prob = W.empty_box((6, 6, 4), name="bicp_planes")
    prob.material[1:3, 2:4, 2:4] = PEC
    part = W.mirror_part(prob, 2, 1)
    maps = fem.mesh_maps(part)
    held = np.asarray(maps.fixed)
    assert held.any()
    A = fem.assemble(part, maps=maps)
    for n_sub in (1, 5):
        L = precond.ic0(A, maps, n_sub).toarray()
        assert np.all(L[held, held] == 1)
        L0 = L.copy()
        L0[held, held] = 0
        assert np.all(L0[held, :] == 0) and np.all(L0[:, held] == 0)
        mask = _pattern_mask(maps, n_sub)
        assert np.abs((L @ L.T - A.toarray())[mask]).max() <= 1e-13 * np.abs(A.data).max()
