"""Plain CPU conjugate gradient for the complex-symmetric FE system.

TEST INFRASTRUCTURE ONLY (imported by tests/, the smoke check and bench.py's
CPU legs; never by the library).

The paper solves the symmetrised system with conjugate gradients and diagonal
preconditioning (Sections 3.1.5 and 4.2.5).  On a complex symmetric (not
Hermitian) matrix the consistent form of CG uses the unconjugated bilinear
form u^T v everywhere (the paper's incomplete Cholesky likewise squares L
entries instead of taking moduli, Eq. 5): this is COCG.  The diagonal
preconditioner is generalised to the 3x3 diagonal blocks of the node rows
(Section 3.1.2 stores three rows per node); any other preconditioner, such as
the block incomplete Cholesky of Section 3.1.5.3 (oracle/precond.py), can be
passed in as the callable M.

Each step follows the textbook order: q = A p, alpha = rho / p^T q,
x += alpha p, r -= alpha q, z = D^{-1} r, rho' = r^T z, p = z + (rho'/rho) p.
"""
from __future__ import annotations

import numpy as np


def block_jacobi_inverse(A):
    """[n_nodes, 3, 3] inverses of the 3x3 diagonal blocks of A."""
    n = A.shape[0] // 3
    Ac = A.tocsr()
    D = np.empty((n, 3, 3), dtype=complex)
    idx = np.arange(n)
    for al in range(3):
        for be in range(3):
            D[:, al, be] = np.asarray(Ac[3 * idx + al, 3 * idx + be]).ravel()
    return np.linalg.inv(D)


def apply_block(Dinv, r):
    return np.einsum("nab,nb->na", Dinv, r.reshape(-1, 3)).reshape(-1)


def cocg(A, b, tol=1e-8, maxiter=100000, x0=None, Dinv=None, M=None):
    """Solve A x = b (A complex symmetric) by preconditioned COCG until the
    recursive residual satisfies ||r||_2 <= tol ||b||_2.  The preconditioner
    is z = M(r) when M is given, else block Jacobi.  Returns (x, iters,
    history of ||r||/||b||)."""
    b = np.asarray(b, dtype=complex).reshape(-1)
    if M is None:
        if Dinv is None:
            Dinv = block_jacobi_inverse(A)
        M = lambda v: apply_block(Dinv, v)  # noqa: E731
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=complex).reshape(-1)
    r = b - A @ x
    nb = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / nb]
    if hist[-1] <= tol:
        return x, 0, hist
    z = M(r)
    p = z.copy()
    rho = r @ z
    it = 0
    while it < maxiter:
        it += 1
        q = A @ p
        alpha = rho / (p @ q)
        x += alpha * p
        r -= alpha * q
        hist.append(np.linalg.norm(r) / nb)
        if hist[-1] <= tol:
            break
        z = M(r)
        rho_new = r @ z
        p = z + (rho_new / rho) * p
        rho = rho_new
    return x, it, hist


def cocg_multi(A, B, tol=1e-8, maxiter=100000):
    """Column-by-column COCG; returns X [n, R] and iteration counts."""
    B = np.asarray(B).reshape(B.shape[0], -1)
    Dinv = block_jacobi_inverse(A)
    X = np.empty_like(B, dtype=complex)
    its = []
    for r in range(B.shape[1]):
        x, it, _ = cocg(A, B[:, r], tol=tol, maxiter=maxiter, Dinv=Dinv)
        X[:, r] = x
        its.append(it)
    return X, its
