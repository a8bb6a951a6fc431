"""Block incomplete Cholesky preconditioner (BICP) of the complex symmetric
FE system, plain FP64 CPU version.

TEST INFRASTRUCTURE ONLY (imported by tests/ and bench.py's CPU legs; never
by the library).

What it computes:

* Section 3.1.5.2, Eq. 5: the incomplete Cholesky factor L (lower
  triangular, A ~ L L^T) built column by column on the pattern of A, with no
  fill outside it:
      L_jj = sqrt(A_jj - sum_{k<j} L_jk^2),
      L_ij = (A_ij - sum_{k<j} L_ik L_jk) / L_jj      for i > j.
  The printed second line has its indices garbled (1/L_ii, A_ji, k < i); the
  form above is the one whose product L L^T reproduces A on the pattern,
  which is what an incomplete Cholesky factor means.  The matrix is complex
  symmetric, so the squares and products are unconjugated (L L^T, not
  L L^H) and sqrt is the principal branch.
* Section 3.1.5.3: the block variant.  The node rows are split into S
  contiguous bands, one per processor, and only the terms whose row and
  column lie in the same band are factored; couplings across bands are
  dropped.  S = 1 is the plain incomplete Cholesky of Section 3.1.5.2.
  Band s holds the nodes floor(s n / S) <= I < floor((s + 1) n / S).
* Eq. 6: z = M^{-1} r = L^{-T} (L^{-1} r), by forward then back substitution.

The pattern of A is that of its 3x3 node blocks (Section 3.1.2 stores the
three rows of a node together): every node pair that shares an active
element couples all nine component pairs, whether or not a value is zero.
"""
from __future__ import annotations

import cmath

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def subdomain_bounds(n_nodes: int, n_sub: int) -> np.ndarray:
    """[S + 1] first node of each band, floor(s n / S) (Section 3.1.5.3:
    each processor holds a contiguous band of node rows)."""
    if n_sub < 1:
        raise ValueError("at least one subdomain")
    s = np.arange(n_sub + 1, dtype=np.int64)
    return (s * n_nodes) // n_sub


def node_subdomain(n_nodes: int, n_sub: int) -> np.ndarray:
    """Band of every node."""
    b = subdomain_bounds(n_nodes, n_sub)
    return np.searchsorted(b, np.arange(n_nodes), side="right") - 1


def lower_pattern_by_columns(maps, n_sub: int):
    """For each scalar column j, the sorted rows i > j of the factor's
    pattern: node blocks (I, J) of A with J <= I in the same band, all nine
    entries of an off-diagonal block and the strict lower triangle of a
    diagonal block."""
    n = 3 * maps.n_act
    sub = node_subdomain(maps.n_act, n_sub)
    cols = [[] for _ in range(n)]
    for I in range(maps.n_act):
        for J in maps.col_idx[maps.row_ptr[I]:maps.row_ptr[I + 1]]:
            J = int(J)
            if J > I or sub[J] != sub[I]:
                continue
            for a in range(3):
                for b in range(3):
                    i, j = 3 * I + a, 3 * J + b
                    if i > j:
                        cols[j].append(i)
    for c in cols:
        c.sort()
    return cols


def ic0(A, maps, n_sub: int = 1):
    """Incomplete Cholesky factor of Eq. 5 restricted to S bands (Section
    3.1.5.3), column by column.  Returns L as a SciPy CSR matrix (lower
    triangular, complex128).  Raises ZeroDivisionError on a zero pivot."""
    n = 3 * maps.n_act
    Ac = A.tocsr()
    a_row = [dict(zip(Ac.indices[Ac.indptr[i]:Ac.indptr[i + 1]].tolist(),
                      Ac.data[Ac.indptr[i]:Ac.indptr[i + 1]].tolist())) for i in range(n)]
    col_rows = lower_pattern_by_columns(maps, n_sub)
    L = [dict() for _ in range(n)]          # L[i][k] = L_ik, filled column by column
    for j in range(n):
        Lj = L[j]                           # holds L_jk for k < j only
        d = a_row[j].get(j, 0j) - sum(v * v for v in Lj.values())
        ljj = cmath.sqrt(d)
        if ljj == 0:
            raise ZeroDivisionError(f"zero pivot in column {j}")
        for i in col_rows[j]:
            Li = L[i]
            t = a_row[i].get(j, 0j) - sum(Li[k] * v for k, v in Lj.items() if k in Li)
            Li[j] = t / ljj
        Lj[j] = ljj
    rows = np.repeat(np.arange(n), [len(r) for r in L])
    cols = np.fromiter((k for r in L for k in r), dtype=np.int64, count=len(rows))
    vals = np.fromiter((v for r in L for v in r.values()), dtype=complex, count=len(rows))
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def apply(L, r):
    """z = (L L^T)^{-1} r by the forward and back substitutions of Eq. 6;
    r may hold several columns."""
    Lc = L.tocsr()
    y = spla.spsolve_triangular(Lc, np.asarray(r, dtype=complex), lower=True)
    return spla.spsolve_triangular(Lc.T.tocsr(), y, lower=False)


def preconditioner(A, maps, n_sub: int = 1):
    """The callable z = M^{-1} r of the block incomplete Cholesky
    preconditioner with S bands, and its factor."""
    L = ic0(A, maps, n_sub)
    return (lambda r: apply(L, r)), L
