"""Multicolor Gauss-Seidel preconditioner of the oracle (test infrastructure only).

The paper's last experiment (§VIII, Fig. 9) runs s-step GMRES with a local
Gauss-Seidel preconditioner, the multicolor Gauss-Seidel of Kokkos Kernels
(Deveci et al. 2016) inside the matrix powers kernel.  The paper gives no
further detail; the reading taken here:

* The rows are colored greedily in natural order on the symmetrized pattern:
  row i takes the smallest color not held by a neighbor j < i (a_ij != 0 or
  a_ji != 0).  Rows of one color are never coupled, so a Gauss-Seidel sweep
  may update all of them at once.
* M^{-1} r is one forward Gauss-Seidel sweep from zero in color order: colors
  0, 1, ... in turn, each row i of the color set to
  z_i = (r_i - sum_{j != i} a_ij z_j) / a_ii with the z values of the colors
  already swept (later colors still zero).  That is z = (D + L)^{-1} r for the
  matrix permuted to color order, D + L its lower triangle.
* Preconditioning is from the right: the matrix powers kernel applies
  A M^{-1}, the Krylov basis spans K_m(A M^{-1}, r0), the least-squares problem
  minimizes the true residual, and the correction is x += M^{-1} Q y.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def greedy_coloring(A) -> np.ndarray:
    """Greedy distance-1 coloring of the symmetrized pattern of A in natural
    row order: color[i] = the smallest color not used by a neighbor j < i."""
    M = A.tocsr() if sp.issparse(A) else sp.csr_matrix((A.vals, A.colind, A.rowptr), shape=(A.n, A.n))
    S = (abs(M) + abs(M).T).tocsr()
    n = M.shape[0]
    color = np.full(n, -1, dtype=np.int64)
    for i in range(n):
        nb = S.indices[S.indptr[i]:S.indptr[i + 1]]
        used = {int(color[j]) for j in nb if j < i}
        c = 0
        while c in used:
            c += 1
        color[i] = c
    return color


def gs_sweep(A, color: np.ndarray, r: np.ndarray) -> np.ndarray:
    """One forward multicolor Gauss-Seidel sweep from z = 0: colors in
    increasing order, every row of a color from the current z (rows of the
    color itself are still zero, so the sum over j != i is the row product)."""
    M = A.tocsr() if sp.issparse(A) else sp.csr_matrix((A.vals, A.colind, A.rowptr), shape=(A.n, A.n))
    d = M.diagonal()
    z = np.zeros_like(r, dtype=np.float64)
    for c in range(int(color.max()) + 1 if color.size else 0):
        rows = np.nonzero(color == c)[0]
        z[rows] = (r[rows] - M[rows, :] @ z) / d[rows]
    return z
