"""Independent numerical checkers used by the oracle's pins (test infrastructure only).

* ``orth_error``  ||I - Q^T Q|| in the 2-norm (symmetric eigenvalues) and the
                  Frobenius norm (the orthogonality error of §IV-§VI).
* ``cond2``       2-norm condition number from singular values.
* ``exact_gram``  X^T Y in exact rational arithmetic (brute force, tiny inputs).
* ``laplace2d_extreme_eigs``  closed-form extreme eigenvalues of the 5-point
                  Laplacian, 4 - 2cos(i pi/(N+1)) - 2cos(j pi/(N+1)).
"""
from __future__ import annotations

from fractions import Fraction
import math
import numpy as np


def orth_error(Q: np.ndarray):
    E = np.eye(Q.shape[1]) - Q.T @ Q
    ev = np.linalg.eigvalsh((E + E.T) / 2)
    return float(np.max(np.abs(ev))) if ev.size else 0.0, float(np.linalg.norm(E))


def cond2(V: np.ndarray) -> float:
    sv = np.linalg.svd(V, compute_uv=False)
    return float(sv[0] / sv[-1])


def exact_gram(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """X^T Y with every product and sum done in exact rationals, then rounded
    once to the nearest double."""
    out = np.zeros((X.shape[1], Y.shape[1]))
    Xf = [[Fraction(float(v)) for v in X[:, i]] for i in range(X.shape[1])]
    Yf = [[Fraction(float(v)) for v in Y[:, j]] for j in range(Y.shape[1])]
    for i, xi in enumerate(Xf):
        for j, yj in enumerate(Yf):
            out[i, j] = float(sum(a * b for a, b in zip(xi, yj)))
    return out


def laplace2d_extreme_eigs(N: int):
    lo = 4.0 - 4.0 * math.cos(math.pi / (N + 1))
    hi = 4.0 + 4.0 * math.cos(math.pi / (N + 1))
    return lo, hi


def arnoldi_residual(Aop, Q: np.ndarray, H: np.ndarray, k: int) -> float:
    """||A Q_{1:k} - Q_{1:k+1} H_{1:k+1,1:k}||_F / (||A||_F ||H||_F)."""
    AQ = np.column_stack([Aop @ Q[:, i] for i in range(k)])
    E = AQ - Q[:, : k + 1] @ H[: k + 1, :k]
    anorm = math.sqrt(float((Aop.multiply(Aop)).sum()))
    return float(np.linalg.norm(E) / (anorm * np.linalg.norm(H[: k + 1, :k])))
