"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the solver or of the orthogonalization
methods: it only builds matrices and vectors from seeds.  Every generator is
deterministic for a given seed (numpy PCG64 via ``default_rng``), so the CPU
oracle and the GPU path see bit-identical inputs.

Workloads (shapes follow the paper's test problems, §VI and §VIII):

* ``laplace2d(N)``  5-point stencil (4, -1) on an N x N grid, Dirichlet,
  lexicographic order (the 2D Laplace of Tables 2 and 3).
* ``laplace3d(N)``  7-point stencil (6, -1) on an N^3 grid (Laplace3D, Table 4).
* ``convdiff2d / convdiff3d``  upwinded convection-diffusion stencils, a
  nonsymmetric stand-in for the paper's CFD matrix (atmosmodl, Table 4).
* ``banded_random(n)``  random diagonally dominant banded CSR with 27 nonzeros
  per row, a stand-in for the wider SuiteSparse rows of Table 4.
* ``logscaled(n, c, kappa)``  X diag(logspace) Y^T panels (the ``Logscaled``
  matrix of the CholQR2 experiment, §VI).
* ``glued(...)``  panels mixed with their predecessors: the first of
  condition kappa_panel, the later ones better conditioned, the accumulated
  condition number growing slowly.
* ``glued_sweep(...)``  panels of exactly kappa_panel each whose column spaces
  draw closer as kappa_mix grows, so the total condition number is swept with
  the panels' own fixed (the ``glued`` experiments of §VI).
* ``tall_basis(n, c)``  N(0,1)/sqrt(n) columns for the standalone block
  orthogonalization benchmark.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "CSR", "laplace2d", "laplace3d", "convdiff2d", "convdiff3d", "banded_random",
    "x_true", "tall_basis", "logscaled", "glued", "glued_sweep", "rng",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(seed))


class CSR:
    """Compressed sparse rows: int64 row pointers, int32 column indices, FP64 values."""

    __slots__ = ("n", "rowptr", "colind", "vals", "name")

    def __init__(self, n, rowptr, colind, vals, name=""):
        self.n = int(n)
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.colind = np.ascontiguousarray(colind, dtype=np.int32)
        self.vals = np.ascontiguousarray(vals, dtype=np.float64)
        self.name = name

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def __repr__(self):
        return f"CSR({self.name}, n={self.n}, nnz={self.nnz})"


def _stencil_csr(dims, offsets, coef_fn, name):
    """Assemble a Dirichlet stencil matrix on a box grid in lexicographic order.

    ``offsets`` lists integer displacement vectors (the centre first);
    ``coef_fn(k)`` returns the coefficient array (one value per grid point) of
    displacement k.  Entries whose neighbour falls outside the grid are dropped.
    Columns within each row come out sorted ascending.
    """
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    idx = np.arange(n, dtype=np.int64)
    coords = np.unravel_index(idx, dims[::-1])[::-1]  # x fastest
    strides = [1]
    for d in dims[:-1]:
        strides.append(strides[-1] * d)
    cols, vals, rows = [], [], []
    for k, off in enumerate(offsets):
        ok = np.ones(n, dtype=bool)
        lin = np.zeros(n, dtype=np.int64)
        for a in range(len(dims)):
            c = coords[a] + off[a]
            ok &= (c >= 0) & (c < dims[a])
            lin += off[a] * strides[a]
        coef = np.broadcast_to(np.asarray(coef_fn(k), dtype=np.float64), (n,))
        rows.append(idx[ok])
        cols.append((idx + lin)[ok])
        vals.append(coef[ok])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSR(n, rowptr, cols.astype(np.int32), vals, name)


def laplace2d(N: int) -> CSR:
    """5-point Laplacian (4 on the diagonal, -1 off) on an N x N grid."""
    offs = [(0, 0), (-1, 0), (1, 0), (0, -1), (0, 1)]
    return _stencil_csr((N, N), offs, lambda k: 4.0 if k == 0 else -1.0, f"laplace2d_{N}")


def laplace3d(N: int) -> CSR:
    """7-point Laplacian (6 on the diagonal, -1 off) on an N^3 grid."""
    offs = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    return _stencil_csr((N, N, N), offs, lambda k: 6.0 if k == 0 else -1.0, f"laplace3d_{N}")


def _upwind(dims, pe_vec, name):
    """-Laplace(u) + w.grad(u), first-order upwind, cell Peclet numbers ``pe_vec``.

    Centre 2*dim + sum|Pe_a|; the upwind neighbour along axis a gets -1-|Pe_a|,
    the downwind one -1.
    """
    nd = len(dims)
    offs = [tuple([0] * nd)]
    coefs = [2.0 * nd + float(np.sum(np.abs(pe_vec)))]
    for a in range(nd):
        for sgn in (-1, 1):
            o = [0] * nd
            o[a] = sgn
            offs.append(tuple(o))
            upwind = (pe_vec[a] > 0 and sgn < 0) or (pe_vec[a] < 0 and sgn > 0)
            coefs.append(-1.0 - abs(pe_vec[a]) if upwind else -1.0)
    return _stencil_csr(dims, offs, lambda k: coefs[k], name)


def convdiff2d(N: int, seed: int) -> CSR:
    """2D upwinded convection-diffusion, Pe ~ U(0,10), flow angle ~ U(0, 2 pi)."""
    g = rng(seed)
    pe = g.uniform(0.0, 10.0)
    th = g.uniform(0.0, 2.0 * np.pi)
    return _upwind((N, N), np.array([pe * np.cos(th), pe * np.sin(th)]), f"convdiff2d_{N}_s{seed}")


def convdiff3d(N: int, seed: int) -> CSR:
    """3D upwinded convection-diffusion (7-point), Pe ~ U(0,10), random direction."""
    g = rng(seed)
    pe = g.uniform(0.0, 10.0)
    d = g.standard_normal(3)
    d /= np.linalg.norm(d)
    return _upwind((N, N, N), pe * d, f"convdiff3d_{N}_s{seed}")


def banded_random(n: int, seed: int, band: int = 1000, offdiag: int = 26) -> CSR:
    """Random banded CSR: ``offdiag`` distinct off-diagonal columns per row in
    [i-band, i+band] (clipped to the matrix, diagonal excluded), N(0,1) values,
    diagonal equal to 1.1 * sum|off-diagonal| + 1 (strictly diagonally
    dominant, nonsymmetric).  The distinct columns come from sorted draws u_1 <=
    ... <= u_k in [0, W-k] shifted by 0..k-1 (W = window size), a vectorized
    sample of k distinct sorted positions; rows whose window holds fewer than
    ``offdiag`` candidates take all of them."""
    g = rng(seed)
    i = np.arange(n, dtype=np.int64)
    lo = np.maximum(0, i - band)
    hi = np.minimum(n, i + band + 1)
    W = hi - lo - 1                                   # candidates without the diagonal
    k = np.minimum(offdiag, W)
    u = np.floor(g.random((n, offdiag)) * (np.maximum(W - k, 0) + 1)[:, None]).astype(np.int64)
    u.sort(axis=1)
    u += np.arange(offdiag)[None, :]
    cols = lo[:, None] + u
    cols = np.where(cols >= i[:, None], cols + 1, cols)   # skip the diagonal
    valid = np.arange(offdiag)[None, :] < k[:, None]
    v = g.standard_normal((n, offdiag)) * valid
    diag = 1.1 * np.abs(v).sum(axis=1) + 1.0
    allc = np.concatenate([np.where(valid, cols, n + 1), i[:, None]], axis=1)
    allv = np.concatenate([v, diag[:, None]], axis=1)
    o = np.argsort(allc, axis=1, kind="stable")
    allc = np.take_along_axis(allc, o, axis=1)
    allv = np.take_along_axis(allv, o, axis=1)
    keep = allc <= n - 1
    counts = keep.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(counts)
    return CSR(n, rowptr, allc[keep].astype(np.int32), allv[keep], f"banded_{n}_s{seed}")


def x_true(n: int, seed: int = 0) -> np.ndarray:
    """Exact solution vector, U(-1, 1) entries."""
    return rng(seed).uniform(-1.0, 1.0, size=n)


def tall_basis(n: int, cols: int, seed: int = 1, dtype=np.float64, ld: int | None = None) -> np.ndarray:
    """N(0,1)/sqrt(n) entries in a column-major n x cols array (Fortran order).

    With ``ld`` > n the array is (ld, cols) with rows n..ld-1 zero.  At large n
    the columns are orthonormal to within about sqrt(cols/n).
    """
    ld = n if ld is None else ld
    out = np.zeros((ld, cols), dtype=dtype, order="F")
    g = rng(seed)
    for c in range(cols):
        out[:n, c] = (g.standard_normal(n) / np.sqrt(n)).astype(dtype)
    return out


def _orthonormal_factor(g, n, c):
    # Random orthonormal columns from the polar-free Gram-Schmidt of a Gaussian matrix
    # via numpy's LAPACK QR; only used to build test panels, never by the solvers.
    z = g.standard_normal((n, c))
    q, r = np.linalg.qr(z)
    return q * np.sign(np.diag(r))


def logscaled(n: int, c: int, kappa: float, seed: int) -> np.ndarray:
    """X diag(logspace(0, -log10 kappa, c)) Y^T with random orthonormal X (n x c)
    and Y (c x c): a panel with 2-norm condition number kappa."""
    g = rng(seed)
    X = _orthonormal_factor(g, n, c)
    Y = _orthonormal_factor(g, c, c)
    sig = np.logspace(0.0, -np.log10(kappa), c)
    return np.asfortranarray((X * sig) @ Y.T)


def glued(n: int, c: int, panels: int, kappa_panel: float, seed: int, growth: float = 2.0) -> np.ndarray:
    """Panels V_j = X_j diag(logspace) Y_j^T of condition kappa_panel, each one
    after the first mixed with its predecessor: V_j += (1 - 1/growth) V_{j-1} W_j
    (W_j Gaussian / sqrt(c)), so consecutive panels are far from orthogonal.
    The first panel keeps condition kappa_panel; the mixing term dominates the
    later panels' small singular values, so their own condition numbers fall
    (to 10-1000 for kappa_panel = 1e5) and the accumulated condition number
    grows only slowly (1e5 -> 1.4e5-2.8e5 over five panels of six columns)."""
    g = rng(seed)
    blocks = []
    for j in range(panels):
        V = logscaled(n, c, kappa_panel, int(g.integers(1 << 31)))
        if j > 0:
            W = g.standard_normal((c, c)) / np.sqrt(c)
            V = V + (1.0 - 1.0 / growth) * (blocks[-1] @ W)
        blocks.append(V)
    return np.asfortranarray(np.concatenate(blocks, axis=1))


def glued_sweep(n: int, c: int, panels: int, kappa_panel: float, kappa_mix: float, seed: int) -> np.ndarray:
    """Big panel of ``panels`` blocks of c columns: every block has 2-norm
    condition number kappa_panel exactly, and the total condition number grows
    with kappa_mix while the blocks' own stays fixed.

    Y = logscaled(n, c * panels, kappa_mix) sets the geometry: block j is
    Q_j diag(logspace(0, -log10 kappa_panel, c)) Z_j^T, with Q_j an orthonormal
    basis of Y's block column j and Z_j a random c x c orthogonal matrix.  The
    larger kappa_mix, the smaller the principal angles between the blocks'
    column spaces.  For 6 blocks of 5 columns at kappa_panel = 1e3 the total
    condition number is 10-300 times kappa_mix for kappa_mix from 1e2 to 1e10
    (measured in the tests).
    """
    g = rng(seed)
    Y = logscaled(n, c * panels, kappa_mix, int(g.integers(1 << 31)))
    sig = np.logspace(0.0, -np.log10(kappa_panel), c)
    out = np.empty((n, c * panels), order="F")
    for j in range(panels):
        Qj = _orthonormal_factor_of(Y[:, j * c:(j + 1) * c])
        Z = _orthonormal_factor(g, c, c)
        out[:, j * c:(j + 1) * c] = (Qj * sig) @ Z.T
    return out


def _orthonormal_factor_of(Y):
    # Orthonormal basis of Y's columns (numpy's LAPACK QR, signs fixed); test
    # inputs only.
    q, r = np.linalg.qr(Y)
    return q * np.sign(np.diag(r))
