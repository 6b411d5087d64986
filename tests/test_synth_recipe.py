"""The seeded input generators (``synth``) against the input recipe they
implement: stencil values and sparsity counts, the upwind coefficients of the
convection-diffusion matrices, the banded matrix's distinct in-band columns and
diagonal dominance, the distributions of x_true and of the benchmark basis, and
the conditioning of the Logscaled and glued panels.  CPU only."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth


def dense(A):
    return sp.csr_matrix((A.vals, A.colind, A.rowptr), shape=(A.n, A.n)).toarray()


def check_csr(A):
    assert A.rowptr[0] == 0 and A.rowptr[-1] == A.nnz == len(A.colind) == len(A.vals)
    assert A.rowptr.dtype == np.int64 and A.colind.dtype == np.int32 and A.vals.dtype == np.float64
    for i in range(A.n):
        c = A.colind[A.rowptr[i]:A.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)              # sorted, no duplicates
        assert c.min() >= 0 and c.max() < A.n


@pytest.mark.parametrize("N", [1, 2, 7])
def test_laplace2d_is_the_5_point_stencil(N):
    A = synth.laplace2d(N)
    check_csr(A)
    assert A.n == N * N and A.nnz == 5 * N * N - 4 * N
    D = dense(A)
    T = 2 * np.eye(N) - np.eye(N, k=1) - np.eye(N, k=-1)
    assert np.array_equal(D, np.kron(np.eye(N), T) + np.kron(T, np.eye(N)))


@pytest.mark.parametrize("N", [1, 3, 5])
def test_laplace3d_is_the_7_point_stencil(N):
    A = synth.laplace3d(N)
    check_csr(A)
    assert A.n == N ** 3 and A.nnz == 7 * N ** 3 - 6 * N * N
    D = dense(A)
    T = 2 * np.eye(N) - np.eye(N, k=1) - np.eye(N, k=-1)
    I = np.eye(N)
    L = np.kron(np.kron(I, I), T) + np.kron(np.kron(I, T), I) + np.kron(np.kron(T, I), I)
    assert np.array_equal(D, L)


@pytest.mark.parametrize("dim,seed", [(2, 1), (2, 9), (3, 4), (3, 11)])
def test_convdiff_is_first_order_upwind(dim, seed):
    """Centre 2 dim + sum |Pe_a|; along each axis the upwind neighbour carries
    -1 - |Pe_a| and the downwind one -1; interior rows sum to zero (an
    M-matrix); the cell Peclet number lies in [0, 10]; nonsymmetric."""
    N = 6
    A = synth.convdiff2d(N, seed) if dim == 2 else synth.convdiff3d(N, seed)
    check_csr(A)
    D = dense(A)
    centre = D[0, 0]
    assert np.all(np.diag(D) == centre)
    strides = [N ** a for a in range(dim)]
    pe = []
    mid = sum(s * (N // 2) for s in strides)          # an interior point
    for s in strides:
        lo, hi = D[mid, mid - s], D[mid, mid + s]
        assert sorted([lo, hi])[1] == -1.0 and min(lo, hi) <= -1.0
        pe.append(-1.0 - min(lo, hi))
    assert centre == pytest.approx(2 * dim + sum(pe), rel=1e-15)
    assert 0.0 <= np.sqrt(sum(p * p for p in pe)) <= 10.0
    assert abs(D[mid].sum()) <= 1e-12 * centre
    assert np.all(D - np.diag(np.diag(D)) <= 0.0)
    assert not np.array_equal(D, D.T)


def test_banded_random_has_distinct_in_band_columns_and_dominant_diagonal():
    n, band, k = 3000, 100, 26
    A = synth.banded_random(n, 5, band=band, offdiag=k)
    check_csr(A)
    for i in range(n):
        c = A.colind[A.rowptr[i]:A.rowptr[i + 1]]
        v = A.vals[A.rowptr[i]:A.rowptr[i + 1]]
        window = min(n, i + band + 1) - max(0, i - band) - 1
        assert len(c) == min(k, window) + 1               # off-diagonals plus the diagonal
        assert i in c and np.all(np.abs(c - i) <= band)
        off = np.abs(v[c != i]).sum()
        assert v[c == i][0] == pytest.approx(1.1 * off + 1.0, rel=1e-15)
    small = synth.banded_random(10, 1, band=1000, offdiag=26)   # window smaller than 26: full rows
    assert np.all(dense(small) != 0.0)
    offv = np.concatenate([A.vals[A.rowptr[i]:A.rowptr[i + 1]][A.colind[A.rowptr[i]:A.rowptr[i + 1]] != i]
                           for i in range(n)])
    assert abs(offv.mean()) < 0.02 and abs(offv.std() - 1.0) < 0.02     # N(0, 1)


def test_x_true_and_the_benchmark_basis():
    x = synth.x_true(200000, 0)
    assert np.array_equal(x, synth.x_true(200000, 0)) and not np.array_equal(x, synth.x_true(200000, 1))
    assert x.min() >= -1.0 and x.max() < 1.0
    assert abs(x.mean()) < 0.01 and abs(x.var() - 1.0 / 3.0) < 0.01       # U(-1, 1)
    n, c = 100000, 8
    X = synth.tall_basis(n, c, seed=1, ld=n + 5)
    assert X.shape == (n + 5, c) and X.flags.f_contiguous and np.all(X[n:] == 0.0)
    G = X[:n].T @ X[:n]
    assert np.all(np.abs(np.diag(G) - 1.0) < 6 * np.sqrt(2.0 / n))          # unit columns
    assert np.max(np.abs(G - np.diag(np.diag(G)))) < 6 / np.sqrt(n)        # orthogonal to sqrt(1/n)


@pytest.mark.parametrize("kappa", [1e3, 1e8, 1e12])
def test_logscaled_panel_has_the_requested_condition_number(kappa):
    V = synth.logscaled(2000, 12, kappa, 3)
    s = np.linalg.svd(V, compute_uv=False)
    assert s[0] == pytest.approx(1.0, rel=1e-10)
    assert s[0] / s[-1] == pytest.approx(kappa, rel=1e-4)
    assert np.allclose(np.log10(s), np.linspace(0.0, -np.log10(kappa), 12), atol=1e-4)


@pytest.mark.parametrize("growth", [2.0, 10.0])
def test_glued_panels_as_documented(growth):
    """The first panel has condition kappa_panel; the later panels are mixed
    with their predecessors (far from orthogonal to them) and better
    conditioned; the accumulated condition number grows, slowly."""
    n, c, p, kp = 3000, 6, 5, 1e5
    V = synth.glued(n, c, p, kp, 7, growth=growth)
    assert V.shape == (n, c * p) and V.flags.f_contiguous
    total = [np.linalg.cond(V[:, :c * (j + 1)]) for j in range(p)]
    own = [np.linalg.cond(V[:, c * j:c * (j + 1)]) for j in range(p)]
    assert own[0] == pytest.approx(kp, rel=1e-6)
    assert all(10.0 <= k <= 1000.0 for k in own[1:])
    assert all(b >= a for a, b in zip(total, total[1:]))
    assert kp < total[-1] < 3 * kp
    for j in range(1, p):      # largest principal-angle cosine with the previous panel
        Qa = np.linalg.qr(V[:, c * (j - 1):c * j])[0]
        Qb = np.linalg.qr(V[:, c * j:c * (j + 1)])[0]
        assert np.linalg.svd(Qa.T @ Qb, compute_uv=False)[0] > 0.5


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_glued_sweep_fixes_the_panels_and_sweeps_the_total(seed):
    n, c, p, kp = 4000, 5, 6, 1e3
    prev = 0.0
    for km in (1e2, 1e4, 1e6, 1e10):
        V = synth.glued_sweep(n, c, p, kp, km, seed)
        assert V.shape == (n, c * p) and V.flags.f_contiguous
        for j in range(p):
            assert np.linalg.cond(V[:, c * j:c * (j + 1)]) == pytest.approx(kp, rel=1e-6)
        tot = np.linalg.cond(V)
        assert 10 * km <= tot <= 300 * km
        assert tot > prev
        prev = tot
