"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these compare the oracle with itself: each check is a closed form, a
library routine for a special case, exact rational arithmetic, a bound printed
in the paper, or a uniqueness property of the QR factorization.
"""
import json
import math
import os

import numpy as np
import scipy.sparse as sp
import pytest

import synth
from oracle import blockortho as bo, krylov as kr, checks

EPS = np.finfo(np.float64).eps
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _sign_fixed_qr(V):
    q, r = np.linalg.qr(V)
    sg = np.where(np.diag(r) < 0, -1.0, 1.0)
    return q * sg, r * sg[:, None]


# ---------------------------------------------------------------- Cholesky
def test_chol_upper_matches_lapack():
    g = synth.rng(11)
    for c in (1, 5, 11, 61):
        B = g.standard_normal((3 * c, c))
        G = B.T @ B
        R, info = bo.chol_upper(G)
        assert info == 0
        L = np.linalg.cholesky(G)
        assert np.allclose(R, L.T, rtol=1e-12, atol=1e-12 * np.abs(L).max())
        assert np.all(np.diag(R) > 0)
        assert np.allclose(np.triu(R), R)


def test_chol_upper_reports_first_bad_pivot():
    G = np.diag([4.0, 1.0, -1.0, 2.0])
    _, info = bo.chol_upper(G)
    assert info == 3
    G = np.array([[1.0, 1.0], [1.0, 1.0]])  # singular: second pivot 0
    _, info = bo.chol_upper(G)
    assert info == 2
    _, info = bo.chol_upper(np.array([[np.nan]]))
    assert info == 1


# ---------------------------------------------------------------- Gram
def test_gram_of_pip_is_exact_dot_product_up_to_rounding():
    """The single reduction [Q, V]^T V of BCGS-PIP equals the exact rational
    dot products to within the classic n*eps*|x|.|y| bound."""
    g = synth.rng(12)
    n, k, s = 37, 3, 4
    Q = g.standard_normal((n, k))
    V = g.standard_normal((n, s))
    X = np.concatenate([Q, V], axis=1)
    ex = checks.exact_gram(X, V)
    got = X.T @ V
    bound = n * EPS * (np.abs(X).T @ np.abs(V))
    assert np.all(np.abs(got - ex) <= bound)


# ---------------------------------------------------------------- QR checkers
def test_hhqr_matches_lapack_qr():
    V = synth.rng(13).standard_normal((200, 9))
    Q, R = bo.hhqr(V)
    q, r = _sign_fixed_qr(V)
    assert np.allclose(Q, q, atol=1e-13)
    assert np.allclose(R, r, atol=1e-12)


def test_cholqr_unique_qr_with_positive_diagonal():
    """QR with a positive R diagonal is unique (Fig. 1 caption), so CholQR of a
    well-conditioned block equals Householder QR (LAPACK)."""
    V = synth.rng(14).standard_normal((500, 6))
    Q, R = bo.cholqr(V)
    q, r = _sign_fixed_qr(V)
    assert np.allclose(R, r, rtol=0, atol=1e-12 * np.abs(r).max())
    assert np.allclose(Q @ R, V, atol=1e-12)
    assert checks.orth_error(Q)[0] < 1e-14


def test_bcgs_pip_equals_qr_of_concatenation():
    """BCGS-PIP of V against an orthonormal Q returns the trailing block column
    of the (unique) QR of [Q, V] (Fig. 4a)."""
    g = synth.rng(15)
    n, k, s = 400, 7, 5
    Q, _ = _sign_fixed_qr(g.standard_normal((n, k)))
    V = g.standard_normal((n, s))
    Qh, P, T = bo.bcgs_pip(Q, V)
    qq, rr = _sign_fixed_qr(np.concatenate([Q, V], axis=1))
    # R of [Q, V] is [[I, P], [0, T]] up to the rounding of Q's orthonormality
    assert np.allclose(rr[:k, k:], P, atol=1e-13)
    assert np.allclose(rr[k:, k:], T, atol=1e-13)
    assert np.allclose(qq[:, k:], Qh, atol=1e-12)
    assert np.allclose(Q @ P + Qh @ T, V, atol=1e-13)


def test_bcgs_pip2_without_previous_blocks_is_cholqr2():
    """§IV-C: with no previous blocks BCGS-PIP2 is CholQR2."""
    V = synth.rng(16).standard_normal((300, 6))
    Qa, Pa, Ta = bo.bcgs_pip2(np.zeros((300, 0)), V)
    Qb, Rb = bo.cholqr2(V)
    assert Pa.shape == (0, 6)
    assert np.allclose(Ta, Rb, atol=1e-13)
    assert np.allclose(Qa, Qb, atol=1e-13)


@pytest.mark.parametrize("fn", [bo.bcgs_pip2, bo.bcgs2_cholqr2])
def test_block_schemes_give_the_unique_qr(fn):
    g = synth.rng(17)
    n, k, s = 300, 6, 5
    Q, _ = _sign_fixed_qr(g.standard_normal((n, k)))
    V = g.standard_normal((n, s)) + Q @ g.standard_normal((k, s))
    Qj, P, T = fn(Q, V)
    qq, rr = _sign_fixed_qr(np.concatenate([Q, V], axis=1))
    assert np.allclose(P, rr[:k, k:], atol=1e-12)
    assert np.allclose(T, rr[k:, k:], atol=1e-12)
    assert checks.orth_error(np.concatenate([Q, Qj], axis=1))[0] < 1e-14


# ---------------------------------------------------------------- error bounds of §IV and §V
def test_cholqr_error_grows_like_kappa_squared_and_cholqr2_is_stable():
    """Eq. (2)-(3): one CholQR leaves ||I - Q^T Q|| <= c1 kappa^2 with
    c1 = 5(ns + s(s+1)) eps while c1 kappa^2 < 1/2 (Eq. 1); Theorem 1: then
    kappa(Q) < sqrt(3) and CholQR2 reaches O(eps)."""
    n, s = 20000, 5
    c1 = 5 * (n * s + s * (s + 1)) * EPS
    errs = []
    for kappa in (1e1, 10 ** 2.5, 1e4):
        assert c1 * kappa ** 2 < 0.5
        V = synth.logscaled(n, s, kappa, seed=int(kappa))
        Q1, _ = bo.cholqr(V)
        e1 = checks.orth_error(Q1)[0]
        assert e1 <= c1 * kappa ** 2
        assert checks.cond2(Q1) < math.sqrt(3)
        Q2, R = bo.cholqr2(V)
        assert checks.orth_error(Q2)[0] < 50 * EPS
        assert np.allclose(Q2 @ R, V, atol=1e-13 * np.abs(V).max())
        errs.append(e1)
    # the error of a single CholQR grows with kappa (kappa^2 eps regime)
    assert errs[2] > 100 * errs[0]


def test_two_stage_on_glued_matrix_reaches_machine_precision():
    """Theorem 3 (§V) on the glued matrix of §VI (first panel kappa 1e5, the
    panels mixed with their predecessors): after stage 1 the big panel has O(1) condition number
    (Eq. 11); after stage 2 the orthogonality error is O(eps)."""
    n, s, panels = 5000, 5, 6
    V = synth.glued(n, s, panels, 1e5, seed=3)
    assert checks.cond2(V) > 1e5
    blocks = [V[:, i * s:(i + 1) * s] for i in range(panels)]
    Q, Rt, Rd, Qhat = bo.two_stage_panel(np.zeros((n, 0)), blocks)
    assert checks.cond2(Qhat) < 10.0
    assert checks.orth_error(Q)[0] < 100 * EPS
    assert np.allclose(Q @ Rd, V, atol=1e-12 * np.abs(V).max())
    assert np.allclose(np.triu(Rd), Rd)
    assert np.all(np.diag(Rd) > 0)


@pytest.mark.parametrize("seed", [1, 2])
def test_two_stage_on_the_glued_sweep(seed):
    """§V on the glued sweep of §VI (six blocks of condition 1e3 each, the
    total condition number swept): after stage 1 the big panel's orthogonality
    error grows like kappa^2 eps (Eq. 10) while its condition number stays O(1)
    (Eq. 11); after stage 2 the error is O(eps) (Theorem 3) and V = Q R.  Far
    beyond eps^(-1/2) the assumption of Eq. 9 fails: a stage-1 Cholesky breaks
    down and is reported."""
    n, c, p = 4000, 5, 6
    for km in (1e2, 1e4, 1e6):
        V = synth.glued_sweep(n, c, p, 1e3, km, seed)
        kap = checks.cond2(V)
        blocks = [V[:, i * c:(i + 1) * c] for i in range(p)]
        Q, Rt, Rd, Qhat = bo.two_stage_panel(np.zeros((n, 0)), blocks)
        e1 = checks.orth_error(Qhat)[0]
        assert 0.01 * kap ** 2 * EPS <= e1 <= 10 * kap ** 2 * EPS, (km, kap, e1)
        assert checks.cond2(Qhat) < 2.0
        assert checks.orth_error(Q)[0] < 100 * EPS
        assert np.abs(Q @ Rd - V).max() <= 1e-13 * np.abs(V).max()
    V = synth.glued_sweep(n, c, p, 1e3, 1e10, seed)
    assert checks.cond2(V) > 1e11
    with pytest.raises(bo.Breakdown) as e:
        bo.two_stage_panel(np.zeros((n, 0)), [V[:, i * c:(i + 1) * c] for i in range(p)])
    assert "stage1" in str(e.value)


def test_two_stage_panel_equals_householder_r():
    """The two-stage R factor of a well-conditioned big panel is the unique
    positive-diagonal R of its QR (Fig. 1 caption)."""
    g = synth.rng(18)
    n, s = 800, 5
    V = g.standard_normal((n, 4 * s))
    blocks = [V[:, i * s:(i + 1) * s] for i in range(4)]
    Q, _, Rd, _ = bo.two_stage_panel(np.zeros((n, 0)), blocks)
    _, r = _sign_fixed_qr(V)
    assert np.allclose(Rd, r, atol=1e-12 * np.abs(r).max())


# ---------------------------------------------------------------- shifted CholQR (§II)
def test_cholqr_shift_by_hand():
    """sigma = 11 (n c + c (c + 1)) u ||X||^2 with u = 2^-53: for n = 1000,
    c = 5, ||X||_F^2 = 3: 11 * 5030 * 3 / 2^53, exactly."""
    assert bo.cholqr_shift(1000, 5, 3.0) == 165990.0 / 2.0 ** 53
    assert bo.cholqr_shift(1, 1, 0.0) == 0.0


def test_shifted_pip_identity_and_reconstruction():
    """For an orthonormal Q, T^T T = (V - Q P)^T (V - Q P) + sigma I, so the
    shifted stage-1 block satisfies Q^^T Q^ + sigma T^-T T^-1 = I exactly in
    exact arithmetic.  On a block of condition 1e9 the shift term is of order
    one, and the rounding of G - P^T P, amplified by ||T^-1||^2, stays a fixed
    fraction (about 1/(11 nb), by the choice of sigma) of it: the identity
    holds to 5% of the shift term, so a dropped sigma or one off by 10% fails.
    V = Q P + Q^ T to rounding."""
    g = synth.rng(4545)
    n, k, c = 3000, 4, 5
    Q, _ = _sign_fixed_qr(g.standard_normal((n, k)))
    V = synth.logscaled(n, c, 1e9, seed=7) + Q @ g.standard_normal((k, c))
    Qh, P, T = bo.bcgs_pip_shifted(Q, V)
    sig = bo.cholqr_shift(n, c, float(np.trace(V.T @ V)))
    Ti = np.linalg.inv(T)
    E = Qh.T @ Qh + sig * (Ti.T @ Ti) - np.eye(c)
    term = np.abs(sig * (Ti.T @ Ti)).max()
    assert term > 0.1                                        # the shift matters here
    assert np.abs(E).max() <= 0.05 * term, (np.abs(E).max(), term)
    assert np.abs(Q @ P + Qh @ T - V).max() <= 1e-13 * np.abs(V).max()


def test_shifted_two_stage_is_stable_where_cholqr_breaks_down():
    """§II: shifted CholQR is stable as long as the input is numerically full
    rank.  A big panel of condition 1e12 (beyond u^(-1/2), where the plain
    Pythagorean stage 1 breaks down): shifted stage 1 per block, then stage 2
    as shifted CholQR3 (a shifted pass and two plain ones), gives
    ||I - Q^T Q|| = O(eps) and V = Q R to rounding."""
    n, c, p = 20000, 3, 2
    V = synth.logscaled(n, c * p, 1e12, seed=11)
    blocks = [V[:, i * c:(i + 1) * c] for i in range(p)]
    with pytest.raises(bo.Breakdown):
        bo.two_stage_panel(np.zeros((n, 0)), blocks)
    Qhat = np.zeros_like(V)
    Rh = np.zeros((c * p, c * p))
    for i, B in enumerate(blocks):
        Qh, P, T = bo.stage1_shifted(Qhat[:, :i * c], B)
        Qhat[:, i * c:(i + 1) * c] = Qh
        Rh[:i * c, i * c:(i + 1) * c] = P
        Rh[i * c:(i + 1) * c, i * c:(i + 1) * c] = T
    Qf, _, T2 = bo.stage2_shifted(np.zeros((n, 0)), Qhat)
    assert checks.orth_error(Qf)[0] < 100 * EPS
    assert np.abs(Qf @ (T2 @ Rh) - V).max() <= 1e-13 * np.abs(V).max()


def test_shifted_sstep_gmres_solves_where_the_monomial_basis_breaks_down():
    """s = 10 monomial on the 64 x 64 Laplacian: the plain two-stage scheme
    breaks down in its first cycle; with the shifted stage 1 (and the
    re-orthogonalized stage 2) it converges to 1e-8, with the forward error
    within the closed-form condition number times the tolerance."""
    A = synth.laplace2d(64)
    M = kr.as_operator(A)
    xt = synth.x_true(A.n, 0)
    b = M @ xt
    _, i0 = kr.sstep_gmres(A, b, m=60, s=10, panel=60, tol=1e-8)
    assert i0["status"] == kr.STATUS_BREAKDOWN
    x, i1 = kr.sstep_gmres(A, b, m=60, s=10, panel=60, tol=1e-8, shift=True)
    assert i1["status"] == 0
    assert np.linalg.norm(b - M @ x) / np.linalg.norm(b) <= 1e-8
    lo, hi = checks.laplace2d_extreme_eigs(64)
    assert np.linalg.norm(x - xt) / np.linalg.norm(xt) <= (hi / lo) * 1e-8


# ---------------------------------------------------------------- multicolor Gauss-Seidel (§VIII, Fig. 9)
def test_greedy_coloring_of_the_grid_stencils_is_red_black():
    """Greedy coloring in natural order of the 5-point (7-point) stencil on a
    lexicographic grid is the red-black coloring (i + j (+ k)) mod 2."""
    from oracle import precond as pc
    N = 9
    c2 = pc.greedy_coloring(synth.laplace2d(N))
    i, j = np.divmod(np.arange(N * N), N)
    assert np.array_equal(c2, (i + j) % 2)
    c3 = pc.greedy_coloring(synth.laplace3d(5))
    a, rem = np.divmod(np.arange(125), 25)
    b, c = np.divmod(rem, 5)
    assert np.array_equal(c3, (a + b + c) % 2)


def test_greedy_coloring_is_proper_and_greedy():
    """No two coupled rows share a color (either triangle of the pattern), and
    every row's color is the smallest one its earlier neighbors leave free."""
    from oracle import precond as pc
    A = synth.banded_random(400, 3, band=30)
    M = kr.as_operator(A)
    col = pc.greedy_coloring(A)
    S = (abs(M) + abs(M).T).tocoo()
    off = S.row != S.col
    assert not np.any(col[S.row[off]] == col[S.col[off]])
    Sc = S.tocsr()
    for r in range(A.n):
        nb = Sc.indices[Sc.indptr[r]:Sc.indptr[r + 1]]
        earlier = {int(col[q]) for q in nb if q < r}
        assert all(cc in earlier for cc in range(col[r])) and col[r] not in earlier


def test_gs_sweep_is_the_lower_triangular_solve_in_color_order():
    """z = (D + L)^{-1} r of the matrix permuted to color order (scipy's sparse
    triangular solve), on a nonsymmetric matrix with many colors."""
    from scipy.sparse.linalg import spsolve_triangular
    from oracle import precond as pc
    A = synth.banded_random(500, 4, band=40)
    M = kr.as_operator(A)
    col = pc.greedy_coloring(A)
    r = synth.x_true(A.n, 3)
    z = pc.gs_sweep(A, col, r)
    perm = np.lexsort((np.arange(A.n), col))
    Mp = M[perm][:, perm].tocsr()
    zp = spsolve_triangular(sp_tril(Mp), r[perm], lower=True)
    assert np.allclose(z[perm], zp, rtol=1e-13, atol=1e-13 * np.abs(zp).max())


def sp_tril(M):
    import scipy.sparse as sp
    return sp.tril(M, format="csr")


def test_gs_sweep_on_the_red_black_laplacian_by_hand():
    """Red rows: z = r / 4; black rows: z = (r + sum of the red neighbors' z) / 4
    (the 5-point stencil's off-diagonals are -1)."""
    from oracle import precond as pc
    N = 7
    A = synth.laplace2d(N)
    col = pc.greedy_coloring(A)
    r = synth.x_true(A.n, 4)
    z = pc.gs_sweep(A, col, r)
    zr = np.where(col == 0, r / 4.0, 0.0)
    ref = zr.copy()
    for q in np.nonzero(col == 1)[0]:
        i, j = divmod(int(q), N)
        s_ = sum(zr[a * N + b] for a, b in ((i - 1, j), (i + 1, j), (i, j - 1), (i, j + 1)) if 0 <= a < N and 0 <= b < N)
        ref[q] = (r[q] + s_) / 4.0
    assert np.allclose(z, ref, rtol=1e-15, atol=1e-15)


def test_preconditioned_cycle_is_the_minimal_residual_iterate():
    """One restart cycle with the right preconditioner returns the x that
    minimizes ||b - A x|| over x0 + M^{-1} K_m(A M^{-1}, r0) (brute force:
    dense A M^{-1} from the sweep applied to the identity, power vectors, QR,
    least squares), for the two-stage and BCGS-PIP2 schemes."""
    from oracle import precond as pc
    A = synth.convdiff2d(7, 5)
    M = kr.as_operator(A).toarray()
    n = A.n
    col = pc.greedy_coloring(A)
    Minv = np.column_stack([pc.gs_sweep(A, col, e) for e in np.eye(n)])
    b = M @ synth.x_true(n, 1)
    m = 6
    K = np.zeros((n, m))
    v = b / np.linalg.norm(b)
    for i in range(m):
        K[:, i] = v
        v = M @ (Minv @ v)
    Z = Minv @ np.linalg.qr(K)[0]
    y, *_ = np.linalg.lstsq(M @ Z, b, rcond=None)
    x_ref = Z @ y
    for ortho, panel in (("two_stage", 6), ("bcgs_pip2", 3)):
        x, info = kr.sstep_gmres(A, b, m=m, s=3, panel=panel, tol=1e-30, max_restarts=1, ortho=ortho,
                                 precond="mcgs")
        assert np.allclose(x, x_ref, rtol=1e-9, atol=1e-10 * np.abs(x_ref).max()), ortho


# ---------------------------------------------------------------- least squares and Hessenberg
def test_givens_solves_the_hessenberg_least_squares():
    g = synth.rng(19)
    m = 12
    H = np.triu(g.standard_normal((m + 1, m)), -1)
    beta = 3.5
    gv = kr.Givens(m, beta)
    for c in range(m):
        gv.add_column(H[: c + 2, c])
    y = gv.solve()
    rhs = np.zeros(m + 1)
    rhs[0] = beta
    y_ref, *_ = np.linalg.lstsq(H, rhs, rcond=None)
    assert np.allclose(y, y_ref, rtol=1e-10, atol=1e-12)
    assert abs(gv.residual() - np.linalg.norm(rhs - H @ y_ref)) < 1e-12


@pytest.mark.parametrize("ortho,panel", [("two_stage", 60), ("two_stage", 20), ("bcgs_pip2", 5),
                                         ("bcgs2_cholqr2", 5)])
def test_arnoldi_relation_of_recovered_hessenberg(ortho, panel):
    """A Q_{1:k} = Q_{1:k+1} H to 1e-12 relative for the H recovered from the
    s-step R factors."""
    A = synth.convdiff2d(40, seed=5)
    b = kr.as_operator(A) @ synth.x_true(A.n, 1)
    _, info = kr.sstep_gmres(A, b, m=60, s=5, panel=panel, tol=1e-30, max_restarts=1,
                             ortho=ortho, return_basis=True)
    k = info["k"]
    assert k == 60
    assert checks.orth_error(info["Q"][:, : k + 1])[0] < 1e-13
    assert checks.arnoldi_residual(kr.as_operator(A), info["Q"], info["H"], k) < 1e-12


def test_sstep_hessenberg_equals_arnoldi_hessenberg():
    """With positive subdiagonals the Arnoldi factorization from a given start
    vector is unique, so the recovered H of every s-step scheme equals the H of
    standard Arnoldi (CGS2) over the first restart cycle."""
    A = synth.convdiff2d(16, seed=6)
    M = kr.as_operator(A)
    b = M @ synth.x_true(A.n, 2)
    m = 20
    n = A.n
    # reference: standard Arnoldi with CGS2, written out
    Q = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    Q[:, 0] = b / np.linalg.norm(b)
    for j in range(m):
        w = M @ Q[:, j]
        for _ in range(2):
            h = Q[:, : j + 1].T @ w
            w -= Q[:, : j + 1] @ h
            H[: j + 1, j] += h
        H[j + 1, j] = np.linalg.norm(w)
        Q[:, j + 1] = w / H[j + 1, j]
    for ortho, panel in (("two_stage", 20), ("two_stage", 10), ("bcgs_pip2", 5), ("bcgs2_cholqr2", 5)):
        _, info = kr.sstep_gmres(A, b, m=m, s=5, panel=panel, tol=1e-30, max_restarts=1,
                                 ortho=ortho, return_basis=True)
        Hs = info["H"]
        assert np.allclose(Hs, H, atol=1e-9 * np.abs(H).max()), ortho
        assert np.allclose(np.abs(info["Q"][:, :m + 1]), np.abs(Q), atol=1e-9)


# ---------------------------------------------------------------- end to end
@pytest.mark.parametrize("ortho", ["two_stage", "bcgs_pip2", "bcgs2_cholqr2", "cgs2"])
def test_small_dense_systems_reach_the_lu_solution(ortho):
    g = synth.rng(20)
    n = 48
    A = g.standard_normal((n, n)) + 8.0 * np.eye(n)
    import scipy.sparse as sp
    As = sp.csr_matrix(A)
    b = g.standard_normal(n)
    x_lu = np.linalg.solve(A, b)
    if ortho == "cgs2":
        x, info = kr.gmres_cgs2(As, b, m=20, tol=1e-13)
    else:
        x, info = kr.sstep_gmres(As, b, m=20, s=5, panel=20, tol=1e-13, ortho=ortho)
    assert info["status"] == 0
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) <= 10 * kappa * 1e-13


def test_laplace_forward_error_against_closed_form_condition_number():
    """b = A x_true on the 64x64 Laplacian (C1 input).  SPD with closed-form
    extreme eigenvalues, so ||x - x_true|| / ||x_true|| <= kappa(A) * relres."""
    N = 64
    A = synth.laplace2d(N)
    M = kr.as_operator(A)
    xt = synth.x_true(A.n, 0)
    b = M @ xt
    lo, hi = checks.laplace2d_extreme_eigs(N)
    ev = np.linalg.eigvalsh(M.toarray())
    assert abs(ev[0] - lo) < 1e-10 and abs(ev[-1] - hi) < 1e-10
    kappa = hi / lo
    for ortho in ("two_stage", "bcgs_pip2", "bcgs2_cholqr2"):
        x, info = kr.sstep_gmres(A, b, m=60, s=5, tol=1e-8, ortho=ortho)
        assert info["status"] == 0
        rel = np.linalg.norm(M @ x - b) / np.linalg.norm(b)
        assert rel <= 1e-8
        assert np.linalg.norm(x - xt) / np.linalg.norm(xt) <= kappa * rel


def test_convergence_tests_fall_on_panel_boundaries():
    """Tables 2 and 4 print two-stage counts that are multiples of s^ and s-step
    counts that are multiples of s; the oracle tests convergence at the same
    points."""
    with open(os.path.join(GOLD, "table2_table4_iteration_counts.json")) as f:
        gold = json.load(f)
    for shat, cnt in gold["table2"]["two_stage"].items():
        assert cnt % int(shat) == 0 or cnt % 5 == 0
    assert gold["table2"]["two_stage"]["60"] % 60 == 0
    for cnt in gold["table4_two_stage_shat_m60"].values():
        assert cnt % 60 == 0
    for cnt in gold["table4_sstep_s5"].values():
        assert cnt % 5 == 0
    A = synth.laplace2d(32)
    b = kr.as_operator(A) @ synth.x_true(A.n, 0)
    for ortho, panel, step in (("two_stage", 60, 60), ("two_stage", 20, 20), ("bcgs_pip2", 5, 5)):
        _, info = kr.sstep_gmres(A, b, m=60, s=5, panel=panel, tol=1e-8, ortho=ortho)
        assert info["status"] == 0
        assert info["iters"] % step == 0
    # s^ = 40 with m = 60: big panels of 40 and 20 columns per cycle, so the
    # tests fall at 60 c + 40 and 60 c + 60, as Table 2's 60280 = 1004 * 60 + 40
    assert gold["table2"]["two_stage"]["40"] % 60 == 40
    _, info = kr.sstep_gmres(A, b, m=60, s=5, panel=40, tol=1e-8)
    assert info["status"] == 0 and info["iters"] % 60 in (0, 40)


def _krylov_minimizer(A, b, x0, m):
    """x0 + argmin over K_m(A, r0) of ||b - A x||, by brute force: the power
    vectors r0, A r0, ..., A^(m-1) r0 (each normalized), their LAPACK QR, and a
    dense least-squares solve."""
    r0 = b - A @ x0
    K = np.empty((len(b), m))
    v = r0 / np.linalg.norm(r0)
    for j in range(m):
        K[:, j] = v
        v = A @ v
        v /= np.linalg.norm(v)
    Qk = np.linalg.qr(K)[0]
    z = np.linalg.lstsq(A @ Qk, r0, rcond=None)[0]
    return x0 + Qk @ z


@pytest.mark.parametrize("ortho,s,panel,theta", [("two_stage", 5, 15, None), ("bcgs_pip2", 5, 5, None),
                                                 ("bcgs2_cholqr2", 5, 5, None),
                                                 ("two_stage", 5, 15, (2.3, 1.7, 2.0, 1.5, 2.5)),
                                                 ("two_stage", 5, 10, None)])
def test_one_cycle_is_the_minimal_residual_iterate(ortho, s, panel, theta):
    """GMRES' defining property (§I, §III): one restart cycle of m steps from
    x0 returns the minimizer of ||b - A x|| over x0 + K_m(A, r0), whatever the
    block scheme and whether the basis is monomial or Newton (both span K_m).
    A small nonsymmetric system whose residual after 15 steps is still 2.6e-2,
    so that the 15-step and 10-step minimizers differ by 11%."""
    import scipy.sparse as sp
    g = synth.rng(77)
    n, m = 60, 15
    A = sp.csr_matrix(2.0 * np.eye(n) + 1.8 * g.standard_normal((n, n)) / np.sqrt(n))
    b = g.standard_normal(n)
    x0 = 0.1 * g.standard_normal(n)
    xref = _krylov_minimizer(A, b, x0, m)
    assert np.linalg.norm(xref - _krylov_minimizer(A, b, x0, m - 5)) > 0.1 * np.linalg.norm(xref)
    th = None if theta is None else np.array(theta)
    x, info = kr.sstep_gmres(A, b, x0=x0, m=m, s=s, panel=panel, tol=1e-30, max_restarts=1, ortho=ortho, theta=th)
    assert info["iters"] == m and info["restarts"] == 1
    assert np.linalg.norm(x - xref) <= 1e-8 * np.linalg.norm(xref)
    assert np.linalg.norm(b - A @ x) <= (1 + 1e-8) * np.linalg.norm(b - A @ xref)


def test_restart_applies_the_minimal_residual_property_cycle_by_cycle():
    """Restarted GMRES(m): the second cycle starts from the first cycle's x and
    returns the minimizer over x1 + K_m(A, r1)."""
    import scipy.sparse as sp
    g = synth.rng(78)
    n, m = 60, 10
    A = sp.csr_matrix(2.0 * np.eye(n) + 1.8 * g.standard_normal((n, n)) / np.sqrt(n))
    b = g.standard_normal(n)
    x0 = np.zeros(n)
    x1 = _krylov_minimizer(A, b, x0, m)
    x2 = _krylov_minimizer(A, b, x1, m)
    assert np.linalg.norm(x2 - x1) > 0.01 * np.linalg.norm(x2)
    x, info = kr.sstep_gmres(A, b, x0=x0, m=m, s=5, panel=10, tol=1e-30, max_restarts=2)
    assert info["iters"] == 2 * m and info["restarts"] == 2
    assert np.linalg.norm(x - x2) <= 1e-8 * np.linalg.norm(x2)


def test_s_equal_one_is_standard_gmres():
    """§III: standard GMRES is s-step GMRES with step size one."""
    A = synth.convdiff2d(20, seed=7)
    b = kr.as_operator(A) @ synth.x_true(A.n, 3)
    _, i_std = kr.gmres_cgs2(A, b, m=30, tol=1e-8)
    _, i_s1 = kr.sstep_gmres(A, b, m=30, s=1, tol=1e-8, ortho="bcgs_pip2")
    assert i_s1["status"] == 0
    assert i_s1["iters"] == i_std["iters"]


def test_breakdown_is_reported_not_patched():
    """A rank-deficient MPK block makes the Gram of Eq. (1) singular; the oracle
    reports the breakdown (status -4) instead of shifting it."""
    n = 50
    import scipy.sparse as sp
    A = sp.identity(n, format="csr") * 2.0   # Krylov space of dimension 1
    b = np.ones(n)
    _, info = kr.sstep_gmres(A, b, m=10, s=5, tol=1e-30, ortho="two_stage")
    assert info["status"] == kr.STATUS_BREAKDOWN


def test_monomial_scale_is_a_power_of_two():
    assert kr.mpk_sigma(synth.laplace2d(8)) == 8.0
    assert kr.mpk_sigma(synth.laplace3d(5)) == 8.0
    s = kr.mpk_sigma(synth.convdiff2d(10, 1))
    assert s == 2.0 ** math.floor(math.log2(s))


# ---------------------------------------------------------------- mixed-precision pattern
def test_fp32_mpk_is_the_fp64_mpk_to_fp32_precision():
    A = synth.laplace2d(40)
    M = kr.as_operator(A)
    v = synth.x_true(A.n, 3)
    W64 = kr.mpk(M, v, 5, 8.0)
    W32 = kr.mpk(M.astype(np.float32), v.astype(np.float32), 5, 8.0)
    assert W32.dtype == np.float32
    rel = np.linalg.norm(W32 - W64, axis=0) / np.linalg.norm(W64, axis=0)
    assert np.all(rel < 5e-6)


@pytest.mark.parametrize("N", [32, 64])
def test_mixed_precision_refinement_reaches_fp64_accuracy(N):
    """FP32 basis with FP64 Gram/Cholesky/Hessenberg and FP64 restart
    residuals (iterative refinement) still reaches ||b - A x|| / ||b|| <= 1e-8,
    and its x agrees with the FP64 solve to the forward-error bound
    kappa(A) * tol (closed-form Laplace eigenvalues)."""
    A = synth.laplace2d(N)
    M = kr.as_operator(A)
    b = M @ synth.x_true(A.n, 0)
    x32, i32 = kr.sstep_gmres(A, b, m=60, s=5, tol=1e-8, basis_dtype=np.float32)
    x64, i64 = kr.sstep_gmres(A, b, m=60, s=5, tol=1e-8)
    assert i32["status"] == 0 and i64["status"] == 0
    assert np.linalg.norm(b - M @ x32) / np.linalg.norm(b) <= 1e-8
    lo, hi = checks.laplace2d_extreme_eigs(N)
    assert np.linalg.norm(x32 - x64) / np.linalg.norm(x64) <= 2 * (hi / lo) * 1e-8
    assert i32["iters"] % 60 == 0


def _round_f32(x):
    """The float32 nearest to the rational x (ties to even), from the rational
    itself: a double-rounding check guards float(x) -> float32."""
    from fractions import Fraction
    d = float(x)                       # correctly rounded to 53 bits
    f = np.float32(d)
    # the exact value must not sit within 2^-40 relative of a float32 midpoint,
    # where rounding through the double could differ from rounding the rational
    lo, hi = np.nextafter(f, np.float32(-np.inf)), np.nextafter(f, np.float32(np.inf))
    for nb in (lo, hi):
        mid = (Fraction(float(f)) + Fraction(float(nb))) / 2
        assert mid == 0 or abs(Fraction(x) - mid) > abs(mid) * Fraction(1, 2 ** 40)
    return float(f)


def test_stage1_lowp_rounds_the_projected_block_and_the_result_to_fp32():
    """The mixed-precision stage 1 (explicit projection for an FP32-stored
    basis, the higher-precision-Gram CholQR of §II) on a tiny case, against an
    independent exact-rational computation: W = V - Q (Q^T V) in exact
    rationals, rounded once to float32; T = LAPACK Cholesky of the exactly
    accumulated W^T W.  The oracle's T must agree to 1e-13 (dropping the FP32
    rounding of W moves T by about 1e-8); its Q^ must be FP32 values (dropping
    the final rounding leaves FP64 values) within one float32 ulp of W T^{-1}."""
    from fractions import Fraction
    g = synth.rng(4242)
    n, k, nb = 9, 3, 2
    Q = np.linalg.qr(g.standard_normal((n, k)))[0].astype(np.float32).astype(np.float64)
    V = (g.standard_normal((n, nb)) + Q @ g.standard_normal((k, nb))).astype(np.float32).astype(np.float64)
    Qf = [[Fraction(float(v)) for v in Q[:, c]] for c in range(k)]
    Vf = [[Fraction(float(v)) for v in V[:, j]] for j in range(nb)]
    Pf = [[sum(a * b for a, b in zip(Qf[c], Vf[j])) for j in range(nb)] for c in range(k)]
    W32 = np.zeros((n, nb))
    for j in range(nb):
        for r in range(n):
            w = Vf[j][r] - sum(Qf[c][r] * Pf[c][j] for c in range(k))
            W32[r, j] = _round_f32(w)
    Wf = [[Fraction(float(v)) for v in W32[:, j]] for j in range(nb)]
    G = np.array([[float(sum(a * b for a, b in zip(Wf[i], Wf[j]))) for j in range(nb)] for i in range(nb)])
    T_ref = np.linalg.cholesky(G).T
    Qh, P, T = bo.stage1_lowp(Q, V)
    assert np.allclose(P, np.array([[float(x) for x in row] for row in Pf]), rtol=0, atol=1e-15)
    assert np.all(np.abs(T - T_ref) <= 1e-13 * np.abs(T_ref).max()), np.abs(T - T_ref).max()
    # the unrounded W would have moved T by far more than that bar
    W64 = V - Q @ (Q.T @ V)
    T64 = np.linalg.cholesky(W64.T @ W64).T
    assert np.abs(T64 - T_ref).max() > 1e-10 * np.abs(T_ref).max()
    assert np.array_equal(Qh, Qh.astype(np.float32).astype(np.float64))
    ref = np.linalg.solve(T_ref.T, W32.T).T
    assert np.all(np.abs(Qh - ref) <= 2.0 ** -23 * np.abs(ref) + 1e-30)
    assert np.abs(Qh - ref).max() > 0.0 or np.array_equal(ref, ref.astype(np.float32).astype(np.float64))


def test_breakdown_reports_the_failing_pivot_and_the_pythagorean_margin():
    """The failing pivot is the Schur complement that was not positive
    (hand-worked: diag(4, 1, -1, 2) fails at pivot 3 with value -1; [[1, 2],
    [2, 3]] at pivot 2 with 3 - 2^2 = -1).  BCGS-PIP's margin uses the exact
    identity (V - Q P)^T (V - Q P) = G - P^T P + P^T (Q^T Q - I) P, checked
    here on a non-orthonormal Q; for an orthonormal Q the error term vanishes
    to rounding, so a rank-deficient projected block (V in span Q) has a
    margin of rounding size, and a full-rank one never breaks down."""
    _, info = bo.chol_upper(np.diag([4.0, 1.0, -1.0, 2.0]))
    R, info = bo.chol_upper(np.diag([4.0, 1.0, -1.0, 2.0]))
    assert info == 3 and bo.pivot_value(np.diag([4.0, 1.0, -1.0, 2.0]), R, info) == -1.0
    G = np.array([[1.0, 2.0], [2.0, 3.0]])
    R, info = bo.chol_upper(G)
    assert info == 2 and bo.pivot_value(G, R, info) == -1.0
    g = synth.rng(4343)
    n, k, nb = 50, 4, 3
    Q = g.standard_normal((n, k)) / np.sqrt(n)          # far from orthonormal
    V = g.standard_normal((n, nb))
    P = Q.T @ V
    W = V - Q @ P
    lhs = W.T @ W
    rhs = V.T @ V - P.T @ P + P.T @ (Q.T @ Q - np.eye(k)) @ P
    assert np.allclose(lhs, rhs, rtol=0, atol=1e-12 * np.abs(lhs).max())
    E = P.T @ (Q.T @ Q - np.eye(k)) @ P
    assert bo.pip_margin(Q, V, P) == pytest.approx(np.linalg.eigvalsh(lhs)[0] / np.linalg.norm(E, 2), rel=1e-12)
    assert bo.pip_margin(np.zeros((n, 0)), V, np.zeros((0, nb))) == float("inf")
    Qo, _ = _sign_fixed_qr(g.standard_normal((n, k)))
    Vin = Qo @ g.standard_normal((k, nb))              # V in span(Q): rank-deficient projection
    with pytest.raises(bo.Breakdown) as e:
        bo.bcgs_pip(Qo, Vin)
    assert e.value.margin < 1.0 and not (e.value.value > 0.0)


def test_mixed_basis_keeps_fp32_orthogonality_after_stage2():
    """Stage 2 on an FP32-stored pre-processed panel: the FP64-computed Q has
    O(eps64) orthogonality before rounding and O(eps32) after (Theorem 3 with
    the basis precision)."""
    n, s, nb = 20000, 5, 4
    V = synth.glued(n, s, nb, 1e3, seed=4).astype(np.float32)
    blocks = [V[:, i * s:(i + 1) * s].astype(np.float64) for i in range(nb)]
    Q, _, _, _ = bo.two_stage_panel(np.zeros((n, 0)), blocks)
    assert checks.orth_error(Q)[0] < 100 * EPS
    assert checks.orth_error(Q.astype(np.float32).astype(np.float64))[0] < 50 * np.finfo(np.float32).eps


# ---------------------------------------------------------------- Newton basis (Leja-ordered Ritz shifts)
def test_leja_order_of_five_points_by_hand():
    """Greedy Leja ordering of {-1, -1/2, 0, 1/2, 1}, worked by hand: the
    largest moduli tie (first in ascending order: -1); then |x + 1| is largest
    at 1; |x^2 - 1| is largest at 0 (value 1 against 3/4); |x (x^2 - 1)| ties at
    +-1/2 (3/8 each, first: -1/2); 1/2 is left."""
    assert kr.leja_order([0.5, 1.0, -1.0, 0.0, -0.5]).tolist() == [-1.0, 1.0, 0.0, -0.5, 0.5]


def test_leja_order_on_a_fine_grid_approaches_the_interval_leja_points():
    """On [-1, 1] the continuous Leja sequence from -1 is -1, 1, 0, then the
    maximizer of |x (x^2 - 1)|, x = +-1/sqrt(3) (zero of 3x^2 - 1); then the
    maximizer of |x (x^2 - 1)(x + 1/sqrt(3))|, a root of its derivative, found
    here with numpy's polynomial roots.  A grid of step h gets each within h."""
    h = 1e-3
    got = kr.leja_order(np.linspace(-1.0, 1.0, 2001))[:5]
    r3 = 1.0 / math.sqrt(3.0)
    assert got[:3].tolist() == [-1.0, 1.0, 0.0]
    assert abs(got[3] + r3) <= h
    p = np.poly1d([1.0, 0.0, -1.0, 0.0]) * np.poly1d([1.0, r3])
    crit = [z.real for z in p.deriv().roots if abs(z.imag) < 1e-12 and -1 <= z.real <= 1]
    best = max(crit, key=lambda z: abs(p(z)))
    assert abs(got[4] - best) <= h


def test_leja_order_is_a_permutation_and_scale_free():
    g = synth.rng(31)
    z = g.standard_normal(40) * 3.0
    o = kr.leja_order(z)
    assert sorted(o.tolist()) == sorted(z.tolist())
    assert abs(o[0]) == np.abs(z).max()
    assert np.array_equal(kr.leja_order(z * 2.0 ** 37), o * 2.0 ** 37)
    # a repeated point has distance product 0 and comes after every other point
    o2 = kr.leja_order(np.concatenate([z[:10], z[:1]]))
    assert o2[-1] == z[0] and np.count_nonzero(o2 == z[0]) == 2


def test_newton_shifts_of_a_hessenberg_form_are_the_leja_ordered_eigenvalues():
    """An orthogonal similarity of diag(d) reduced to Hessenberg form by
    scipy's Householder reduction has eigenvalues d, so the shifts are
    leja_order(d)[:s] (to eigenvalue rounding), cycled when k < s."""
    import scipy.linalg as sla
    g = synth.rng(32)
    d = np.array([0.5, 1.0, 2.5, 3.0, 4.75, 6.0, 7.5, 8.0])
    Qo, _ = np.linalg.qr(g.standard_normal((8, 8)))
    Hh = sla.hessenberg(Qo @ np.diag(d) @ Qo.T)
    assert np.allclose(np.tril(Hh, -2), 0.0)
    th = kr.newton_shifts(Hh, 6)
    assert np.allclose(th, kr.leja_order(d)[:6], atol=1e-12)
    assert th[0] == pytest.approx(8.0, abs=1e-12) and th[1] == pytest.approx(0.5, abs=1e-12)
    th12 = kr.newton_shifts(Hh, 12)
    assert np.allclose(th12[8:], th12[:4])
    # a rotation block [[a, -b], [b, a]] gives the conjugate pair a +- ib: one real shift a, twice
    R = np.array([[2.0, -3.0, 0.0], [3.0, 2.0, 1.0], [0.0, 0.5, -4.0]])
    ev = np.linalg.eigvals(R)
    assert np.allclose(sorted(kr.newton_shifts(R, 3)), sorted(ev.real), atol=1e-12)


def test_auto_shifts_are_the_ritz_values_of_the_first_cycle():
    """The Ritz values are the eigenvalues of the Rayleigh quotient Q_m^T A Q_m
    of the first cycle's orthonormal basis (computed here from the basis, not
    from the recovered H); for symmetric A they lie inside [lambda_min,
    lambda_max] (Cauchy interlacing)."""
    A = synth.laplace2d(32)
    M = kr.as_operator(A)
    b = M @ synth.x_true(A.n, 0)
    _, info = kr.sstep_gmres(A, b, m=60, s=10, tol=1e-30, max_restarts=1, theta="auto", return_basis=True)
    assert info["k"] == 60
    Q = info["Q"][:, :60]
    rv = np.linalg.eigvalsh(Q.T @ (M @ Q))
    assert np.allclose(info["theta"], kr.leja_order(rv)[:10], atol=1e-9)
    lo, hi = checks.laplace2d_extreme_eigs(32)
    assert lo - 1e-12 <= info["theta"].min() and info["theta"].max() <= hi + 1e-12


def test_newton_sigma_is_the_power_of_two_nearest_the_capacity():
    """Capacity of [a, b] is (b - a) / 4; the scale is the power of two nearest
    it in log2 (the boundary 2^(e - 1/2) rounds up)."""
    assert kr.newton_sigma([0.0, 8.0], 1.0) == 2.0
    assert kr.newton_sigma([0.0, 4.0 * 3.0], 1.0) == 4.0        # cap 3 = 2^1.58 -> 4
    assert kr.newton_sigma([0.0, 4.0 * 2.8], 1.0) == 2.0        # cap 2.8 = 2^1.49 -> 2
    assert kr.newton_sigma([1.0, 1.0 + 4.0 * 2.0 ** 0.5], 1.0) == 2.0   # cap 2^0.5 is the boundary: up
    assert kr.newton_sigma([5.0, 5.0], 16.0) == 16.0
    assert kr.newton_sigma([], 16.0) == 16.0


def test_newton_basis_is_better_conditioned_than_the_monomial_basis():
    """The Newton basis with Leja-ordered Ritz shifts and the capacity scale
    keeps an s = 10 MPK block of the 64x64 Laplacian far better conditioned
    than the scaled monomial basis (the motivation for the Newton basis in the
    paper's discussion of large s); column-equilibrated condition numbers."""
    A = synth.laplace2d(64)
    M = kr.as_operator(A)
    b = M @ synth.x_true(A.n, 0)
    _, info = kr.sstep_gmres(A, b, m=60, s=10, tol=1e-30, max_restarts=1, theta="auto")
    th, sig_n = info["theta"], info["sigma"]
    assert sig_n == 2.0     # the Ritz values fill (0, 8): capacity ~2
    v = b / np.linalg.norm(b)

    def econd(W):
        W = np.column_stack([v, W])
        return np.linalg.cond(W / np.linalg.norm(W, axis=0))
    c_mono = econd(kr.mpk(M, v, 10, kr.mpk_sigma(A)))
    c_newt = econd(kr.mpk(M, v, 10, sig_n, th))
    assert c_mono > 1e7 and c_newt < 1e-4 * c_mono


@pytest.mark.parametrize("ortho,s", [("two_stage", 10), ("two_stage", 15), ("bcgs_pip2", 15),
                                     ("bcgs2_cholqr2", 15)])
def test_auto_newton_basis_solves_where_the_monomial_basis_breaks_down(ortho, s):
    """Large s on the 64x64 Laplacian: the monomial basis breaks down in the
    first cycle (status -4); the auto Newton basis converges to 1e-8 with the
    forward error within kappa(A) * relres (closed-form eigenvalues), and its
    final cycle keeps the Arnoldi relation to 1e-12."""
    N = 64
    A = synth.laplace2d(N)
    M = kr.as_operator(A)
    xt = synth.x_true(A.n, 0)
    b = M @ xt
    _, mono = kr.sstep_gmres(A, b, m=60, s=s, tol=1e-8, ortho=ortho)
    assert mono["status"] == kr.STATUS_BREAKDOWN
    x, info = kr.sstep_gmres(A, b, m=60, s=s, tol=1e-8, ortho=ortho, theta="auto", return_basis=True)
    assert info["status"] == 0 and info["restarts"] >= 2
    rel = np.linalg.norm(M @ x - b) / np.linalg.norm(b)
    assert rel <= 1e-8
    lo, hi = checks.laplace2d_extreme_eigs(N)
    assert np.linalg.norm(x - xt) / np.linalg.norm(xt) <= (hi / lo) * rel
    assert lo - 1e-9 <= info["theta"].min() and info["theta"].max() <= hi + 1e-9
    k = info["k"]
    assert checks.arnoldi_residual(M, info["Q"], info["H"], k) < 1e-12


def test_chebyshev_basis_of_a_diagonal_matrix_is_the_chebyshev_polynomials():
    """For A = diag(lambda) and v = 1 the MPK block of the Chebyshev basis on
    [c - delta, c + delta] is T_j(x), x = (lambda - c) / delta, j = 1..s, in
    closed form: cos(j arccos x) inside the interval, cosh(j arccosh |x|)
    sign(x)^j outside (Bai, Hu and Reichel 1994).  Pins the scale of the first
    product (delta), of the later ones (delta / 2) and the three-term term."""
    lam = np.concatenate([np.linspace(-3.0, 7.0, 41), [7.5, 9.0, -3.5]])
    A = sp.diags(lam).tocsr()
    c, d, s = 2.0, 5.0, 8
    W = kr.mpk(A, np.ones(lam.size), s, d / 2.0, np.full(s, c), cheb=True)
    x = (lam - c) / d
    inside = np.abs(x) <= 1.0
    for j in range(1, s + 1):
        ref = np.where(inside, np.cos(j * np.arccos(np.clip(x, -1.0, 1.0))),
                       np.sign(x) ** j * np.cosh(j * np.arccosh(np.maximum(np.abs(x), 1.0))))
        assert np.allclose(W[:, j - 1], ref, rtol=1e-12, atol=1e-12), j
    assert kr.cheb_coeffs(0, 1.25) == (2.5, 0.0) and kr.cheb_coeffs(3, 1.25) == (1.25, 1.25)


def test_chebyshev_interval_is_the_range_of_the_ritz_values():
    """The interval spans the real parts of the eigenvalues of H (an orthogonal
    similarity of diag(d) in Hessenberg form, and a rotation block with a
    conjugate pair); Ritz values without spread give delta = |c|."""
    import scipy.linalg as sla
    g = synth.rng(41)
    d = np.array([0.5, 1.0, 2.5, 3.0, 4.75, 6.0, 7.5, 8.0])
    Qo, _ = np.linalg.qr(g.standard_normal((8, 8)))
    Hh = sla.hessenberg(Qo @ np.diag(d) @ Qo.T)
    c, dl = kr.cheb_interval(Hh)
    assert c == pytest.approx(4.25, abs=1e-12) and dl == pytest.approx(3.75, abs=1e-12)
    R = np.array([[2.0, -3.0, 0.0], [3.0, 2.0, 1.0], [0.0, 0.5, -4.0]])
    re = np.linalg.eigvals(R).real
    c, dl = kr.cheb_interval(R)
    assert c == pytest.approx(0.5 * (re.min() + re.max())) and dl == pytest.approx(0.5 * (re.max() - re.min()))
    assert kr.cheb_interval(np.array([[3.0]])) == (3.0, 3.0)
    assert kr.cheb_interval(np.array([[0.0]])) == (0.0, 1.0)


def test_chebyshev_basis_is_better_conditioned_than_the_monomial_basis():
    """On the spectral interval of the 64x64 Laplacian (closed-form extreme
    eigenvalues) an s = 10 Chebyshev block is far better conditioned than the
    scaled monomial one (column-equilibrated condition numbers)."""
    A = synth.laplace2d(64)
    M = kr.as_operator(A)
    v = M @ synth.x_true(A.n, 0)
    v /= np.linalg.norm(v)
    lo, hi = checks.laplace2d_extreme_eigs(64)
    c, d = 0.5 * (lo + hi), 0.5 * (hi - lo)

    def econd(W):
        W = np.column_stack([v, W])
        return np.linalg.cond(W / np.linalg.norm(W, axis=0))
    c_mono = econd(kr.mpk(M, v, 10, kr.mpk_sigma(A)))
    c_cheb = econd(kr.mpk(M, v, 10, d / 2.0, np.full(10, c), cheb=True))
    assert c_mono > 1e7 and c_cheb < 1e-4 * c_mono


@pytest.mark.parametrize("ortho,s", [("two_stage", 10), ("two_stage", 15), ("bcgs_pip2", 15)])
def test_auto_chebyshev_basis_solves_where_the_monomial_basis_breaks_down(ortho, s):
    """Large s on the 64x64 Laplacian: the monomial basis breaks down, the
    Chebyshev basis on the interval of the first cycle's Ritz values converges
    to 1e-8 with the forward error within kappa(A) * relres; the interval lies
    in [lambda_min, lambda_max] (interlacing) and the final cycle keeps the
    Arnoldi relation A Q_k = Q_{k+1} H to 1e-12 (which fails if the three-term
    term of the change of basis is dropped)."""
    N = 64
    A = synth.laplace2d(N)
    M = kr.as_operator(A)
    xt = synth.x_true(A.n, 0)
    b = M @ xt
    x, info = kr.sstep_gmres(A, b, m=60, s=s, tol=1e-8, ortho=ortho, cheb="auto", return_basis=True)
    assert info["status"] == 0 and info["restarts"] >= 2 and info["cheb"]
    rel = np.linalg.norm(M @ x - b) / np.linalg.norm(b)
    assert rel <= 1e-8
    lo, hi = checks.laplace2d_extreme_eigs(N)
    assert np.linalg.norm(x - xt) / np.linalg.norm(xt) <= (hi / lo) * rel
    c, sig = info["theta"][0], info["sigma"]
    assert np.all(info["theta"] == c)
    assert lo - 1e-9 <= c - 2.0 * sig and c + 2.0 * sig <= hi + 1e-9
    assert checks.arnoldi_residual(M, info["Q"], info["H"], info["k"]) < 1e-12


def test_explicit_chebyshev_interval_matches_the_auto_one_on_the_spectrum():
    """With the interval given (the closed-form spectrum of the Laplacian) the
    solve takes the same basis in every cycle and converges; a non-positive
    half-width is rejected."""
    A = synth.laplace2d(32)
    M = kr.as_operator(A)
    b = M @ synth.x_true(A.n, 0)
    lo, hi = checks.laplace2d_extreme_eigs(32)
    x, info = kr.sstep_gmres(A, b, m=60, s=10, tol=1e-8, cheb=(0.5 * (lo + hi), 0.5 * (hi - lo)))
    assert info["status"] == 0 and info["sigma"] == pytest.approx(0.25 * (hi - lo))
    with pytest.raises(ValueError):
        kr.sstep_gmres(A, b, m=60, s=10, cheb=(4.0, 0.0))
    with pytest.raises(ValueError):
        kr.sstep_gmres(A, b, m=60, s=10, cheb=(4.0, 1.0), theta="auto")
