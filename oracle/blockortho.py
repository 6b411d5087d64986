"""Block orthogonalization kernels of the paper, FP64, restated from its text.

Oracle (test infrastructure only).  Conventions: column blocks are numpy arrays
of shape (n, c); an "R factor" is upper triangular with a non-negative diagonal
(Fig. 1 caption: BlkOrth returns Q R = V, Q^T Q = I, R upper triangular with
non-negative diagonal).

Cholesky breakdown (a non-positive or NaN pivot) is reported, never patched:
``chol_upper`` returns the 1-based index of the first bad pivot.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular


class Breakdown(Exception):
    """Cholesky of a Gram matrix failed (the Gram is not numerically SPD).

    This is the failure mode excluded by the stability conditions Eq. (1),
    Eq. (5) and Eq. (9) of the paper.  ``pivot`` is 1-based; ``value`` is the
    failing pivot (the Schur complement that was not positive).  A breakdown of
    BCGS-PIP also carries ``margin``: the smallest eigenvalue of the explicitly
    projected block's Gram (V - Q P)^T (V - Q P) over the 2-norm of the
    Pythagorean identity's error P^T (Q^T Q - I) P (§IV-C: G - P^T P equals the
    projected Gram only for an orthonormal Q).  A margin below one means the
    pivot's sign is decided by Q's loss of orthogonality, itself rounding
    amplified by earlier blocks' condition numbers, not by the data."""

    def __init__(self, pivot: int, where: str = "", value: float = float("nan"),
                 margin: float = float("inf")):
        super().__init__(f"Cholesky breakdown at pivot {pivot} {where}")
        self.pivot = pivot
        self.where = where
        self.value = value
        self.margin = margin


def chol_upper(G: np.ndarray):
    """Upper-triangular Cholesky factor R with G = R^T R (Fig. 3 caption: Chol(G)
    returns the upper-triangular factor).  Column-oriented (left-looking)
    textbook loops.  Returns (R, info): info = 0 on success, else the 1-based
    index of the first pivot that is not positive (or NaN)."""
    G = np.asarray(G, dtype=np.float64)
    c = G.shape[0]
    R = np.zeros((c, c))
    for j in range(c):
        for i in range(j):
            R[i, j] = (G[i, j] - np.dot(R[:i, i], R[:i, j])) / R[i, i]
        d = G[j, j] - np.dot(R[:j, j], R[:j, j])
        if not (d > 0.0):  # catches NaN as well
            return R, j + 1
        R[j, j] = np.sqrt(d)
    return R, 0


def pivot_value(G: np.ndarray, R: np.ndarray, info: int) -> float:
    """The failing pivot of ``chol_upper(G)`` that returned (R, info > 0):
    G_jj minus the squares of the column's entries already computed."""
    j = info - 1
    return float(G[j, j] - np.dot(R[:j, j], R[:j, j]))


def pip_margin(Q: np.ndarray, V: np.ndarray, P: np.ndarray) -> float:
    """lambda_min((V - Q P)^T (V - Q P)) / ||P^T (Q^T Q - I) P||_2 (inf for an
    exactly orthonormal or empty Q): how far the projected block is from
    rank deficiency, in units of the error the Pythagorean shortcut of BCGS-PIP
    makes when Q is not orthonormal (only computed on a breakdown)."""
    k = Q.shape[1]
    if k == 0:
        return float("inf")
    W = V - Q @ P
    lmin = float(np.linalg.eigvalsh(W.T @ W)[0])
    E = P.T @ (Q.T @ Q - np.eye(k)) @ P
    en = float(np.linalg.norm(E, 2))
    return float("inf") if en == 0.0 else lmin / en


def right_trsm_upper(V: np.ndarray, R: np.ndarray) -> np.ndarray:
    """V R^{-1} for upper-triangular R (the TRSM of CholQR, §VII)."""
    return solve_triangular(R, V.T, trans="T", lower=False).T


def cholqr(V: np.ndarray, where: str = "cholqr"):
    """CholQR (Fig. 3a): G = V^T V; R = Chol(G); Q = V R^{-1}."""
    G = V.T @ V
    R, info = chol_upper(G)
    if info:
        raise Breakdown(info, where, pivot_value(G, R, info))
    return right_trsm_upper(V, R), R


def cholqr2(V: np.ndarray, where: str = "cholqr2"):
    """CholQR2 (Fig. 3b): CholQR applied twice, R = R2 R1 (§IV-B, Theorem 1)."""
    Q1, R1 = cholqr(V, where + "/1")
    Q, R2 = cholqr(Q1, where + "/2")
    return Q, R2 @ R1


def bcgs(Q: np.ndarray, V: np.ndarray):
    """BCGS inter-block step (Fig. 2a): R_{1:j-1,j} = Q^T V; V^ = V - Q R_{1:j-1,j}."""
    P = Q.T @ V
    return V - Q @ P, P


def bcgs2_cholqr2(Q: np.ndarray, V: np.ndarray, where: str = "bcgs2"):
    """BCGS2 with CholQR2 (Fig. 2b with the CholQR2 option, §IV-B): BCGS, then
    CholQR2 of the projected block, then BCGS again, then CholQR.  Five
    reductions per block.  Returns (Q_j, P, T) with
    V = Q P + Q_j T, where P = P1 + P2 T1 and T = T2 T1."""
    if Q.shape[1] == 0:
        Qj, T = cholqr2(V, where + "/cholqr2")
        return Qj, np.zeros((0, V.shape[1])), T
    Vh, P1 = bcgs(Q, V)
    Vt, T1 = cholqr2(Vh, where + "/cholqr2")
    Vt2, P2 = bcgs(Q, Vt)
    Qj, T2 = cholqr(Vt2, where + "/cholqr")
    return Qj, P1 + P2 @ T1, T2 @ T1


def bcgs_pip(Q: np.ndarray, V: np.ndarray, where: str = "bcgs_pip"):
    """BCGS with Pythagorean inner product (Fig. 4a, §IV-C).

    One reduction: [P; G] = [Q, V]^T V.  By the block Pythagorean theorem the
    Gram matrix of the projected block V - Q P is G - P^T P, so
    T = Chol(G - P^T P) and Q^_j = (V - Q P) T^{-1}.  Returns (Q^_j, P, T) with
    V = Q P + Q^_j T.  With no previous block (Q has 0 columns) this is CholQR."""
    k = Q.shape[1]
    X = np.concatenate([Q, V], axis=1)
    PG = X.T @ V                      # the single reduction
    P = PG[:k, :]
    G = PG[k:, :]
    S = G - P.T @ P
    T, info = chol_upper(S)
    if info:
        raise Breakdown(info, where, pivot_value(S, T, info), pip_margin(Q, V, P))
    W = V - Q @ P
    return right_trsm_upper(W, T), P, T


UNIT_ROUNDOFF = 2.0 ** -53


def cholqr_shift(n: int, c: int, fro2: float) -> float:
    """Shift of shifted CholQR (Fukaya, Kannan, Nakatsukasa, Zhang, Yamamoto,
    SIAM J. Sci. Comput. 2020; cited in §II as the remedy for CholQR's
    instability): sigma = 11 (n c + c (c + 1)) u ||X||^2 for an n x c block X,
    u the unit roundoff.  ||X||_2^2 is bounded here by the Frobenius norm
    squared ``fro2`` (the trace of the block's Gram), which keeps the
    guarantee (a larger shift)."""
    return 11.0 * (n * c + c * (c + 1)) * UNIT_ROUNDOFF * fro2


def bcgs_pip_shifted(Q: np.ndarray, V: np.ndarray, where: str = "bcgs_pip_shifted"):
    """BCGS-PIP with a shifted Cholesky (§II's shifted CholQR inside the
    Pythagorean step of Fig. 4a): [P; G] = [Q, V]^T V; T = Chol(G - P^T P +
    sigma I) with sigma = cholqr_shift(n, nb, trace(G)); Q^ = (V - Q P) T^{-1}.
    V = Q P + Q^ T still holds, but Q^ is only well conditioned, not
    orthonormal: Q^^T Q^ = I - sigma (T^T T)^{-1} for an orthonormal Q.
    Returns (Q^, P, T)."""
    k = Q.shape[1]
    n, c = V.shape
    X = np.concatenate([Q, V], axis=1)
    PG = X.T @ V                      # the single reduction
    P = PG[:k, :]
    G = PG[k:, :]
    S = G - P.T @ P + cholqr_shift(n, c, float(np.trace(G))) * np.eye(c)
    T, info = chol_upper(S)
    if info:
        raise Breakdown(info, where, pivot_value(S, T, info), pip_margin(Q, V, P))
    W = V - Q @ P
    return right_trsm_upper(W, T), P, T


def bcgs_pip2(Q: np.ndarray, V: np.ndarray, where: str = "bcgs_pip2"):
    """BCGS-PIP2 (Fig. 4b, §IV-C): BCGS-PIP applied twice.

    (Q^, P1, T1) = PIP(Q, V); (Q_j, P2, T2) = PIP(Q, Q^).  Since
    V = Q P1 + Q^ T1 and Q^ = Q P2 + Q_j T2:  V = Q (P1 + P2 T1) + Q_j (T2 T1)."""
    Qh, P1, T1 = bcgs_pip(Q, V, where + "/1")
    Qj, P2, T2 = bcgs_pip(Q, Qh, where + "/2")
    return Qj, P1 + P2 @ T1, T2 @ T1


def stage1(Qacc: np.ndarray, V: np.ndarray, where: str = "stage1"):
    """First stage of the two-stage scheme (§V, Fig. 5): one BCGS-PIP of the new
    panel V against everything accumulated, [Q_{1:l-1}, Q^_{l:j-1}] (the
    pre-processing that keeps the big panel well conditioned, Eq. (10)-(11))."""
    return bcgs_pip(Qacc, V, where)


def stage1_lowp(Qacc: np.ndarray, V: np.ndarray, where: str = "stage1", store=np.float32):
    """First stage for a basis stored in lower precision (the mixed-precision
    pattern).  The block Pythagorean identity G - P^T P of BCGS-PIP assumes the
    stored basis is orthonormal; an FP32-stored basis is orthonormal only to
    about eps32, so the identity cancels to a non-positive pivot as soon as a
    new MPK vector's component outside the basis falls below ~sqrt(eps32) of
    its norm.  Here the projected block's Gram is formed explicitly instead:
    P = Q^T V (FP64 products of the stored values); W = V - Q P rounded to the
    storage precision; T = Chol(W^T W) in FP64 (the higher-precision Gram of
    the mixed-precision CholQR of §II); Q^ = W T^{-1} rounded to storage.
    Inputs are the stored (FP32) values widened to FP64.  Returns
    (Q^ in FP64 holding storage-precision values, P, T)."""
    P = Qacc.T @ V
    W = (V - Qacc @ P).astype(store).astype(np.float64)
    G = W.T @ W
    T, info = chol_upper(G)
    if info:
        raise Breakdown(info, where, pivot_value(G, T, info))
    return right_trsm_upper(W, T).astype(store).astype(np.float64), P, T


def stage1_shifted(Qacc: np.ndarray, V: np.ndarray, where: str = "stage1"):
    """Stage 1 with the shifted Cholesky (``bcgs_pip_shifted``): the block is
    pre-processed to a well-conditioned one even where the unshifted
    Pythagorean Cholesky would break down on an ill-conditioned MPK block."""
    return bcgs_pip_shifted(Qacc, V, where)


def stage2_shifted(Qfin: np.ndarray, Qhat: np.ndarray, where: str = "stage2"):
    """Stage 2 after shifted stage-1 blocks: shifted CholQR3 (Fukaya et al.:
    one shifted pass, then CholQR twice) of the big panel, each pass a
    BCGS-PIP against Q_fin.  The shifted stage-1 blocks are well conditioned
    but not orthonormal, so the panel's condition number can reach
    u^(-1/2); the shifted pass brings it to O(1) and the two plain passes to
    orthonormal.  Returns (Q, P, T) with Q^ = Q_fin P + Q T: pass i gives
    (P_i, T_i) and P = P_a + P_b T_a + P_c T_b T_a, T = T_c T_b T_a."""
    Qa, P, T = bcgs_pip_shifted(Qfin, Qhat, where + "/shifted")
    Q = Qa
    for q in ("second", "third"):
        Q, Pq, Tq = bcgs_pip(Qfin, Q, where + "/" + q)
        P = P + Pq @ T
        T = Tq @ T
    return Q, P, T


def stage2(Qfin: np.ndarray, Qhat: np.ndarray, where: str = "stage2"):
    """Second stage (§V, Fig. 5): BCGS-PIP of the pre-processed big panel
    Q^_{l:t} against the finished basis Q_{1:l-1}.  With l = 1 (big panel equal
    to the whole restart cycle) this is CholQR of all columns (§V)."""
    return bcgs_pip(Qfin, Qhat, where)


def combine_two_stage(Rhat_top: np.ndarray, Rhat_diag: np.ndarray, P2: np.ndarray, T2: np.ndarray):
    """R factor of the big panel after stage 2 (§V).

    Stage 1 gave V_{l:t} = Q_{1:l-1} Rhat_top + Q^_{l:t} Rhat_diag; stage 2 gave
    Q^_{l:t} = Q_{1:l-1} P2 + Q_{l:t} T2.  Hence
    V_{l:t} = Q_{1:l-1} (Rhat_top + P2 Rhat_diag) + Q_{l:t} (T2 Rhat_diag)."""
    return Rhat_top + P2 @ Rhat_diag, T2 @ Rhat_diag


def two_stage_panel(Qfin: np.ndarray, blocks, where: str = "two_stage"):
    """Two-stage orthogonalization of one big panel made of pre-generated
    blocks (the synthetic-matrix experiments of §VI, Fig. 8).

    ``blocks`` are the panels V_l..V_t (each n x s).  Stage 1 runs BCGS-PIP of
    each panel against [Q_{1:l-1}, Q^_{l:j-1}]; stage 2 runs BCGS-PIP of the
    whole big panel against Q_{1:l-1}.  Returns (Q_{l:t}, R_top, R_diag, Qhat)
    with [V_l..V_t] = Q_{1:l-1} R_top + Q_{l:t} R_diag."""
    k0 = Qfin.shape[1]
    ncol = sum(b.shape[1] for b in blocks)
    Qhat = np.zeros((Qfin.shape[0], ncol))
    Rhat = np.zeros((k0 + ncol, ncol))
    c = 0
    for j, V in enumerate(blocks):
        Qacc = np.concatenate([Qfin, Qhat[:, :c]], axis=1)
        Qh, P, T = stage1(Qacc, V, f"{where}/stage1/block{j}")
        nb = V.shape[1]
        Qhat[:, c:c + nb] = Qh
        Rhat[:k0 + c, c:c + nb] = P
        Rhat[k0 + c:k0 + c + nb, c:c + nb] = T
        c += nb
    Q, P2, T2 = stage2(Qfin, Qhat, f"{where}/stage2")
    Rt, Rd = combine_two_stage(Rhat[:k0, :], Rhat[k0:, :], P2, T2)
    return Q, Rt, Rd, Qhat


def hhqr(V: np.ndarray):
    """Householder QR with a non-negative R diagonal (the HHQR option of Fig. 2b,
    §IV-A).  Independent checker: textbook reflections, one column at a time.
    Returns (Q, R) with Q of shape (n, c)."""
    A = np.array(V, dtype=np.float64, copy=True)
    n, c = A.shape
    vs = []
    for j in range(c):
        x = A[j:, j].copy()
        alpha = np.linalg.norm(x)
        v = x.copy()
        v[0] += alpha if x[0] >= 0 else -alpha
        vn = np.linalg.norm(v)
        if vn > 0:
            v /= vn
            A[j:, j:] -= 2.0 * np.outer(v, v @ A[j:, j:])
        vs.append(v)
    R = np.triu(A[:c, :])
    Q = np.zeros((n, c))
    Q[:c, :c] = np.eye(c)
    for j in reversed(range(c)):
        v = vs[j]
        Q[j:, :] -= 2.0 * np.outer(v, v @ Q[j:, :])
    sgn = np.where(np.diag(R) < 0, -1.0, 1.0)
    return Q * sgn, R * sgn[:, None]
