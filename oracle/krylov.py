"""GMRES solvers of the oracle, FP64, restated from the paper (test infrastructure only).

* ``gmres_cgs2``   standard restarted GMRES(m), Arnoldi with classical
                   Gram-Schmidt twice (the "GMRES + CGS2" arm of Table 3, §I).
* ``sstep_gmres``  s-step GMRES (Fig. 1, §III) with BlkOrth one of
                   ``two_stage`` (§V, Fig. 5), ``bcgs_pip2`` (§IV-C, Fig. 4b) or
                   ``bcgs2_cholqr2`` (§IV-B, Fig. 2b).

The paper's Fig. 1 pseudocode is not in its source; the solver loop below restates
the method from §III and §V:

* A restart cycle starts from q_1 = r / ||r||, r = b - A x.
* Each s-step block runs the matrix powers kernel (MPK, §I, §III) from the last
  column of the previous block (for the two-stage scheme, the pre-processed
  column Q^_{j-1}; §V), producing s new vectors, then block-orthogonalizes them.
* MPK uses the monomial basis (§VI uses monomial throughout) with a power-of-two
  scale sigma, v_{i+1} = (A v_i - theta_i v_i) / sigma; sigma is exact in
  binary floating point, theta = 0 is the plain monomial basis.
* Convergence is tested where the basis becomes orthonormal: after each big
  panel (two-stage) or block (one-stage schemes); Table 2 and Table 4 report
  iteration counts that are multiples of the big-panel width.
* The upper Hessenberg H with A Q_{1:k} = Q_{1:k+1} H is recovered from the
  R factors (``hessenberg_columns``), then the least-squares problem
  min ||g_0 e_1 - H y|| is solved with Givens rotations.
"""
from __future__ import annotations

import math
import numpy as np
import scipy.sparse as sp

from . import blockortho as bo

STATUS_OK = 0
STATUS_MAXIT = 1
STATUS_BREAKDOWN = -4
STATUS_NAN = -5


def as_operator(A):
    """CSR object from ``synth`` (n, rowptr, colind, vals) -> scipy CSR matrix."""
    if sp.issparse(A):
        return A.tocsr()
    return sp.csr_matrix((A.vals, A.colind, A.rowptr), shape=(A.n, A.n))


def mpk_sigma(A) -> float:
    """Power-of-two scale for the monomial basis: 2^floor(log2 ||A||_inf)."""
    M = as_operator(A)
    rs = np.asarray(abs(M).sum(axis=1)).ravel()
    top = float(rs.max()) if rs.size else 1.0
    if not (top > 0.0):
        return 1.0
    return float(2.0 ** math.floor(math.log2(top)))


def mpk(M, v: np.ndarray, s: int, sigma: float, theta=None, minv=None, cheb=False) -> np.ndarray:
    """Matrix powers kernel, standard (non communication-avoiding) form (§III):
    s sparse matrix-vector products in sequence, w_1 = (A v - theta_0 v)/sigma,
    w_i = (A w_{i-1} - theta_{i-1} w_{i-1})/sigma.  With a right
    preconditioner (``minv`` applies M^{-1}) each product is A M^{-1} w (the
    preconditioner applied with every SpMV, §I).  ``cheb``: the three-term
    recurrence of the Chebyshev basis (``cheb_coeffs``), with y_0 = v and
    y_{i+1} = (A y_i - theta_i y_i - nu_i y_{i-1}) / sigma_i.  Returns the
    n x s block [y_1 .. y_s]."""
    n = v.shape[0]
    dt = v.dtype
    W = np.zeros((n, s), dtype=dt)
    prev, prev2 = v, None
    for i in range(s):
        y = M @ (prev if minv is None else minv(prev))
        if theta is not None and theta[i] != 0.0:
            y = y - dt.type(theta[i]) * prev
        sig_i, nu_i = cheb_coeffs(i, sigma) if cheb else (sigma, 0.0)
        if nu_i != 0.0:
            y = y - dt.type(nu_i) * prev2
        W[:, i] = y / dt.type(sig_i)
        prev, prev2 = W[:, i], prev
    return W


def cheb_coeffs(i: int, sigma: float):
    """Coefficients (sigma_i, nu_i) of product i (0-based within an s-step block)
    of the Chebyshev basis, A y_i = sigma_i y_{i+1} + c y_i + nu_i y_{i-1}: the
    Chebyshev polynomials T_i((z - c) / delta) of the interval [c - delta,
    c + delta] (Bai, Hu and Reichel 1994, named with the Newton basis in §VI),
    T_1 = x, T_{i+1} = 2 x T_i - T_{i-1}, give sigma_0 = delta and sigma_i = nu_i
    = delta / 2 for i >= 1; with sigma = delta / 2 that is (2 sigma, 0) for the
    block's first product and (sigma, sigma) for the others."""
    return (2.0 * sigma, 0.0) if i == 0 else (sigma, sigma)


def cheb_interval(H):
    """Interval [c - delta, c + delta] of the Chebyshev basis from the Ritz values
    of a first standard GMRES cycle (the eigenvalues of the square k x k
    Hessenberg matrix H_k): c and delta are the midpoint and half-length of the
    range of their real parts.  Ritz values that span no interval give delta =
    |c| (or 1 when c = 0), so that the basis stays defined."""
    Hk = np.asarray(H, dtype=np.float64)
    if Hk.shape[0] == 0:
        return 0.0, 1.0
    re = np.linalg.eigvals(Hk).real
    lo, hi = float(re.min()), float(re.max())
    c, d = 0.5 * (lo + hi), 0.5 * (hi - lo)
    if not (d > 0.0) or not math.isfinite(d):
        d = abs(c) if c != 0.0 else 1.0
    return c, d


class Givens:
    """Incremental QR of an upper Hessenberg matrix by Givens rotations and the
    right-hand side g (standard GMRES least squares, Saad and Schultz 1986)."""

    def __init__(self, m: int, g0: float):
        self.m = m
        self.Rg = np.zeros((m + 1, m))
        self.cs = np.zeros(m)
        self.sn = np.zeros(m)
        self.g = np.zeros(m + 1)
        self.g[0] = g0
        self.k = 0

    def add_column(self, h: np.ndarray):
        """Append column k of H (entries 0..k+1) and rotate it."""
        k = self.k
        col = np.array(h[: k + 2], dtype=np.float64, copy=True)
        for i in range(k):
            a, b = col[i], col[i + 1]
            col[i] = self.cs[i] * a + self.sn[i] * b
            col[i + 1] = -self.sn[i] * a + self.cs[i] * b
        a, b = col[k], col[k + 1]
        r = math.hypot(a, b)
        if r == 0.0:
            c, s = 1.0, 0.0
        else:
            c, s = a / r, b / r
        self.cs[k], self.sn[k] = c, s
        col[k] = r
        col[k + 1] = 0.0
        self.Rg[: k + 2, k] = col
        gk = self.g[k]
        self.g[k] = c * gk
        self.g[k + 1] = -s * gk
        self.k = k + 1

    def residual(self) -> float:
        return abs(self.g[self.k])

    def solve(self) -> np.ndarray:
        k = self.k
        y = np.zeros(k)
        for i in reversed(range(k)):
            y[i] = (self.g[i] - np.dot(self.Rg[i, i + 1:k], y[i + 1:k])) / self.Rg[i, i]
        return y


def gmres_cgs2(A, b, x0=None, m=60, tol=1e-8, max_restarts=1000):
    """Standard restarted GMRES(m) with CGS2 Arnoldi (Table 3 "GMRES + CGS2").
    Tests convergence every iteration.  Returns (x, info dict)."""
    M = as_operator(A)
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    bnorm = np.linalg.norm(b)
    iters = 0
    hist = []
    status = STATUS_MAXIT
    restarts = 0
    for cyc in range(max_restarts):
        r = b - M @ x
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta / bnorm <= tol:
            status = STATUS_OK
            break
        restarts += 1
        Q = np.zeros((n, m + 1))
        Q[:, 0] = r / beta
        gv = Givens(m, beta)
        H = np.zeros((m + 1, m))
        k = 0
        for j in range(m):
            w = M @ Q[:, j]
            h1 = Q[:, : j + 1].T @ w
            w = w - Q[:, : j + 1] @ h1
            h2 = Q[:, : j + 1].T @ w
            w = w - Q[:, : j + 1] @ h2
            h = h1 + h2
            hn = np.linalg.norm(w)
            H[: j + 1, j] = h
            H[j + 1, j] = hn
            if hn > 0:
                Q[:, j + 1] = w / hn
            gv.add_column(H[: j + 2, j])
            iters += 1
            k = j + 1
            if gv.residual() / bnorm <= tol or hn == 0:
                break
        y = gv.solve()
        x = x + Q[:, :k] @ y
    else:
        r = b - M @ x
        hist.append(np.linalg.norm(r) / bnorm)
    return x, dict(status=status, iters=iters, restarts=restarts, relres=hist[-1], history=hist)


def hessenberg_columns(Rfin, C, start_final, s, sigma, theta, c_lo, c_hi, H, cheb=False):
    """Columns c_lo..c_hi-1 of the upper Hessenberg H with A Q_{1:k} = Q_{1:k+1} H.

    SpMV number c (0-based) reads input y_c and writes raw column c+1, with
    A y_c = sigma w_{c+1} + theta_c y_c.  In final (orthonormal) coordinates:
      a_c = e_c        if c starts a block whose start column was already final,
      a_c = C[:, c]    if c starts a block from a pre-processed column q^_c,
      a_c = Rfin[:, c] otherwise (y_c is the raw MPK output w_c);
      b_c = sigma Rfin[:, c+1] + theta_c a_c.
    With the Chebyshev basis (``cheb``) A y_c = sigma_c w_{c+1} + theta_c y_c +
    nu_c y_{c-1} (``cheb_coeffs`` of c mod s), so b_c = sigma_c Rfin[:, c+1] +
    theta_c a_c + nu_c a_{c-1}; nu_c = 0 at a block's first column, so a_{c-1}
    is always a column of the same block.
    With A_k = [a_0..a_{k-1}] upper triangular and B_k = [b_0..b_{k-1}],
    H = B_k A_k^{-1}, solved one column at a time (H A = B)."""
    mp1 = Rfin.shape[0]

    def coords(c):
        if c % s == 0:
            a = np.zeros(mp1)
            if start_final[c]:
                a[c] = 1.0
            else:
                a[:] = C[:, c]
            return a
        return Rfin[:, c].copy()

    for c in range(c_lo, c_hi):
        a = coords(c)
        sig_c, nu_c = cheb_coeffs(c % s, sigma) if cheb else (sigma, 0.0)
        bcol = sig_c * Rfin[:, c + 1] + (theta[c % s] * a if theta is not None else 0.0)
        if nu_c != 0.0:
            bcol = bcol + nu_c * coords(c - 1)
        acc = bcol.copy()
        for i in range(c):
            acc -= H[:, i] * a[i]
        H[:, c] = acc / a[c]
    return H


def leja_order(z) -> np.ndarray:
    """Leja ordering of real points (Reichel, BIT 30, 1990), the ordering that
    the Newton-basis s-step GMRES of Bai, Hu and Reichel (1994) gives its
    shifts so that the shifted products stay well conditioned: the first point
    has the largest modulus, every later one maximizes the product of its
    distances to the points already taken.  The candidates are scanned in
    ascending order and a tie goes to the first maximum; the distances are
    scaled by 2^-e with max|z| <= 2^e (exact) so that the products neither
    overflow nor depend on the scale.  Returns all the points in Leja order."""
    x = np.sort(np.asarray(z, dtype=np.float64).ravel())
    if x.size == 0:
        return x
    top = float(np.max(np.abs(x)))
    scale = 1.0 if top == 0.0 else 2.0 ** -math.frexp(top)[1]
    order = [int(np.argmax(np.abs(x)))]
    left = np.ones(x.size, dtype=bool)
    left[order[0]] = False
    prod = np.ones(x.size)
    while left.any():
        prod = prod * np.abs((x - x[order[-1]]) * scale)
        cand = np.where(left, prod, -1.0)
        i = int(np.argmax(cand))
        order.append(i)
        left[i] = False
    return x[np.array(order)]


def newton_shifts(H, s: int) -> np.ndarray:
    """Shifts theta_0..theta_{s-1} of the Newton basis, from the Ritz values of
    a first standard GMRES cycle (the eigenvalues of the square k x k
    Hessenberg matrix H_k with A Q_k = Q_{k+1} H): their real parts in Leja
    order, the first s of them (repeated cyclically when k < s).  The real
    parts keep the basis recurrence real; a conjugate pair gives one real
    shift twice, and the repeat has distance product 0, so it comes last."""
    Hk = np.asarray(H, dtype=np.float64)
    k = Hk.shape[0]
    if k == 0:
        return np.zeros(s)
    ritz = np.linalg.eigvals(Hk)
    pts = leja_order(ritz.real)
    return np.array([pts[i % k] for i in range(s)])


def newton_sigma(theta, fallback: float) -> float:
    """Scale of the Newton basis: the power of two nearest (in log2) to the
    capacity of the interval [min theta, max theta], a quarter of its length
    (the logarithmic capacity of a real interval).  Dividing each shifted
    product by it keeps the Newton basis columns of comparable norm, as
    ||A||_inf does for the monomial basis.  ``fallback`` when the shifts span
    no interval.  Nearest in log2: cap = f 2^e with f in [1/2, 1) rounds up to
    2^e when f >= 2^-1/2, else down to 2^(e-1)."""
    th = np.asarray(theta, dtype=np.float64)
    cap = 0.25 * (float(th.max()) - float(th.min())) if th.size else 0.0
    if not (cap > 0.0) or not math.isfinite(cap):
        return float(fallback)
    f, e = math.frexp(cap)
    return math.ldexp(1.0, e if f >= math.sqrt(0.5) else e - 1)


def sstep_gmres(A, b, x0=None, m=60, s=5, panel=None, tol=1e-8, max_restarts=1000,
                ortho="two_stage", sigma=None, theta=None, return_basis=False, basis_dtype=np.float64,
                shift=False, precond=None, cheb=None):
    """s-step GMRES (Fig. 1, §III) with the chosen block orthogonalization.

    ``panel`` is the second step size s^ of the two-stage scheme (§V); it must
    satisfy s | s^ and s | m.  When s^ does not divide m, the last big panel of
    each restart cycle holds the remaining m mod s^ columns: stage 2 also runs
    at the restart (the reading that Table 2's counts for s^ = 40, m = 60
    imply: 60280 = 1004 * 60 + 40).  ``theta`` is None (monomial basis), s Newton shifts,
    or "auto": the first cycle runs with s = s^ = 1 (standard GMRES through the
    same block machinery), ``newton_shifts`` turns its Hessenberg matrix into s
    shifts, and every later cycle uses the Newton basis with them, scaled by
    ``newton_sigma`` unless ``sigma`` is given.  ``cheb`` selects the Chebyshev
    basis instead (``cheb_coeffs``): an interval (c, delta), or "auto", where the
    first cycle is standard GMRES as for theta = "auto" and ``cheb_interval``
    turns its Hessenberg matrix into the interval; the MPK shift is c and its
    scale delta / 2.  ``ortho`` in {"two_stage", "bcgs_pip2", "bcgs2_cholqr2"}.
    ``precond="mcgs"`` (FP64 basis) preconditions from the right with one
    forward multicolor Gauss-Seidel sweep (``oracle.precond``, the local
    Gauss-Seidel of §VIII, Fig. 9): the MPK applies A M^{-1}, the correction is
    x += M^{-1} Q y, and the MPK scale is 1 unless ``sigma`` is given.
    ``shift=True`` (two-stage, FP64 basis) runs stage 1 with the shifted
    Cholesky of ``blockortho.stage1_shifted`` and stage 2 as shifted CholQR3
    of the big panel (``blockortho.stage2_shifted``).
    ``basis_dtype=np.float32`` is the mixed-precision pattern: the basis is
    stored in FP32 and the MPK runs in FP32 on an FP32 copy of A, while every
    Gram product and sum, the Cholesky factors, the Hessenberg/Givens work, x
    and the restart residual stay FP64 (higher-precision Gram accumulation, as
    in the mixed-precision CholQR of §II).  Stage 1 then forms the projected
    block's Gram explicitly (``blockortho.stage1_lowp``) because the
    Pythagorean identity assumes an orthonormal stored basis.  Each restart
    cycle is one FP64 iterative-refinement step: r = b - A x in FP64, A d = r
    solved with the FP32 basis, x += d.

    Returns (x, info dict) with status, iteration count (SpMVs inside restart
    cycles), restarts, the explicit relative residual, the breakdown location
    (``breakdown_block``: s-step block j, or m/s + p for the stage 2 of big
    panel p; ``breakdown_pivot``: 1-based; ``breakdown_value``: the failing
    pivot; ``breakdown_margin``: ``Breakdown.margin``), and, when
    ``return_basis``, the last cycle's Q, H and g0 (for Arnoldi-relation tests)."""
    M = as_operator(A)
    n = b.shape[0]
    lowp = np.dtype(basis_dtype) == np.float32
    if cheb is not None and theta is not None:
        raise ValueError("theta and cheb are exclusive")
    auto = isinstance(theta, str) or isinstance(cheb, str)
    if auto and (theta if cheb is None else cheb) != "auto":
        raise ValueError("theta must be None, s shifts or 'auto'; cheb None, (c, delta) or 'auto'")
    use_cheb = cheb is not None
    th = None if auto else theta
    s_req = s
    Mb = M.astype(np.float32) if lowp else M
    f64 = np.float64
    if panel is None:
        panel = m
    if ortho != "two_stage":
        panel = s
    if m % s or panel % s or panel > m:
        raise ValueError("need s | panel, s | m and panel <= m")
    panel_req = panel
    minv = None
    if precond is not None:
        if precond != "mcgs" or lowp:
            raise ValueError("precond must be 'mcgs' (FP64 basis)")
        from . import precond as pc
        colors = pc.greedy_coloring(M)
        minv = lambda v: pc.gs_sweep(M, colors, v)  # noqa: E731
    sig = (1.0 if minv is not None else mpk_sigma(A)) if sigma is None else float(sigma)
    cheb_on = False                     # the current cycle's basis is the Chebyshev one
    if use_cheb and not auto:
        c0, d0 = float(cheb[0]), float(cheb[1])
        if not (d0 > 0.0):
            raise ValueError("the Chebyshev half-width delta must be positive")
        th, sig, cheb_on = np.full(s, c0), 0.5 * d0, True
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    bnorm = np.linalg.norm(b)
    iters = 0
    restarts = 0
    hist = []
    status = STATUS_MAXIT
    last = {}
    err_where = None
    breakdown = (-1, 0, float("nan"), float("inf"))
    for cyc in range(max_restarts):
        r = b - M @ x
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if not np.isfinite(beta):
            status = STATUS_NAN
            break
        if beta / bnorm <= tol:
            status = STATUS_OK
            break
        restarts += 1
        # theta = "auto": the first cycle is standard GMRES (s = 1, one SpMV per
        # block) whose Hessenberg matrix gives the Ritz values for the shifts.
        # For the two-stage scheme it also takes s^ = 1, i.e. every vector is
        # re-orthogonalized at once (CGS-P twice, the BCGS-PIP2 form): with
        # s = 1 and a wide big panel the single Pythagorean pass loses
        # orthogonality as the residual falls and breaks down near convergence.
        first = auto and th is None
        s = 1 if first else s_req
        panel = (1 if first else panel_req) if ortho == "two_stage" else s
        Q = np.zeros((n, m + 1), dtype=basis_dtype)
        Q[:, 0] = r / beta
        Rhat = np.zeros((m + 1, m + 1))
        Rhat[0, 0] = 1.0
        Rfin = np.zeros((m + 1, m + 1))
        C = np.zeros((m + 1, m + 1))
        final = np.zeros(m + 1, dtype=bool)
        start_final = np.zeros(m + 1, dtype=bool)
        H = np.zeros((m + 1, m))
        if ortho == "two_stage":
            lo, hi = 0, panel          # first big panel: columns 0..s^ (s^+1 vectors)
        else:
            final[0] = True            # q_1 = r/||r|| is already orthonormal
            C[0, 0] = 1.0
            Rfin[0, 0] = 1.0
        gv = None
        k_used = 0
        done = False
        where_blk = 0
        try:
            for j in range(m // s):
                where_blk = j
                st = s * j
                start_final[st] = final[st]
                W = mpk(Mb, Q[:, st], s, sig, th, minv, cheb=cheb_on)
                cols = slice(st + 1, st + s + 1)
                if ortho == "two_stage":
                    st1 = bo.stage1_lowp if lowp else (bo.stage1_shifted if shift else bo.stage1)
                    Qh, P, T = st1(Q[:, : st + 1].astype(f64), W.astype(f64), f"cycle{cyc}/block{j}")
                    Q[:, cols] = Qh
                    Rhat[: st + 1, cols] = P
                    Rhat[cols, cols] = T
                    t = st + s
                    if t < hi:
                        continue
                    where_blk = m // s + (t - 1) // panel
                    st2 = bo.stage2_shifted if (shift and not lowp) else bo.stage2
                    Qn, P2, T2 = st2(Q[:, :lo].astype(f64), Q[:, lo:t + 1].astype(f64), f"cycle{cyc}/stage2@{t}")
                    Q[:, lo:t + 1] = Qn
                    C[:lo, lo:t + 1] = P2
                    C[lo:t + 1, lo:t + 1] = T2
                    final[lo:t + 1] = True
                    top, diag = bo.combine_two_stage(Rhat[:lo, lo:t + 1], Rhat[lo:t + 1, lo:t + 1], P2, T2)
                    Rfin[:lo, lo:t + 1] = top
                    Rfin[lo:t + 1, lo:t + 1] = diag
                    c_lo = max(lo - 1, 0)
                    lo, hi = t + 1, min(t + panel, m)
                else:
                    fn = bo.bcgs_pip2 if ortho == "bcgs_pip2" else bo.bcgs2_cholqr2
                    Qj, P, T = fn(Q[:, : st + 1].astype(f64), W.astype(f64), f"cycle{cyc}/block{j}")
                    Q[:, cols] = Qj
                    Rfin[: st + 1, cols] = P
                    Rfin[cols, cols] = T
                    C[st + 1:st + s + 1, st + 1:st + s + 1] = np.eye(s)
                    final[cols] = True
                    t = st + s
                    c_lo = st
                if gv is None:
                    gv = Givens(m, beta * C[0, 0])
                hessenberg_columns(Rfin, C, start_final, s, sig, th, c_lo, t, H, cheb=cheb_on)
                for c in range(c_lo, t):
                    gv.add_column(H[: c + 2, c])
                k_used = t
                if gv.residual() / bnorm <= tol:
                    done = True
                    break
        except bo.Breakdown as e:
            status = STATUS_BREAKDOWN
            err_where = str(e)
            breakdown = (where_blk, e.pivot, e.value, e.margin)
            break
        y = gv.solve()
        dx = Q[:, :k_used].astype(f64) @ y
        x = x + (dx if minv is None else minv(dx))
        iters += k_used
        last = dict(Q=Q, H=H, g0=beta * C[0, 0], k=k_used, Rfin=Rfin, C=C)
        if auto and th is None:
            if use_cheb:
                c0, d0 = cheb_interval(H[:k_used, :k_used])
                th, sig, cheb_on = np.full(s_req, c0), 0.5 * d0, True
            else:
                th = newton_shifts(H[:k_used, :k_used], s_req)
                if sigma is None:
                    sig = newton_sigma(th, sig)
    else:
        r = b - M @ x
        hist.append(np.linalg.norm(r) / bnorm)
    info = dict(status=status, iters=iters, restarts=restarts, relres=hist[-1], history=hist,
                sigma=sig, where=err_where, breakdown_block=breakdown[0], breakdown_pivot=breakdown[1],
                breakdown_value=breakdown[2], breakdown_margin=breakdown[3],
                theta=None if th is None else np.asarray(th, dtype=np.float64), cheb=cheb_on)
    if return_basis:
        info.update(last)
    return x, info
