"""Shifted CholQR (§II, Fukaya et al. 2020) in the two-stage scheme on the
GPU, against the oracle's shifted arm (``blockortho.bcgs_pip_shifted``,
``stage2_shifted``, ``sstep_gmres(shift=True)``).

Bars: on a well-conditioned block R within 1e-12 of each column's norm (the
shift is then far below the data and both sides compute the same sigma); on a
block of condition 1e9, the properties the shift fixes, checked on the GPU's
output (V = Q P + Q^ T to 1e-13; Q^^T Q^ + sigma T^-T T^-1 = I to 5% of the
shift term) and T within 1e-6 of the oracle's (the shifted Gram's condition
number, at most 1/(11 n nb u), bounds the amplification of the two sides'
different rounding); solves: the oracle's status, x within 1e-6 relative at
relative residual 1e-8, iterations within +-s.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import blockortho as bo, krylov as kr

pytestmark = pytest.mark.gpu


def run_shifted(capi, Q, V):
    n, nb = V.shape
    k = 0 if Q is None else Q.shape[1]
    buf = torch.zeros(k + nb, n + n % 2, dtype=torch.float64, device="cuda")    # 16-byte aligned columns
    if k:
        buf[:k, :n] = torch.tensor(Q.T)
    buf[k:, :n] = torch.tensor(V.T)
    Qd = buf[:k].T[:n] if k else None
    Vd = buf[k:].T[:n]
    R = torch.zeros(nb, k + nb, dtype=torch.float64, device="cuda").T
    work = torch.empty(capi.workspace_bytes(n, k, nb), dtype=torch.uint8, device="cuda")
    st = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    capi.ortho_stage1_shifted(Qd, Vd, R, work, st, k=k)
    torch.cuda.synchronize()
    return Vd.cpu().numpy(), R.cpu().numpy(), int(st.item())


@pytest.mark.parametrize("n,k,nb", [(40003, 0, 5), (40003, 20, 5), (5001, 7, 10), (777, 3, 1)])
def test_shifted_stage1_well_conditioned_matches_oracle(lib, n, k, nb):
    from paper_2402_15033_gb300 import capi
    g = synth.rng(5100 + n + k)
    Q = bo.hhqr(g.standard_normal((n, k)))[0] if k else None
    V = g.standard_normal((n, nb)) + (Q @ g.standard_normal((k, nb)) if k else 0.0)
    Vg, Rg, st = run_shifted(capi, Q, V)
    assert st == 0
    Qh, P, T = bo.bcgs_pip_shifted(np.zeros((n, 0)) if Q is None else Q, V)
    Rref = np.concatenate([P, T], 0)
    scale = np.linalg.norm(Rref, axis=0)
    assert np.all(np.abs(Rg - Rref) <= 1e-12 * scale[None, :])
    assert np.max(np.linalg.norm(Vg - Qh, axis=0)) <= 1e-12


def test_shifted_stage1_ill_conditioned_block(lib):
    from paper_2402_15033_gb300 import capi
    g = synth.rng(4545)
    n, k, c = 3000, 4, 5
    Q = bo.hhqr(g.standard_normal((n, k)))[0]
    V = synth.logscaled(n, c, 1e9, seed=7) + Q @ g.standard_normal((k, c))
    Vg, Rg, st = run_shifted(capi, Q, V)
    assert st == 0
    P, T = Rg[:k], Rg[k:]
    assert np.abs(Q @ P + Vg @ T - V).max() <= 1e-13 * np.abs(V).max()
    sig = bo.cholqr_shift(n, c, float(np.trace(V.T @ V)))
    Ti = np.linalg.inv(T)
    term = np.abs(sig * (Ti.T @ Ti)).max()
    E = Vg.T @ Vg + sig * (Ti.T @ Ti) - np.eye(c)
    assert term > 0.1 and np.abs(E).max() <= 0.05 * term, (np.abs(E).max(), term)
    _, Pr, Tr = bo.bcgs_pip_shifted(Q, V)
    assert np.abs(T - Tr).max() <= 1e-6 * np.abs(Tr).max()
    assert np.abs(P - Pr).max() <= 1e-12 * np.abs(Pr).max()
    # the unshifted Pythagorean Cholesky breaks down on this block
    from test_gpu_ortho import run_pip
    assert run_pip(capi, Q, V, stage=1)[2] != 0


def solve(capi, A, b, **opts):
    S = capi.Solver.from_csr(A, capi.default_opts(**opts))
    x = np.zeros(A.n)
    rc, res = S.solve(b, x)
    S.close()
    return rc, res, x


@pytest.mark.parametrize("arith", [0, 1, 2])
@pytest.mark.parametrize("N,m,s,panel", [(20, 60, 5, 60), (40, 30, 5, 30), (48, 60, 5, 20)])
def test_shifted_solver_matches_oracle(lib, arith, N, m, s, panel):
    """s = 5 monomial, where the path is decided by the data: the 20^2 system
    breaks down near the end of its first cycle without the shift, the other
    two do not; FP64, double-float and tensor-core arithmetic meet the
    solver's parity bars against the oracle's shifted arm."""
    from paper_2402_15033_gb300 import capi
    A = synth.laplace2d(N)
    b = kr.as_operator(A) @ synth.x_true(A.n, 0)
    rc, res, x = solve(capi, A, b, m=m, s=s, panel=panel, tol=1e-8, arith=arith, shift=capi.GMRES_SHIFT_CHOLQR3)
    xr, info = kr.sstep_gmres(A, b, m=m, s=s, panel=panel, tol=1e-8, shift=True)
    assert info["status"] == 0
    assert rc == capi.GMRES_OK, (res, capi.last_error())
    assert res["relres_true"] <= 1e-8
    assert abs(res["iters"] - info["iters"]) <= s, (res["iters"], info["iters"])
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-6


@pytest.mark.parametrize("arith", [0, 1, 2])
@pytest.mark.parametrize("panel", [60, 20])
def test_shifted_solver_s10_monomial(lib, arith, panel):
    """s = 10 with the monomial basis on the 64^2 Laplacian: the plain scheme
    breaks down in the oracle with a breakdown margin below 1
    (its pivot is decided by rounding, R-8), so the GPU breaks down too or, if
    rounding lets it through, converges to the tolerance; with the shift both
    converge.  The basis is so ill conditioned (the shift engages in every
    block) that rounding decides the path: x is compared where it is unique,
    within the closed-form forward-error bound kappa(A) tol of x_true (and
    twice that of the oracle's x), and the restart cycles within one of the
    oracle's (convergence is tested once per big panel)."""
    from paper_2402_15033_gb300 import capi
    from oracle import checks
    A = synth.laplace2d(64)
    xt = synth.x_true(A.n, 0)
    b = kr.as_operator(A) @ xt
    rc0, res0, _ = solve(capi, A, b, m=60, s=10, panel=panel, tol=1e-8, arith=arith)
    _, info0 = kr.sstep_gmres(A, b, m=60, s=10, panel=panel, tol=1e-8)
    # (the cycle in which it breaks down differs between x86 and Arm numpy)
    assert info0["status"] == kr.STATUS_BREAKDOWN and info0["breakdown_margin"] < 1.0
    assert rc0 == capi.GMRES_ERR_BREAKDOWN or (rc0 == capi.GMRES_OK and res0["relres_true"] <= 1e-8)
    rc, res, x = solve(capi, A, b, m=60, s=10, panel=panel, tol=1e-8, arith=arith, shift=1)
    xr, info = kr.sstep_gmres(A, b, m=60, s=10, panel=panel, tol=1e-8, shift=True)
    assert info["status"] == 0
    assert rc == capi.GMRES_OK, (res, capi.last_error())
    assert res["relres_true"] <= 1e-8
    assert abs(res["restarts"] - info["restarts"]) <= 1, (res["restarts"], info["restarts"])
    lo, hi = checks.laplace2d_extreme_eigs(64)
    kap = hi / lo
    assert np.linalg.norm(x - xt) / np.linalg.norm(xt) <= kap * 1e-8
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 2 * kap * 1e-8


def test_shifted_bcgs_pip2_mode(lib):
    """panel = s (the BCGS-PIP2 scheme) with the shift: stage 2 of every block
    is shifted CholQR3 of the block."""
    from paper_2402_15033_gb300 import capi
    A = synth.laplace2d(48)
    b = kr.as_operator(A) @ synth.x_true(A.n, 4)
    rc, res, x = solve(capi, A, b, m=60, s=5, panel=5, tol=1e-8, shift=1, ortho=capi.GMRES_ORTHO_BCGS_PIP2)
    xr, info = kr.sstep_gmres(A, b, m=60, s=5, panel=5, tol=1e-8, shift=True)
    assert info["status"] == 0 and rc == 0
    assert abs(res["iters"] - info["iters"]) <= 5
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-6
