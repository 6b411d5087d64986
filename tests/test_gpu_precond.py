"""Multicolor Gauss-Seidel right preconditioner (§VIII, Fig. 9) on the GPU
against the oracle (``oracle.precond`` and ``sstep_gmres(precond="mcgs")``).

Bars: one sweep z = M^{-1} r element by element within 1e-13 relative (the
same coloring and color order on both sides; row sums in CSR order, FMA on the
GPU); solves: the oracle's status, x within 1e-6 relative at relative residual
1e-8, iterations within +-s, and the same Newton shifts."""
import numpy as np
import pytest
import torch

import synth
from oracle import krylov as kr, precond as pc

pytestmark = pytest.mark.gpu

GENS = {"lap2d": lambda: synth.laplace2d(64), "cd2d": lambda: synth.convdiff2d(50, 3),
        "banded": lambda: synth.banded_random(3000, 2, band=200), "lap3d": lambda: synth.laplace3d(16)}


@pytest.mark.parametrize("gen", list(GENS) + ["banded_wide"])
def test_gauss_seidel_sweep_matches_oracle(lib, gen):
    from paper_2402_15033_gb300 import capi
    A = GENS[gen]() if gen != "banded_wide" else synth.banded_random(20011, 5)
    S = capi.Solver.from_csr(A, capi.default_opts(precond=capi.GMRES_PRECOND_MCGS))
    r = synth.x_true(A.n, 11)
    rd = torch.tensor(r, device="cuda")
    zd = torch.full_like(rd, np.nan)
    S.precond_apply(rd, zd)
    S.close()
    z_ref = pc.gs_sweep(A, pc.greedy_coloring(A), r)
    z = zd.cpu().numpy()
    assert np.all(np.abs(z - z_ref) <= 1e-13 * np.abs(z_ref).max()), np.abs(z - z_ref).max()


def solve(capi, A, b, **kw):
    S = capi.Solver.from_csr(A, capi.default_opts(precond=capi.GMRES_PRECOND_MCGS, **kw))
    x = np.zeros(A.n)
    rc, res = S.solve(b, x)
    S.close()
    return rc, res, x


@pytest.mark.parametrize("gen,m,s,panel", [("lap2d", 60, 5, 60), ("cd2d", 30, 5, 30), ("banded", 30, 5, 30),
                                           ("lap3d", 60, 5, 60), ("lap2d", 60, 10, 60), ("lap2d", 60, 5, 20)])
def test_preconditioned_newton_solver_matches_oracle(lib, gen, m, s, panel):
    """The Newton basis with automatic shifts (the preconditioned operator has
    many eigenvalues at 1, where monomial powers lose rank)."""
    from paper_2402_15033_gb300 import capi
    A = GENS[gen]()
    b = kr.as_operator(A) @ synth.x_true(A.n, 0)
    rc, res, x = solve(capi, A, b, m=m, s=s, panel=panel, tol=1e-8, basis=capi.GMRES_BASIS_NEWTON_AUTO)
    xr, info = kr.sstep_gmres(A, b, m=m, s=s, panel=panel, tol=1e-8, theta="auto", precond="mcgs")
    assert info["status"] == 0
    assert rc == capi.GMRES_OK, (res, capi.last_error())
    assert res["relres_true"] <= 1e-8
    assert abs(res["iters"] - info["iters"]) <= s, (res["iters"], info["iters"])
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-6
    th = np.array(res["theta"][:s])
    assert np.allclose(th, info["theta"], rtol=0, atol=1e-7 * np.abs(info["theta"]).max())
    _, i0 = kr.sstep_gmres(A, b, m=m, s=s, panel=panel, tol=1e-8, theta="auto")
    assert info["iters"] < i0["iters"]                  # the preconditioner pays


@pytest.mark.parametrize("arith", [0, 1, 2])
def test_preconditioned_monomial_and_arithmetics(lib, arith):
    """The monomial basis where it holds (upwinded convection-diffusion), in
    FP64, double-float and tensor-core arithmetic."""
    from paper_2402_15033_gb300 import capi
    A = GENS["cd2d"]()
    b = kr.as_operator(A) @ synth.x_true(A.n, 0)
    rc, res, x = solve(capi, A, b, m=30, s=5, panel=30, tol=1e-8, arith=arith)
    xr, info = kr.sstep_gmres(A, b, m=30, s=5, panel=30, tol=1e-8, precond="mcgs")
    assert info["status"] == 0 and rc == capi.GMRES_OK
    assert abs(res["iters"] - info["iters"]) <= 5
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-6


def test_zero_diagonal_is_rejected(lib):
    from paper_2402_15033_gb300 import capi
    A = synth.laplace2d(8)
    vals = A.vals.copy()
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    vals[(A.colind == rows) & (rows == 5)] = 0.0
    with pytest.raises(capi.GmresError) as e:
        capi.Solver(A.n, A.rowptr, A.colind, vals, capi.default_opts(precond=capi.GMRES_PRECOND_MCGS))
    assert e.value.code == capi.GMRES_ERR_ARG and "diagonal" in str(e.value)
