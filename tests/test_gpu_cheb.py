"""GMRES_BASIS_CHEBYSHEV(_AUTO) on the GPU against the oracle's cheb basis:
per s-step block the MPK forms T_i((A - cI)/delta) y_0 by the three-term
recurrence and the Hessenberg recovery uses the tridiagonal change of basis.
Bars: the oracle's status, x within 1e-6 relative at relative residual 1e-8,
iterations within +-s, and (auto) the same interval to the agreement of two
eigenvalue computations on two recovered Hessenberg matrices."""
import numpy as np
import pytest

import synth
from oracle import checks, krylov as kr

pytestmark = pytest.mark.gpu

ORTHO = {"two_stage": 0, "bcgs_pip2": 1, "bcgs2_cholqr2": 2}


def solve_gpu(capi, A, b, **opts):
    S = capi.Solver.from_csr(A, capi.default_opts(**opts))
    x = np.zeros(A.n)
    rc, res = S.solve(b, x)
    S.close()
    return rc, res, x


def check(capi, A, b, m, s, panel, ortho="two_stage", arith=0, tol=1e-8, interval=None, **extra):
    if interval is None:
        gopts = dict(basis=capi.GMRES_BASIS_CHEBYSHEV_AUTO)
        cheb = "auto"
    else:
        gopts = dict(basis=capi.GMRES_BASIS_CHEBYSHEV, theta=list(interval))
        cheb = interval
    rc, res, x = solve_gpu(capi, A, b, m=m, s=s, panel=panel, tol=tol, arith=arith, ortho=ORTHO[ortho],
                           **gopts, **extra)
    xr, info = kr.sstep_gmres(A, b, m=m, s=s, panel=panel, tol=tol, ortho=ortho, cheb=cheb)
    assert info["status"] == 0 and info["cheb"]
    assert rc == capi.GMRES_OK, (res, capi.last_error())
    assert res["relres_true"] <= tol
    assert abs(res["iters"] - info["iters"]) <= s, (res["iters"], info["iters"])
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-6
    c = res["theta"][0]
    assert all(t == c for t in res["theta"][:s]) and all(t == 0.0 for t in res["theta"][s:])
    scale = abs(info["theta"][0]) + 2.0 * info["sigma"]
    assert abs(c - info["theta"][0]) <= 1e-7 * scale and abs(res["sigma"] - info["sigma"]) <= 1e-7 * scale
    return rc, res, info


@pytest.mark.parametrize("N,m,s,panel,ortho", [(64, 60, 10, 60, "two_stage"), (64, 60, 15, 60, "two_stage"),
                                               (64, 60, 10, 20, "two_stage"), (64, 60, 15, 15, "bcgs_pip2"),
                                               (64, 60, 15, 15, "bcgs2_cholqr2"), (40, 48, 16, 48, "two_stage")])
def test_laplace2d_auto_chebyshev_matches_oracle(lib, N, m, s, panel, ortho):
    from paper_2402_15033_gb300 import capi
    A = synth.laplace2d(N)
    b = kr.as_operator(A) @ synth.x_true(A.n, 0)
    check(capi, A, b, m, s, panel, ortho)


def test_monomial_breaks_down_where_chebyshev_converges(lib):
    """s = 10 on the 64x64 Laplacian: the monomial basis breaks down in the
    first cycle; the Chebyshev basis on the spectral interval (closed form)
    and on the Ritz interval converge."""
    from paper_2402_15033_gb300 import capi
    A = synth.laplace2d(64)
    b = kr.as_operator(A) @ synth.x_true(A.n, 0)
    rc, res, _ = solve_gpu(capi, A, b, m=60, s=10, panel=60, tol=1e-8)
    assert rc == capi.GMRES_ERR_BREAKDOWN and res["restarts"] == 1
    lo, hi = checks.laplace2d_extreme_eigs(64)
    _, res_e, _ = check(capi, A, b, 60, 10, 60, interval=(0.5 * (lo + hi), 0.5 * (hi - lo)))
    assert res_e["sigma"] == 0.25 * (hi - lo)
    _, res_a, _ = check(capi, A, b, 60, 10, 60)
    assert res_a["restarts"] >= 2


@pytest.mark.parametrize("arith", [1, 2])
def test_auto_chebyshev_with_dd_and_tensor_core_arithmetic(lib, arith):
    from paper_2402_15033_gb300 import capi
    A = synth.laplace2d(64)
    b = kr.as_operator(A) @ synth.x_true(A.n, 0)
    check(capi, A, b, 60, 10, 60, arith=arith)


@pytest.mark.parametrize("gen,N,seed,panel", [("convdiff2d", 48, 3, 60), ("convdiff3d", 28, 1, 20)])
def test_nonsymmetric_auto_chebyshev_matches_oracle(lib, gen, N, seed, panel):
    """Upwinded convection-diffusion: complex Ritz values, the interval of their
    real parts."""
    from paper_2402_15033_gb300 import capi
    A = synth.convdiff2d(N, seed) if gen == "convdiff2d" else synth.convdiff3d(N, seed)
    b = kr.as_operator(A) @ synth.x_true(A.n, 1)
    check(capi, A, b, 60, 10, panel)


def test_preconditioned_chebyshev_matches_oracle(lib):
    """Right multicolor Gauss-Seidel with the Chebyshev basis of A M^{-1}: the
    three-term term reads the unpreconditioned previous basis vector."""
    from paper_2402_15033_gb300 import capi
    A = synth.convdiff2d(48, 3)
    b = kr.as_operator(A) @ synth.x_true(A.n, 1)
    rc, res, x = solve_gpu(capi, A, b, m=60, s=10, panel=60, tol=1e-8, precond=capi.GMRES_PRECOND_MCGS,
                           basis=capi.GMRES_BASIS_CHEBYSHEV_AUTO)
    xr, info = kr.sstep_gmres(A, b, m=60, s=10, panel=60, tol=1e-8, precond="mcgs", cheb="auto")
    assert info["status"] == 0 and rc == 0, capi.last_error()
    assert abs(res["iters"] - info["iters"]) <= 10
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-6


def test_mixed_precision_auto_chebyshev(lib):
    """FP32 basis with the auto Chebyshev basis at s = 10 (3D Laplacian):
    converges to 1e-8 by FP64 refinement, x within 1e-6 of the FP64 oracle's."""
    from paper_2402_15033_gb300 import capi
    A = synth.laplace3d(24)
    M = kr.as_operator(A)
    b = M @ synth.x_true(A.n, 0)
    rc, res, x = solve_gpu(capi, A, b, m=60, s=10, panel=60, tol=1e-8, precision=capi.GMRES_PREC_MIXED,
                           basis=capi.GMRES_BASIS_CHEBYSHEV_AUTO)
    assert rc == 0, capi.last_error()
    assert np.linalg.norm(b - M @ x) / np.linalg.norm(b) <= 1e-8
    xr, info = kr.sstep_gmres(A, b, m=60, s=10, panel=60, tol=1e-8, cheb="auto")
    assert info["status"] == 0
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-6


def test_bad_interval_and_batches_are_rejected(lib):
    from paper_2402_15033_gb300 import capi
    A = synth.laplace2d(16)
    for th in ([4.0, 0.0], [4.0, -1.0], [float("nan"), 1.0]):
        with pytest.raises(capi.GmresError) as e:
            capi.Solver.from_csr(A, capi.default_opts(m=30, s=5, panel=30, basis=capi.GMRES_BASIS_CHEBYSHEV, theta=th))
        assert e.value.code == capi.GMRES_ERR_ARG
    with pytest.raises(capi.GmresError) as e:
        capi.Batch([A, A], capi.default_opts(m=30, s=5, panel=30, basis=capi.GMRES_BASIS_CHEBYSHEV_AUTO))
    assert e.value.code == capi.GMRES_ERR_ARG
