"""GMRES_BASIS_NEWTON_AUTO on the GPU against the oracle's theta="auto": the
first cycle is standard GMRES (s = 1), its Ritz values in Leja order become
the Newton shifts, later cycles run the s-step Newton basis with the capacity
scale.  Bars: the oracle's status, x within 1e-6 relative at relative residual
1e-8, iterations within +-s, and the same shifts and scale (the shifts to the
agreement of two eigenvalue computations on two recovered Hessenberg
matrices, the scale exactly)."""
import numpy as np
import pytest

import synth
from oracle import krylov as kr

pytestmark = pytest.mark.gpu

ORTHO = {"two_stage": 0, "bcgs_pip2": 1, "bcgs2_cholqr2": 2}


def solve_gpu(capi, A, b, **opts):
    S = capi.Solver.from_csr(A, capi.default_opts(**opts))
    x = np.zeros(A.n)
    rc, res = S.solve(b, x)
    S.close()
    return rc, res, x


def check_auto(capi, A, b, m, s, panel, ortho="two_stage", arith=0, tol=1e-8):
    rc, res, x = solve_gpu(capi, A, b, m=m, s=s, panel=panel, tol=tol, arith=arith, ortho=ORTHO[ortho],
                           basis=capi.GMRES_BASIS_NEWTON_AUTO)
    xr, info = kr.sstep_gmres(A, b, m=m, s=s, panel=panel, tol=tol, ortho=ortho, theta="auto")
    assert info["status"] == 0
    assert rc == capi.GMRES_OK, (res, capi.last_error())
    assert res["relres_true"] <= tol
    assert abs(res["iters"] - info["iters"]) <= s, (res["iters"], info["iters"])
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-6
    th = np.array(res["theta"][:s])
    scale = np.abs(info["theta"]).max()
    assert np.allclose(th, info["theta"], rtol=0, atol=1e-7 * scale), (th, info["theta"])
    assert res["sigma"] == info["sigma"]
    assert all(t == 0.0 for t in res["theta"][s:])
    return rc, res, info


@pytest.mark.parametrize("N,m,s,panel,ortho", [(64, 60, 10, 60, "two_stage"), (64, 60, 15, 60, "two_stage"),
                                               (64, 60, 10, 20, "two_stage"), (64, 60, 15, 15, "bcgs_pip2"),
                                               (64, 60, 15, 15, "bcgs2_cholqr2"), (40, 48, 16, 48, "two_stage")])
def test_laplace2d_auto_newton_matches_oracle(lib, N, m, s, panel, ortho):
    from paper_2402_15033_gb300 import capi
    A = synth.laplace2d(N)
    b = kr.as_operator(A) @ synth.x_true(A.n, 0)
    check_auto(capi, A, b, m, s, panel, ortho)


def test_monomial_breaks_down_where_auto_newton_converges(lib):
    """s = 10 on the 64x64 Laplacian: the monomial basis breaks down in the
    first cycle on the GPU as in the oracle; the auto Newton basis converges."""
    from paper_2402_15033_gb300 import capi
    A = synth.laplace2d(64)
    b = kr.as_operator(A) @ synth.x_true(A.n, 0)
    rc, res, _ = solve_gpu(capi, A, b, m=60, s=10, panel=60, tol=1e-8)
    assert rc == capi.GMRES_ERR_BREAKDOWN and res["restarts"] == 1
    rc, res, info = check_auto(capi, A, b, 60, 10, 60)
    assert res["restarts"] >= 2


@pytest.mark.parametrize("arith", [1, 2])
def test_auto_newton_with_dd_and_tensor_core_arithmetic(lib, arith):
    from paper_2402_15033_gb300 import capi
    A = synth.laplace2d(64)
    b = kr.as_operator(A) @ synth.x_true(A.n, 0)
    check_auto(capi, A, b, 60, 10, 60, arith=arith)


@pytest.mark.parametrize("gen,N,seed,panel", [("convdiff2d", 48, 3, 60), ("convdiff3d", 28, 1, 20),
                                              ("convdiff3d", 28, 1, 60)])
def test_nonsymmetric_auto_newton_matches_oracle(lib, gen, N, seed, panel):
    """Upwinded convection-diffusion (complex Ritz values: real parts as
    shifts).  The first cycles of these cases end well above the tolerance, so
    the s = 1 Pythagorean steps near the end of the first cycle are not
    rounding ties."""
    from paper_2402_15033_gb300 import capi
    A = synth.convdiff2d(N, seed) if gen == "convdiff2d" else synth.convdiff3d(N, seed)
    b = kr.as_operator(A) @ synth.x_true(A.n, 1)
    check_auto(capi, A, b, 60, 10, panel)


def test_invariant_start_vector_in_the_first_cycle(lib):
    """A = 2 I: the Krylov space has dimension one, so the first (s = 1) step's
    projected vector is zero up to rounding.  The oracle reports a breakdown
    in the first cycle (its stage-1 block 0 or, numbered after the m stage-1
    blocks of s = 1, its stage-2 panel 0); the GPU either breaks down at one of
    the two as well (and picks no shifts) or, when rounding leaves both pivots
    positive, stops at once with x = b / 2."""
    import scipy.sparse as sp
    from paper_2402_15033_gb300 import capi
    n = 5000
    M = (sp.identity(n, format="csr") * 2.0).tocsr()
    A = synth.CSR(n, M.indptr, M.indices, M.data, "2I")
    b = np.ones(n)
    _, info = kr.sstep_gmres(A, b, m=30, s=5, panel=30, tol=1e-8, theta="auto")
    assert info["status"] == kr.STATUS_BREAKDOWN and info["breakdown_block"] in (0, 30) and info["theta"] is None
    rc, res, x = solve_gpu(capi, A, b, m=30, s=5, panel=30, tol=1e-8, basis=capi.GMRES_BASIS_NEWTON_AUTO)
    if rc == capi.GMRES_ERR_BREAKDOWN:
        assert res["breakdown_block"] in (0, 30) and res["theta"] == [0.0] * 16
    else:
        assert rc == capi.GMRES_OK and np.allclose(x, b / 2, rtol=1e-8)


@pytest.mark.parametrize("gen,N,seed,iters", [("laplace3d", 16, 0, 59), ("convdiff3d", 16, 4, 45)])
def test_first_cycle_convergence_keeps_the_shifts(lib, gen, N, seed, iters):
    """Problems that converge inside the first (s = 1, every step checked)
    cycle stop at the oracle's step and still report the shifts its Hessenberg
    matrix gives, as the oracle does."""
    from paper_2402_15033_gb300 import capi
    A = synth.laplace3d(N) if gen == "laplace3d" else synth.convdiff3d(N, seed)
    b = kr.as_operator(A) @ synth.x_true(A.n, 0 if gen == "laplace3d" else 1)
    rc, res, info = check_auto(capi, A, b, 60, 10, 60)
    assert res["restarts"] == 1 and info["restarts"] == 1 and info["iters"] == iters
    assert abs(res["iters"] - iters) <= 1


def test_chosen_shifts_reused_with_the_newton_basis(lib):
    """The shifts and scale an auto solve reports, passed back as
    GMRES_BASIS_NEWTON, give the oracle's Newton-basis solve with those shifts."""
    from paper_2402_15033_gb300 import capi
    A = synth.laplace2d(64)
    b = kr.as_operator(A) @ synth.x_true(A.n, 0)
    rc, res, _ = solve_gpu(capi, A, b, m=60, s=10, panel=60, tol=1e-8, basis=capi.GMRES_BASIS_NEWTON_AUTO)
    assert rc == 0
    th = list(res["theta"][:10])
    rc2, res2, x2 = solve_gpu(capi, A, b, m=60, s=10, panel=60, tol=1e-8, basis=capi.GMRES_BASIS_NEWTON,
                              theta=th, sigma=res["sigma"])
    xr, info = kr.sstep_gmres(A, b, m=60, s=10, panel=60, tol=1e-8, theta=np.array(th), sigma=res["sigma"])
    assert rc2 == 0 and info["status"] == 0
    assert abs(res2["iters"] - info["iters"]) <= 10
    assert np.linalg.norm(x2 - xr) / np.linalg.norm(xr) <= 1e-6
    assert res2["theta"][:10] == th and res2["sigma"] == res["sigma"]


def test_mixed_precision_auto_newton(lib):
    """FP32 basis with the auto Newton basis at s = 10 (3D Laplacian): converges
    to 1e-8 by FP64 refinement, x within 1e-6 of the FP64 oracle's."""
    from paper_2402_15033_gb300 import capi
    A = synth.laplace3d(24)
    M = kr.as_operator(A)
    b = M @ synth.x_true(A.n, 0)
    rc, res, x = solve_gpu(capi, A, b, m=60, s=10, panel=60, tol=1e-8, precision=capi.GMRES_PREC_MIXED,
                           basis=capi.GMRES_BASIS_NEWTON_AUTO)
    assert rc == 0, capi.last_error()
    assert np.linalg.norm(b - M @ x) / np.linalg.norm(b) <= 1e-8
    xr, info = kr.sstep_gmres(A, b, m=60, s=10, panel=60, tol=1e-8, theta="auto")
    assert info["status"] == 0
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-6
    assert np.allclose(res["theta"][:10], info["theta"], atol=1e-6 * np.abs(info["theta"]).max())


def test_served_auto_request_equals_the_lone_solve(lib):
    from paper_2402_15033_gb300 import capi
    reqs = []
    for i, A in enumerate([synth.laplace2d(48), synth.convdiff2d(40, 2)]):
        b = kr.as_operator(A) @ synth.x_true(A.n, i)
        o = capi.default_opts(m=60, s=10, panel=60, tol=1e-8, basis=capi.GMRES_BASIS_NEWTON_AUTO)
        reqs.append((A, b, o))
    srv = capi.Server(max_active=4)
    ids = [srv.submit(A, b, opts=o) for A, b, o in reqs]
    got = [srv.wait(i) for i in ids]
    srv.stop()
    for (A, b, o), (x, r) in zip(reqs, got):
        S = capi.Solver.from_csr(A, o)
        x1 = np.zeros(A.n)
        rc1, r1 = S.solve(b, x1)
        S.close()
        assert r["status"] == rc1 == 0
        assert r["iters"] == r1["iters"] and r["theta"] == r1["theta"]
        assert np.array_equal(x, x1)


def test_batched_engine_rejects_auto_shifts(lib):
    from paper_2402_15033_gb300 import capi
    A = synth.laplace2d(16)
    with pytest.raises(capi.GmresError) as e:
        capi.Batch([A, A], capi.default_opts(m=30, s=5, panel=30, basis=capi.GMRES_BASIS_NEWTON_AUTO))
    assert e.value.code == capi.GMRES_ERR_ARG
