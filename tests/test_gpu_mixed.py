"""Mixed-precision pattern on the GPU: FP32 basis and MPK, FP64 Gram products
and sums, FP64 Cholesky/Hessenberg/Givens, FP64 restart residual (iterative
refinement).  Parity with the oracle's mixed arm (``basis_dtype=float32``) and
the error against the FP64 oracle solution, per result.

Tolerances: R entries within 1e-12 * ||R[:, j]|| (the FP32 inputs widen
exactly, all arithmetic is FP64); updated FP32 columns within 2 FP32 ulps of
the oracle's FP64 result rounded to FP32 (relative 2.4e-7, scaled by kappa(T));
solutions: relative residual <= 1e-8 in FP64, x within 1e-6 of the FP64
oracle's x, iterations within one restart cycle of the mixed oracle's (FP32
rounding differences in the MPK can move a convergence test by a cycle)."""
import numpy as np
import pytest
import torch

import synth
from oracle import blockortho as bo, krylov as kr

pytestmark = pytest.mark.gpu
EPS32 = np.finfo(np.float32).eps


def run_f32(capi, Q, V, stage):
    n, nb = V.shape
    k = 0 if Q is None else Q.shape[1]
    ld = (n + 3) // 4 * 4   # FP32 columns stay 16-byte aligned
    buf = torch.zeros(k + nb, ld, dtype=torch.float32, device="cuda")
    if k:
        buf[:k, :n] = torch.tensor(Q.T)
    buf[k:, :n] = torch.tensor(V.T)
    Qd = buf[:k].T[:n] if k else None
    Vd = buf[k:].T[:n]
    R = torch.zeros(nb, k + nb, dtype=torch.float64, device="cuda").T
    work = torch.empty(capi.workspace_bytes(n, k, nb), dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    (capi.ortho_stage1_f32 if stage == 1 else capi.ortho_stage2_f32)(Qd, Vd, R, work, st, k=k)
    torch.cuda.synchronize()
    return Vd.cpu().numpy(), R.cpu().numpy(), int(st.item())


@pytest.mark.parametrize("n,k,nb,stage", [(50001, 11, 5, 1), (4097, 0, 10, 1), (30000, 0, 61, 2), (8000, 20, 21, 2)])
def test_f32_ortho_matches_oracle(lib, n, k, nb, stage):
    from paper_2402_15033_gb300 import capi
    g = synth.rng(300 + n)
    Q = bo.hhqr(g.standard_normal((n, k)))[0].astype(np.float32) if k else None
    V = (g.standard_normal((n, nb)) / np.sqrt(n)).astype(np.float32)
    Vg, Rg, st = run_f32(capi, Q, V, stage)
    assert st == 0
    Qh, P, T = bo.bcgs_pip(np.zeros((n, 0)) if Q is None else Q.astype(np.float64), V.astype(np.float64))
    Rref = np.concatenate([P, T], 0)
    scale = np.linalg.norm(Rref, axis=0)
    assert np.all(np.abs(Rg - Rref) <= 1e-12 * scale[None, :])
    kap = max(1.0, np.linalg.cond(T))
    ref32 = Qh.astype(np.float32).astype(np.float64)
    err = np.abs(Vg.astype(np.float64) - ref32)
    assert np.all(err <= 2 * EPS32 * kap * np.abs(ref32).max(axis=0)[None, :])


def mixed_vs_oracle(capi, A, b, m, s, panel, tol=1e-8):
    S = capi.Solver.from_csr(A, capi.default_opts(m=m, s=s, panel=panel, tol=tol, precision=capi.GMRES_PREC_MIXED))
    x = np.zeros(A.n)
    rc, res = S.solve(b, x)
    S.close()
    xm, im = kr.sstep_gmres(A, b, m=m, s=s, panel=panel, tol=tol, basis_dtype=np.float32)
    x64, i64 = kr.sstep_gmres(A, b, m=m, s=s, panel=panel, tol=tol)
    assert im["status"] == 0
    assert rc == capi.GMRES_OK, res
    M = kr.as_operator(A)
    assert np.linalg.norm(b - M @ x) / np.linalg.norm(b) <= tol
    assert res["relres_true"] <= tol
    assert abs(res["iters"] - im["iters"]) <= m, (res["iters"], im["iters"])
    assert res["ir_steps"] == res["restarts"]
    ref = x64 if i64["status"] == 0 else xm
    err = np.linalg.norm(x - ref) / np.linalg.norm(ref)
    assert err <= 1e-6, err
    return res, err


@pytest.mark.parametrize("N,m,s,panel", [(64, 60, 5, 60), (48, 60, 5, 20), (32, 30, 5, 30)])
def test_mixed_laplace2d(lib, N, m, s, panel):
    from paper_2402_15033_gb300 import capi
    A = synth.laplace2d(N)
    b = kr.as_operator(A) @ synth.x_true(A.n, 0)
    mixed_vs_oracle(capi, A, b, m, s, panel)


@pytest.mark.parametrize("N,s", [(20, 5), (20, 10), (24, 10)])
def test_mixed_laplace3d(lib, N, s):
    """The mixed-precision configuration's stencil (3D 7-point) at small size,
    including s = 10."""
    from paper_2402_15033_gb300 import capi
    A = synth.laplace3d(N)
    b = kr.as_operator(A) @ synth.x_true(A.n, 0)
    mixed_vs_oracle(capi, A, b, 60, s, 60)


def test_mixed_convection_diffusion(lib):
    from paper_2402_15033_gb300 import capi
    A = synth.convdiff2d(50, 3)
    b = kr.as_operator(A) @ synth.x_true(A.n, 4)
    mixed_vs_oracle(capi, A, b, 30, 5, 30)


@pytest.mark.parametrize("gen,N,s,m", [("laplace2d", 64, 10, 60), ("laplace3d", 24, 10, 60), ("convdiff2d", 50, 5, 30),
                                       ("laplace2d", 48, 15, 60)])
def test_mixed_double_float_gram_newton_auto(lib, gen, N, s, m):
    """The served configuration: FP32 basis and MPK, every Gram accumulated in
    double-float (about 2^-48, on the FP32 pipe) instead of FP64, FP64 Cholesky,
    Hessenberg and refinement, Newton basis with automatic shifts.  Converges to
    1e-8, x within 1e-6 of the FP64 oracle's, iterations within m of the
    oracle's mixed-precision arm (FP64 Gram accumulation, same shifts rule)."""
    from paper_2402_15033_gb300 import capi
    A = getattr(synth, gen)(N) if gen != "convdiff2d" else synth.convdiff2d(N, 3)
    M = kr.as_operator(A)
    b = M @ synth.x_true(A.n, 0)
    S = capi.Solver.from_csr(A, capi.default_opts(m=m, s=s, panel=m, tol=1e-8, precision=capi.GMRES_PREC_MIXED,
                                                  arith=capi.GMRES_ARITH_DD, basis=capi.GMRES_BASIS_NEWTON_AUTO))
    x = np.zeros(A.n)
    rc, res = S.solve(b, x)
    S.close()
    assert rc == capi.GMRES_OK, (res, capi.last_error())
    assert np.linalg.norm(b - M @ x) / np.linalg.norm(b) <= 1e-8
    xm, im = kr.sstep_gmres(A, b, m=m, s=s, panel=m, tol=1e-8, basis_dtype=np.float32, theta="auto")
    x64, i64 = kr.sstep_gmres(A, b, m=m, s=s, panel=m, tol=1e-8, theta="auto")
    assert im["status"] == 0 and i64["status"] == 0
    assert abs(res["iters"] - im["iters"]) <= m, (res["iters"], im["iters"])
    assert np.linalg.norm(x - x64) / np.linalg.norm(x64) <= 1e-6
    assert np.allclose(res["theta"][:s], im["theta"], atol=1e-5 * np.abs(im["theta"]).max())
