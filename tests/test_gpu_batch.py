"""Batched solver (many uneven systems per launch, one CUDA graph per restart
cycle) against the oracle, and the property that makes it safe to batch: each
system's result is the same alone and in the mix."""
import numpy as np
import pytest

import synth
from oracle import krylov as kr

pytestmark = pytest.mark.gpu


def mix(nsys, seed, nmin=2000, nmax=20000):
    """Half 2D upwinded convection-diffusion, half random banded (27 nnz/row),
    sizes log-uniform in [nmin, nmax]: the batched configuration's recipe at
    test scale."""
    g = synth.rng(seed)
    mats = []
    for i in range(nsys):
        n = int(np.exp(g.uniform(np.log(nmin), np.log(nmax))))
        if i % 2 == 0:
            mats.append(synth.convdiff2d(int(np.ceil(np.sqrt(n))), seed * 1000 + i))
        else:
            mats.append(synth.banded_random(n, seed * 1000 + i, band=min(1000, n // 4)))
    bs = [kr.as_operator(A) @ synth.x_true(A.n, i) for i, A in enumerate(mats)]
    return mats, bs


def solve_batch(capi, mats, bs, **kw):
    B = capi.Batch(mats, capi.default_opts(**kw))
    xs = [np.zeros(A.n) for A in mats]
    rc, res = B.solve(bs, xs)
    return B, rc, res, xs


def test_mixed_batch_matches_oracle(lib):
    from paper_2402_15033_gb300 import capi
    mats, bs = mix(8, 1)
    B, rc, res, xs = solve_batch(capi, mats, bs, m=40, s=5, panel=40, tol=1e-8, precision=capi.GMRES_PREC_MIXED)
    B.close()
    assert rc == capi.GMRES_OK, [r["status"] for r in res]
    for A, b, x, r in zip(mats, bs, xs, res):
        M = kr.as_operator(A)
        assert np.linalg.norm(b - M @ x) / np.linalg.norm(b) <= 1e-8
        xm, im = kr.sstep_gmres(A, b, m=40, s=5, panel=40, tol=1e-8, basis_dtype=np.float32)
        assert im["status"] == 0
        assert abs(r["iters"] - im["iters"]) <= 40, (A.name, r["iters"], im["iters"])
        assert np.linalg.norm(x - xm) / np.linalg.norm(xm) <= 1e-6


def test_fp64_batch_matches_single_solver(lib):
    """The batch and the single-system solver run the same kernels: same status
    and iteration count per system, x equal up to the restart residual's
    summation order; converged systems also match the oracle."""
    from paper_2402_15033_gb300 import capi
    mats = [synth.laplace2d(N) for N in (20, 33, 47, 64)] + [synth.convdiff2d(40, 3)]
    bs = [kr.as_operator(A) @ synth.x_true(A.n, 0) for A in mats]
    B, rc, res, xs = solve_batch(capi, mats, bs, m=60, s=5, panel=60, tol=1e-8)
    B.close()
    for A, b, x, r in zip(mats, bs, xs, res):
        S = capi.Solver.from_csr(A, capi.default_opts(m=60, s=5, panel=60, tol=1e-8))
        xsg = np.zeros(A.n)
        rc1, r1 = S.solve(b, xsg)
        S.close()
        assert rc1 == r["status"], (A.name, rc1, r["status"])
        if rc1 != 0:
            continue
        assert r1["iters"] == r["iters"], (A.name, r1["iters"], r["iters"])
        assert np.linalg.norm(x - xsg) / np.linalg.norm(xsg) <= 1e-10
        xo, io = kr.sstep_gmres(A, b, m=60, s=5, panel=60, tol=1e-8)
        if io["status"] == kr.STATUS_BREAKDOWN:
            # the oracle's pivot is decided by rounding (the Pythagorean
            # shortcut's error exceeds the projected block's smallest Gram
            # eigenvalue, margin < 1): the GPU's converged residual is verified
            # on the host instead
            assert io["breakdown_margin"] < 1.0, (A.name, io["where"], io["breakdown_margin"])
            assert np.linalg.norm(b - kr.as_operator(A) @ x) / np.linalg.norm(b) <= 1e-8
            continue
        assert abs(io["iters"] - r["iters"]) <= 5
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-6
    assert sum(1 for r in res if r["status"] == 0) >= 4


def test_same_result_alone_and_in_the_mix(lib):
    """Each system solved in a batch of one and inside the full batch gives
    bit-identical x and the same iteration count: per-system reductions use a
    split and order that depend on that system alone."""
    from paper_2402_15033_gb300 import capi
    mats, bs = mix(6, 2)
    kw = dict(m=40, s=5, panel=40, tol=1e-8, precision=capi.GMRES_PREC_MIXED)
    B, rc, res, xs = solve_batch(capi, mats, bs, **kw)
    B.close()
    for i, (A, b) in enumerate(zip(mats, bs)):
        B1, rc1, res1, xs1 = solve_batch(capi, [A], [b], **kw)
        B1.close()
        assert res1[0]["status"] == res[i]["status"]
        assert res1[0]["iters"] == res[i]["iters"]
        assert np.array_equal(xs1[0], xs[i]), i


def test_autotune_changes_speed_not_results(lib):
    from paper_2402_15033_gb300 import capi
    mats, bs = mix(5, 3)
    B = capi.Batch(mats, capi.default_opts(m=40, s=5, panel=40, tol=1e-8, precision=capi.GMRES_PREC_MIXED))
    x1 = [np.zeros(A.n) for A in mats]
    rc1, r1 = B.solve(bs, x1)
    t = B.autotune()
    assert t["gram_grid"] >= 1 and t["row_grid"] >= 1 and t["gram_ms"] > 0
    x2 = [np.zeros(A.n) for A in mats]
    rc2, r2 = B.solve(bs, x2)
    B.close()
    assert rc1 == rc2 == capi.GMRES_OK
    for a, b in zip(x1, x2):
        assert np.array_equal(a, b)


def test_breakdown_in_one_system_leaves_the_others_alone(lib):
    from paper_2402_15033_gb300 import capi
    n = 500
    bad = synth.CSR(n, np.arange(n + 1), np.arange(n, dtype=np.int32), np.full(n, 2.0))
    good = synth.laplace2d(30)
    mats = [good, bad, synth.laplace2d(25)]
    bs = [kr.as_operator(A) @ synth.x_true(A.n, 1) for A in mats]
    B, rc, res, xs = solve_batch(capi, mats, bs, m=20, s=5, panel=20, tol=1e-8)
    B.close()
    assert rc == capi.GMRES_ERR_BREAKDOWN
    assert res[1]["status"] == capi.GMRES_ERR_BREAKDOWN and res[1]["breakdown_block"] == 0
    for i in (0, 2):
        assert res[i]["status"] == 0 and res[i]["relres_true"] <= 1e-8


def test_footprint_counts_the_basis(lib):
    from paper_2402_15033_gb300 import capi
    mats, _ = mix(3, 4)
    o = capi.default_opts(m=40, s=5, panel=40, precision=capi.GMRES_PREC_MIXED)
    f = capi.Batch.footprint(mats, o)
    rows = sum((A.n + 31) // 32 * 32 for A in mats)
    assert f >= rows * 41 * 4
