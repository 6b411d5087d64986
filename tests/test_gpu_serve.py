"""Serving loop with continuous batching: requests of different sizes,
matrices and options, admitted by device footprint, served concurrently; each
result is the same alone and in the mix."""
import time

import numpy as np
import pytest

import synth
from oracle import krylov as kr

pytestmark = pytest.mark.gpu


def requests(seed):
    """2D Laplace and 3D upwinded convection-diffusion, s in {5, 10},
    m in {30, 60}, FP64 and mixed precision: the serving configuration's mix
    at test scale."""
    from paper_2402_15033_gb300 import capi
    g = synth.rng(seed)
    out = []
    for i in range(8):
        if i % 2 == 0:
            A = synth.laplace2d(int(g.choice([24, 32, 40, 48])))
        else:
            A = synth.convdiff3d(int(g.choice([10, 12, 14])), seed * 100 + i)
        s = int(g.choice([5, 10]))
        m = int(g.choice([30, 60]))
        prec = capi.GMRES_PREC_MIXED if i % 3 == 0 else capi.GMRES_PREC_FP64
        panel = 10 if s == 10 else (m if i % 4 else 10)
        o = capi.default_opts(m=m, s=s, panel=panel, tol=1e-8, precision=prec, max_restarts=400)
        b = kr.as_operator(A) @ synth.x_true(A.n, i)
        out.append((A, b, o))
    return out


def test_served_results_equal_lone_solves(lib):
    from paper_2402_15033_gb300 import capi
    reqs = requests(5)
    srv = capi.Server(max_active=8)
    ids = [srv.submit(A, b, opts=o) for A, b, o in reqs]
    got = [srv.wait(i) for i in ids]
    st = srv.stats()
    srv.stop()
    assert st["completed"] == len(reqs) and st["mem_in_use"] == 0
    assert st["p99_ms"] >= st["p50_ms"] > 0 and st["solves_per_s"] > 0
    for (A, b, o), (x, r) in zip(reqs, got):
        S = capi.Solver.from_csr(A, o)
        x1 = np.zeros(A.n)
        rc1, r1 = S.solve(b, x1)
        S.close()
        assert r["status"] == rc1, (A.name, r["status"], rc1)
        assert r["iters"] == r1["iters"]
        assert np.array_equal(x, x1), A.name
        if rc1 == 0:
            assert np.linalg.norm(b - kr.as_operator(A) @ x) / np.linalg.norm(b) <= 1e-8


def test_admission_by_footprint_serializes_under_a_tight_budget(lib):
    from paper_2402_15033_gb300 import capi
    reqs = requests(6)
    fps = [capi.footprint(A.n, A.nnz, o) for A, b, o in reqs]
    srv = capi.Server(mem_budget=max(fps) + 1024, max_active=8)
    ids = [srv.submit(A, b, opts=o) for A, b, o in reqs]
    res = [srv.wait(i) for i in ids]
    st = srv.stats()
    srv.stop()
    assert st["completed"] == len(reqs) and st["rejected"] == 0
    assert all(r[1]["status"] in (0, 1, -4) for r in res)


def test_request_larger_than_the_budget_is_rejected(lib):
    from paper_2402_15033_gb300 import capi
    A = synth.laplace2d(64)
    b = kr.as_operator(A) @ synth.x_true(A.n, 0)
    srv = capi.Server(mem_budget=1 << 20, max_active=2)
    rid = srv.submit(A, b)
    x, r = srv.wait(rid)
    st = srv.stats()
    srv.stop()
    assert r["status"] == capi.GMRES_ERR_OOM and st["rejected"] == 1


def test_wait_on_an_unknown_or_collected_id_is_an_argument_error(lib):
    """wait returns GMRES_ERR_ARG, without blocking, for an id the server never
    issued and for one whose result was already collected."""
    import ctypes as C
    from paper_2402_15033_gb300 import capi
    A = synth.laplace2d(16)
    b = kr.as_operator(A) @ synth.x_true(A.n, 0)
    srv = capi.Server(max_active=2)
    rid = srv.submit(A, b, opts=capi.default_opts(m=30, s=5, panel=30))
    x, r = srv.wait(rid)
    assert r["status"] == 0
    wait = capi.load().gmres_server_wait
    res = capi.gmres_result()
    assert wait(srv.h, rid, None, C.byref(res), -1.0) == capi.GMRES_ERR_ARG
    assert wait(srv.h, rid + 1000, None, C.byref(res), -1.0) == capi.GMRES_ERR_ARG
    srv.stop()


def test_late_small_request_overtakes_a_running_long_one(lib):
    """Continuous batching, not a queue: a small request submitted after a long
    one has started is admitted alongside it and finishes first."""
    from paper_2402_15033_gb300 import capi
    big = synth.laplace2d(512)
    bb = kr.as_operator(big) @ synth.x_true(big.n, 0)
    small = synth.laplace2d(16)
    bs = kr.as_operator(small) @ synth.x_true(small.n, 1)
    srv = capi.Server(max_active=4)
    # a tolerance near the FP64 floor: the long solve runs hundreds of cycles
    rb = srv.submit(big, bb, opts=capi.default_opts(m=60, s=5, panel=60, tol=1e-15, max_restarts=400))
    time.sleep(0.2)
    rs = srv.submit(small, bs, opts=capi.default_opts(m=20, s=5, panel=20, tol=1e-8))
    xs, r_small = srv.wait(rs)
    assert srv.wait(rb, timeout=0.0) is None      # the long solve is still running
    xb, r_big = srv.wait(rb)
    srv.stop()
    assert r_small["status"] == 0
    assert r_big["status"] in (capi.GMRES_OK, capi.GMRES_WARN_MAXIT)
    assert r_big["restarts"] > r_small["restarts"]


def test_served_mixed_double_float_newton_requests_equal_lone_solves(lib):
    """The benchmark's served configuration (FP32 basis, double-float Gram,
    Newton basis with automatic shifts) gives every request the same result in
    the mix as alone, bit for bit."""
    from paper_2402_15033_gb300 import capi
    reqs = []
    for i, A in enumerate([synth.laplace2d(40), synth.convdiff3d(14, 5), synth.laplace2d(64), synth.convdiff3d(12, 9)]):
        b = kr.as_operator(A) @ synth.x_true(A.n, i)
        o = capi.default_opts(m=30 if i % 2 else 60, s=10 if i < 2 else 5, panel=30 if i % 2 else 60, tol=1e-8,
                              precision=capi.GMRES_PREC_MIXED, arith=capi.GMRES_ARITH_DD,
                              basis=capi.GMRES_BASIS_NEWTON_AUTO, max_restarts=400)
        reqs.append((A, b, o))
    srv = capi.Server(max_active=8)
    ids = [srv.submit(A, b, opts=o) for A, b, o in reqs]
    got = [srv.wait(i) for i in ids]
    srv.stop()
    for (A, b, o), (x, r) in zip(reqs, got):
        S = capi.Solver.from_csr(A, o)
        x1 = np.zeros(A.n)
        rc1, r1 = S.solve(b, x1)
        S.close()
        assert r["status"] == rc1 == 0, (A.name, r["status"], rc1)
        assert r["iters"] == r1["iters"] and r["theta"] == r1["theta"]
        assert np.array_equal(x, x1), A.name
        assert np.linalg.norm(b - kr.as_operator(A) @ x) / np.linalg.norm(b) <= 1e-8
