"""Parity of the standalone two-stage orthogonalization calls (stage 1 and
stage 2, one BCGS-PIP each, §IV-C Fig. 4a and §V Fig. 5) with the CPU oracle.

Tolerance (FP64 in and out, double-float arithmetic of ~2^-48 relative
accuracy inside): every R entry within 1e-12 * ||R[:, j]||_2 (the column norm
equals ||V[:, j]||, the scale of the Gram entries it comes from), widened by
kappa(T)/100 for blocks with kappa(T) > 100, and every output column of Q^
within 1e-12 * kappa_T of the oracle's, where kappa_T is the condition number
of T (the triangular solve amplifies rounding differences by at most that
factor).
"""
import numpy as np
import pytest
import torch

import synth
from oracle import blockortho as bo

pytestmark = pytest.mark.gpu


def colmajor(a, dev="cuda"):
    """numpy (n, c) -> CUDA tensor view with column-major layout (stride (1, n))."""
    return torch.tensor(np.asarray(a).T.copy(), dtype=torch.float64, device=dev).T


def run_pip(capi, Q, V, stage=1, ld_pad=0):
    n, nb = V.shape
    k = 0 if Q is None else Q.shape[1]
    ld = n + ld_pad
    buf = torch.zeros(k + nb, ld, dtype=torch.float64, device="cuda")
    if k:
        buf[:k, :n] = torch.tensor(Q.T)
    buf[k:, :n] = torch.tensor(V.T)
    Qd = buf[:k].T[:n] if k else None
    Vd = buf[k:].T[:n]
    R = torch.full((nb, k + nb + 3), np.nan, dtype=torch.float64, device="cuda").T
    work = torch.empty(capi.workspace_bytes(n, k, nb), dtype=torch.uint8, device="cuda")
    st = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    fn = capi.ortho_stage1 if stage == 1 else capi.ortho_stage2
    fn(Qd, Vd, R, work, st, k=k)
    torch.cuda.synchronize()
    return Vd.cpu().numpy(), R[: k + nb].cpu().numpy(), int(st.item())


def assert_pip_parity(Q, V, Vg, Rg, st):
    k = 0 if Q is None else Q.shape[1]
    Qh, P, T = bo.bcgs_pip(np.zeros((V.shape[0], 0)) if Q is None else Q, V)
    Rref = np.concatenate([P, T], 0)
    assert st == 0
    scale = np.linalg.norm(Rref, axis=0)
    # The Gram is accurate to ~2^-48 (double-float); Cholesky passes that on to R
    # amplified by up to kappa(T): 1e-12 for well-conditioned blocks, scaled by
    # kappa(T)/100 beyond that.
    tol = 1e-12 * max(1.0, np.linalg.cond(T) / 100.0)
    assert np.all(np.abs(Rg - Rref) <= tol * scale[None, :]), np.max(np.abs(Rg - Rref) / scale)
    assert np.all(np.tril(Rg[k:], -1) == 0.0)
    kap = np.linalg.cond(T)
    err = np.linalg.norm(Vg - Qh, axis=0)
    assert np.all(err <= 1e-12 * max(1.0, kap)), (err.max(), kap)


@pytest.mark.parametrize("n,k,nb", [(1, 0, 1), (37, 0, 5), (129, 1, 5), (4099, 6, 5), (5000, 56, 5),
                                    (12345, 11, 10), (3001, 30, 16), (777, 3, 1)])
def test_stage1_matches_oracle(lib, n, k, nb):
    from paper_2402_15033_gb300 import capi
    g = synth.rng(100 + n + k)
    if n < k + nb:
        pytest.skip("needs n >= k + nb")
    Q = bo.hhqr(g.standard_normal((n, k)))[0] if k else None
    V = g.standard_normal((n, nb)) + (Q @ g.standard_normal((k, nb)) if k else 0.0)
    Vg, Rg, st = run_pip(capi, Q, V, stage=1, ld_pad=(n % 2))
    assert_pip_parity(Q, V, Vg, Rg, st)


@pytest.mark.parametrize("n,k,nb", [(61, 0, 61), (2000, 0, 61), (70001, 0, 61), (3333, 20, 21),
                                    (4000, 70, 40), (9000, 0, 17), (5000, 120, 64), (3001, 192, 64)])
def test_stage2_matches_oracle(lib, n, k, nb):
    from paper_2402_15033_gb300 import capi
    g = synth.rng(200 + n + k)
    Q = bo.hhqr(g.standard_normal((n, k)))[0] if k else None
    V = g.standard_normal((n, nb)) / np.sqrt(n)
    Vg, Rg, st = run_pip(capi, Q, V, stage=2)
    assert_pip_parity(Q, V, Vg, Rg, st)


def test_two_stage_sequence_matches_oracle_on_ill_conditioned_panels(lib):
    """Blocks of the glued matrix (panel kappa 1e5): stage 1 per block, then
    stage 2 on the whole big panel.  After stage 2 ||I - Q^T Q|| = O(eps)
    (Theorem 3) on the GPU as well, and R agrees with the oracle within the
    attainable kappa^2 eps level of the stage-1 Cholesky (Eq. 2)."""
    from paper_2402_15033_gb300 import capi
    n, s, nblk = 20000, 5, 6
    V = synth.glued(n, s, nblk, 1e5, seed=9)
    Qref, Rt, Rd, Qhat_ref = bo.two_stage_panel(np.zeros((n, 0)), [V[:, i * s:(i + 1) * s] for i in range(nblk)])
    ncol = s * nblk
    buf = torch.tensor(V.T.copy(), device="cuda")
    B = buf.T
    Rh = torch.zeros(ncol, ncol, dtype=torch.float64, device="cuda").T
    work = torch.empty(capi.workspace_bytes(n, ncol, ncol), dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    for j in range(nblk):
        c0 = j * s
        capi.ortho_stage1(B[:, :c0] if c0 else None, B[:, c0:c0 + s], Rh[:c0 + s, c0:c0 + s], work, st, k=c0)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
    Qhat = B.cpu().numpy()
    from oracle import checks
    assert checks.cond2(Qhat) < 10
    R2 = torch.zeros(ncol, ncol, dtype=torch.float64, device="cuda").T
    capi.ortho_stage2(None, B, R2, work, st, k=0)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Qg = B.cpu().numpy()
    assert checks.orth_error(Qg)[0] < 100 * np.finfo(float).eps
    Rfin = R2.cpu().numpy() @ Rh.cpu().numpy()
    assert np.allclose(Rfin, Rd, rtol=0, atol=1e-9 * np.abs(Rd).max())
    assert np.allclose(Qg @ Rfin, V, atol=1e-12 * np.abs(V).max())


def test_breakdown_status_and_v_untouched(lib):
    """A block with a zero column has a singular Gram (violates Eq. (1)):
    d_status reports the 1-based pivot and V is left unchanged."""
    from paper_2402_15033_gb300 import capi
    g = synth.rng(7)
    n = 500
    V = g.standard_normal((n, 5))
    V[:, 3] = 0.0
    Vg, Rg, st = run_pip(capi, None, V, stage=1)
    assert st == 4
    assert np.array_equal(Vg, V)


def test_nan_input_is_a_breakdown_not_a_fault(lib):
    from paper_2402_15033_gb300 import capi
    V = synth.rng(8).standard_normal((300, 4))
    V[17, 2] = np.nan
    Vg, Rg, st = run_pip(capi, None, V, stage=1)
    assert st == 3


def test_workspace_reuse_and_repeatability(lib):
    """Two calls on the same workspace give bit-identical results (the
    second-level reduce runs in a fixed CTA order and the counters re-arm)."""
    from paper_2402_15033_gb300 import capi
    g = synth.rng(9)
    n, k, nb = 100003, 20, 5
    Q = bo.hhqr(g.standard_normal((n, k)))[0]
    V = g.standard_normal((n, nb))
    a = run_pip(capi, Q, V)
    b = run_pip(capi, Q, V)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.slow
def test_full_size_ortho_bench_sampled(lib):
    """The benchmark's workload (n = 4,194,304 x 61, column 0 plus 12 blocks of
    5 through stage 1, then stage 2 on all 61 columns) against the oracle: all
    R entries, and sampled rows of the final Q."""
    from paper_2402_15033_gb300 import capi
    n, s, nblk = 4194304, 5, 12
    ncol = 1 + s * nblk
    B0 = synth.tall_basis(n, ncol, seed=1)
    buf = torch.tensor(B0.T.copy(), device="cuda")
    B = buf.T
    B[:, 0] /= torch.linalg.norm(B[:, 0])
    Rh = torch.zeros(ncol, ncol, dtype=torch.float64, device="cuda").T
    work = torch.empty(capi.workspace_bytes(n, ncol, ncol), dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    for j in range(nblk):
        c0 = 1 + j * s
        capi.ortho_stage1(B[:, :c0], B[:, c0:c0 + s], Rh[:c0 + s, c0:c0 + s], work, st, k=c0)
    R2 = torch.zeros(ncol, ncol, dtype=torch.float64, device="cuda").T
    capi.ortho_stage2(None, B, R2, work, st, k=0)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    # oracle on the same input
    X = np.array(B0, copy=True)
    X[:, 0] /= np.linalg.norm(X[:, 0])
    Rh_ref = np.zeros((ncol, ncol))
    for j in range(nblk):
        c0 = 1 + j * s
        Qh, P, T = bo.stage1(X[:, :c0], X[:, c0:c0 + s])
        X[:, c0:c0 + s] = Qh
        Rh_ref[:c0, c0:c0 + s] = P
        Rh_ref[c0:c0 + s, c0:c0 + s] = T
    Qf, _, T2 = bo.stage2(np.zeros((n, 0)), X)
    R2g = R2.cpu().numpy()
    Rhg = Rh.cpu().numpy()
    sc = np.linalg.norm(T2, axis=0)
    assert np.all(np.abs(R2g - T2) <= 1e-12 * sc[None, :])
    msk = np.triu(np.ones((ncol, ncol), bool), 1)
    msk[:, 0] = False
    scale = np.maximum(np.linalg.norm(Rh_ref, axis=0), 1e-300)
    assert np.all(np.abs(Rhg - Rh_ref)[msk] <= (1e-12 * scale[None, :].repeat(ncol, 0))[msk])
    rows = synth.rng(3).choice(n, 4096, replace=False)
    Qs = B[torch.tensor(rows, device="cuda")].cpu().numpy()
    assert np.max(np.abs(Qs - Qf[rows])) <= 1e-12


def run_pip_dd(capi, Q, V, ld_pad=0):
    """ortho_gram_chol_dd + ortho_update_dd (double-float arithmetic)."""
    n, nb = V.shape
    k = 0 if Q is None else Q.shape[1]
    ld = n + ld_pad
    buf = torch.zeros(k + nb, ld, dtype=torch.float64, device="cuda")
    if k:
        buf[:k, :n] = torch.tensor(Q.T)
    buf[k:, :n] = torch.tensor(V.T)
    Qd = buf[:k].T[:n] if k else None
    Vd = buf[k:].T[:n]
    R = torch.zeros(nb, k + nb, dtype=torch.float64, device="cuda").T
    work = torch.empty(capi.workspace_bytes(n, k, nb), dtype=torch.uint8, device="cuda")
    st = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    capi.ortho_gram_chol_dd(Qd, Vd, R, work, st, k=k)
    capi.ortho_update(Qd, Vd, R, st, k=k, dd=True)
    torch.cuda.synchronize()
    return Vd.cpu().numpy(), R.cpu().numpy(), int(st.item())


@pytest.mark.parametrize("n,k,nb", [(40003, 0, 5), (40003, 30, 5), (30001, 0, 61), (20011, 20, 21), (9999, 3, 12)])
def test_double_float_halves_match_oracle(lib, n, k, nb):
    """GMRES_ARITH_DD (opt-in): same parity bars on well-conditioned blocks."""
    from paper_2402_15033_gb300 import capi
    g = synth.rng(400 + n + k)
    Q = bo.hhqr(g.standard_normal((n, k)))[0] if k else None
    V = g.standard_normal((n, nb)) / np.sqrt(n) + (Q @ g.standard_normal((k, nb)) / 4 if k else 0.0)
    Vg, Rg, st = run_pip_dd(capi, Q, V, ld_pad=n % 2)
    assert_pip_parity(Q, V, Vg, Rg, st)


@pytest.mark.parametrize("scale_exp", [-40, -20, 20, 40])
def test_double_float_range(lib, scale_exp):
    """The double-float kernels keep their relative accuracy for inputs scaled
    within the documented range: R scales exactly with the input, Q^ does not
    change."""
    from paper_2402_15033_gb300 import capi
    g = synth.rng(77)
    n, k, nb = 20011, 7, 5
    Q = bo.hhqr(g.standard_normal((n, k)))[0]
    V = g.standard_normal((n, nb))
    sc = 2.0 ** scale_exp
    Vg, Rg, st = run_pip_dd(capi, Q, V * sc, ld_pad=1)
    assert st == 0
    Qh, P, T = bo.bcgs_pip(Q, V)
    Rref = np.concatenate([P, T], 0) * sc
    scale = np.linalg.norm(Rref, axis=0)
    assert np.all(np.abs(Rg - Rref) <= 1e-12 * scale[None, :])
    assert np.max(np.abs(Vg - Qh)) <= 1e-12
