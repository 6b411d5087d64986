"""The synthetic orthogonality experiment of §VI (Figs. 3-4) on the CUDA
kernels: the glued sweep, six blocks of five columns whose own condition
number is fixed (1e3) while the whole panel's is swept.  Each block goes
through stage 1 (one BCGS-PIP against all accumulated columns), then the big
panel through stage 2, in the three arithmetics (FP64 pipe, exact-slice
tensor cores, tensor cores with the digit basis).

Bars, from the paper's bounds (eps = 2^-52):
* after stage 1, ||I - Q^^T Q^|| at most 10 kappa^2 eps (Eq. 10, an upper
  bound) and at least 1e-3 kappa^2 eps (not a bound of the paper: it shows the
  sweep reaches the kappa^2 eps regime; the GPU's fixed-order FMA sums lose
  somewhat less than the oracle's, about 0.008 kappa^2 eps at kappa 1.4e6),
  and kappa(Q^) < 2 (Eq. 11);
* after stage 2, ||I - Q^T Q|| < 100 eps (Theorem 3) and V = Q R to 1e-13;
* R (stage 2 times stage 1) within 100 kappa eps ||R|| of the oracle's (the
  perturbation bound of a QR factor for a backward-stable method);
* beyond eps^(-1/2) (total condition 1e11) a stage-1 Cholesky breaks down and
  is reported (the assumption of Eq. 9 fails); the oracle's failing pivot there
  is decided by rounding (margin < 1), so the GPU's may be another block's.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import blockortho as bo, checks

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps
N, C, P = 4000, 5, 6


def gpu_two_stage(capi, V, arith):
    """Stage 1 per block and stage 2 on the big panel on the GPU.  Returns
    (Q^ after stage 1, Q, R_stage1, R_stage2, statuses)."""
    n, ncol = V.shape
    buf = torch.tensor(np.asarray(V).T.copy(), device="cuda")
    B = buf.T
    Rh = torch.zeros(ncol, ncol, dtype=torch.float64, device="cuda").T
    R2 = torch.zeros(ncol, ncol, dtype=torch.float64, device="cuda").T
    work = torch.empty(capi.workspace_bytes(n, ncol, ncol), dtype=torch.uint8, device="cuda")
    st = torch.zeros(P + 1, dtype=torch.int32, device="cuda")
    capc = 32
    dig = torch.zeros(capi.digits_bytes(n, capc), dtype=torch.uint8, device="cuda") if arith == "tcd" else None
    for j in range(P):
        k = C * j
        Q = B[:, :k] if k else None
        Vj, Rb, sj = B[:, k:k + C], Rh[:k + C, k:k + C], st[j:j + 1]
        if arith == "fp64":
            capi.ortho_stage1(Q, Vj, Rb, work, sj, k=k)
        elif arith == "tc":
            capi.ortho_gram_chol_tc(Q, Vj, Rb, work, sj, k=k)
            capi.ortho_update(Q, Vj, Rb, sj, k=k, tc=True)
        else:
            capi.ortho_gram_chol_tcd(Q, Vj, Rb, work, sj, dig, capc, k, k=k)
            capi.ortho_update_tcd(Q, Vj, Rb, sj, dig, capc, k=k)
    torch.cuda.synchronize()
    Qhat = B.cpu().numpy().copy()
    s1 = st[:P].cpu().numpy().copy()
    if np.any(s1 != 0):
        return Qhat, None, Rh.cpu().numpy(), None, st.cpu().numpy()
    if arith == "fp64":
        capi.ortho_stage2(None, B, R2, work, st[P:], k=0)
    elif arith == "tc":
        capi.ortho_gram_chol_tc(None, B, R2, work, st[P:], k=0)
        capi.ortho_update(None, B, R2, st[P:], k=0, tc=True)
    else:
        capi.ortho_gram_chol_tcd(None, B, R2, work, st[P:], dig, capc, ncol, k=0)
        capi.ortho_update(None, B, R2, st[P:], k=0, tc=True)
    torch.cuda.synchronize()
    return Qhat, B.cpu().numpy(), Rh.cpu().numpy(), R2.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("arith", ["fp64", "tc", "tcd"])
@pytest.mark.parametrize("seed", [1, 2])
def test_glued_sweep_stage_bounds_on_the_gpu(lib, arith, seed):
    from paper_2402_15033_gb300 import capi
    for km in (1e2, 1e4, 1e6):
        V = synth.glued_sweep(N, C, P, 1e3, km, seed)
        kap = checks.cond2(V)
        Qhat, Q, Rh, R2, st = gpu_two_stage(capi, V, arith)
        assert np.all(st == 0), (km, st)
        e1 = checks.orth_error(Qhat)[0]
        assert 1e-3 * kap ** 2 * EPS <= e1 <= 10 * kap ** 2 * EPS, (km, kap, e1)
        assert checks.cond2(Qhat) < 2.0
        assert checks.orth_error(Q)[0] < 100 * EPS
        R = R2 @ Rh
        assert np.abs(Q @ R - V).max() <= 1e-13 * np.abs(V).max()
        _, _, Rd, _ = bo.two_stage_panel(np.zeros((N, 0)), [V[:, i * C:(i + 1) * C] for i in range(P)])
        assert np.abs(R - Rd).max() <= 100 * kap * EPS * np.abs(Rd).max(), (km, np.abs(R - Rd).max())


@pytest.mark.parametrize("arith", ["fp64", "tc", "tcd"])
def test_glued_sweep_breakdown_beyond_eps_to_the_minus_half(lib, arith):
    from paper_2402_15033_gb300 import capi
    V = synth.glued_sweep(N, C, P, 1e3, 1e10, 1)
    assert checks.cond2(V) > 1e11
    with pytest.raises(bo.Breakdown) as e:
        bo.two_stage_panel(np.zeros((N, 0)), [V[:, i * C:(i + 1) * C] for i in range(P)])
    assert "stage1" in e.value.where and e.value.margin < 1.0
    _, _, _, _, st = gpu_two_stage(capi, V, arith)
    assert np.any(st[:P] != 0), st
    j = int(np.nonzero(st[:P])[0][0])
    assert 1 <= st[j] <= C
