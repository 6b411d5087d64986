"""ortho_plan: the two-stage orthogonalization of one panel in one library
call, on host and device buffers.  It runs the same kernels in the same order
as the ortho_* calls, so its outputs equal theirs bit for bit (FP64 and
tensor-core arithmetic, host and device pointers, two runs in a row on one
plan); a breakdown comes back as GMRES_ERR_BREAKDOWN with the block's status."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def calls(capi, B, s, nblk, tc):
    """The benchmark's sequence through the ortho_* calls on the device view B."""
    n, ncol = B.shape
    Rh = torch.zeros(ncol, ncol, dtype=torch.float64, device="cuda").T
    R2 = torch.zeros(ncol, ncol, dtype=torch.float64, device="cuda").T
    work = torch.empty(capi.workspace_bytes(n, ncol, ncol), dtype=torch.uint8, device="cuda")
    st = torch.zeros(nblk + 1, dtype=torch.int32, device="cuda")
    dig = torch.zeros(capi.digits_bytes(n, ncol), dtype=torch.uint8, device="cuda")
    if tc:
        capi.digits_fill(B[:, :1], 0, dig, ncol)
    for j in range(nblk):
        k = 1 + s * j
        Q, V, Rb = B[:, :k], B[:, k:k + s], Rh[:k + s, k:k + s]
        if tc:
            capi.ortho_gram_chol_tcd(Q, V, Rb, work, st[j:j + 1], dig, ncol, k, k=k)
            capi.ortho_update_tcd(Q, V, Rb, st[j:j + 1], dig, ncol, k=k)
        else:
            capi.ortho_stage1(Q, V, Rb, work, st[j:j + 1], k=k)
    if tc:
        capi.ortho_gram_chol_tcd(None, B, R2, work, st[nblk:], dig, ncol, ncol, k=0)
        capi.ortho_update(None, B, R2, st[nblk:], k=0, tc=True)
    else:
        capi.ortho_stage2(None, B, R2, work, st[nblk:], k=0)
    torch.cuda.synchronize()
    return B.cpu().numpy(), Rh.cpu().numpy(), R2.cpu().numpy()


@pytest.mark.parametrize("n,s,nblk,tc", [(100003, 5, 12, True), (100003, 5, 12, False), (4096, 10, 6, True),
                                         (70001, 3, 3, False)])
def test_plan_equals_the_ortho_calls_on_host_and_device(lib, n, s, nblk, tc):
    from paper_2402_15033_gb300 import capi
    ncol = 1 + s * nblk
    X = synth.tall_basis(n, ncol, seed=21)
    X[:, 0] /= np.linalg.norm(X[:, 0])
    buf = torch.zeros(ncol, n + n % 2, dtype=torch.float64, device="cuda")    # 16-byte aligned columns
    buf[:, :n] = torch.tensor(X.T.copy())
    ref_Q, ref_Rh, ref_R2 = calls(capi, buf.T[:n], s, nblk, tc)
    plan = capi.OrthoPlan(n, s, nblk, capi.GMRES_ARITH_TC if tc else capi.GMRES_ARITH_FP64)
    # host buffers (page-locked), two runs in a row
    Xh = torch.tensor(X.T.copy()).pin_memory()
    for _ in range(2):
        Qh = torch.empty_like(Xh).pin_memory()
        Rh = torch.full((ncol, ncol), np.nan, dtype=torch.float64).pin_memory()
        R2 = torch.full((ncol, ncol), np.nan, dtype=torch.float64).pin_memory()
        rc, st = plan.run(Xh.T, Qh.T, Rh.T, R2.T, on_device=False)
        assert rc == 0 and not any(st)
        assert np.array_equal(Qh.T.numpy(), ref_Q)
        assert np.array_equal(R2.T.numpy(), ref_R2)
        blk = ~np.tril(np.ones((ncol, ncol), bool))
        blk[:, 0] = False
        assert np.array_equal(Rh.T.numpy()[blk], ref_Rh[blk])
    # device buffers, in place (X = Q)
    Xd = torch.tensor(X.T.copy(), device="cuda")
    R2d = torch.zeros(ncol, ncol, dtype=torch.float64, device="cuda")
    rc, st = plan.run(Xd.T, Xd.T, None, R2d.T, on_device=True)
    assert rc == 0
    assert np.array_equal(Xd.T.cpu().numpy(), ref_Q) and np.array_equal(R2d.T.cpu().numpy(), ref_R2)
    plan.close()


def test_plan_reports_a_breakdown(lib):
    from paper_2402_15033_gb300 import capi
    n, s, nblk = 5000, 5, 3
    ncol = 1 + s * nblk
    X = synth.tall_basis(n, ncol, seed=22)
    X[:, 0] /= np.linalg.norm(X[:, 0])
    X[:, 8] = 0.0                             # block 1 holds a zero column: its Gram is singular
    plan = capi.OrthoPlan(n, s, nblk, capi.GMRES_ARITH_FP64)
    Q = np.empty_like(X, order="F")
    rc, st = plan.run(np.asfortranarray(X), Q, on_device=False)
    plan.close()
    assert rc == capi.GMRES_ERR_BREAKDOWN and st[0] == 0 and st[1] > 0
