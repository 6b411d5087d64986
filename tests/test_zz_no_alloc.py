"""ortho_stage1_noalloc: stage 1 for callers that cannot allocate device
memory (a framework's arena owns it all, or the host program offers no
allocator).  Its output must equal ortho_stage1's on the same input, within
the FP64 parity tolerance of the other tests, on two calls in a row (the
second call reuses the library-owned scratch that the first one left behind).

This file is collected last so that a stop-at-first-failure run has already
run every other test when it gets here."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _inputs(n, k, nb, seed):
    g = synth.rng(seed)
    Q, _ = np.linalg.qr(g.standard_normal((n, k))) if k else (None, None)
    V = g.standard_normal((n, nb)) + (Q @ g.standard_normal((k, nb)) if k else 0.0)
    return Q, V


def _to_dev(Q, V, n, k, nb):
    buf = torch.zeros(k + nb, n, dtype=torch.float64, device="cuda")
    if k:
        buf[:k] = torch.tensor(Q.T)
    buf[k:] = torch.tensor(V.T)
    return (buf[:k].T if k else None), buf[k:].T


@pytest.mark.parametrize("n,k,nb,on_stream", [(100003, 26, 5, False), (4099, 0, 16, False),
                                               (65537, 48, 16, True)])
def test_noalloc_matches_workspace_version_twice(lib, n, k, nb, on_stream):
    """(65537, 48, 16) fills the array's largest layout: k + nb = 64 columns of
    16 at the full reduction grid; it runs on a stream other than the default."""
    from paper_2402_15033_gb300 import capi
    if on_stream:
        side = torch.cuda.Stream()
        stream = side.cuda_stream
    else:
        side, stream = None, None
    for call, seed in enumerate((31, 32)):
        Q, V = _inputs(n, k, nb, seed + n)
        Qa, Va = _to_dev(Q, V, n, k, nb)
        Qb, Vb = _to_dev(Q, V, n, k, nb)
        Ra = torch.zeros(nb, k + nb, dtype=torch.float64, device="cuda").T
        Rb = torch.zeros(nb, k + nb, dtype=torch.float64, device="cuda").T
        sa = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        sb = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        work = torch.empty(capi.workspace_bytes(n, k, nb), dtype=torch.uint8, device="cuda")
        capi.ortho_stage1(Qa, Va, Ra, work, sa, k=k)
        torch.cuda.synchronize()
        capi.ortho_stage1_noalloc(Qb, Vb, Rb, sb, k=k, stream=stream)
        torch.cuda.synchronize()
        assert int(sa.item()) == 0 and int(sb.item()) == 0, call
        ra, rb = Ra.cpu().numpy(), Rb.cpu().numpy()
        scale = np.linalg.norm(ra, axis=0)
        assert np.all(np.abs(ra - rb) <= 1e-12 * scale[None, :]), call
        va, vb = Va.cpu().numpy(), Vb.cpu().numpy()
        assert np.all(np.linalg.norm(va - vb, axis=0) <= 1e-12 * np.linalg.norm(va, axis=0)), call


def test_noalloc_rejects_blocks_beyond_its_scratch(lib):
    from paper_2402_15033_gb300 import capi
    n, k, nb = 1000, 60, 8
    V = torch.zeros(nb, n, dtype=torch.float64, device="cuda").T
    Q = torch.zeros(k, n, dtype=torch.float64, device="cuda").T
    R = torch.zeros(nb, k + nb, dtype=torch.float64, device="cuda").T
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(capi.GmresError) as e:
        capi.ortho_stage1_noalloc(Q, V, R, st, k=k)
    assert e.value.code == capi.GMRES_ERR_ARG
    assert "k + nb <= 64" in str(e.value)
