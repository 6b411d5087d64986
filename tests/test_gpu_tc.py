"""Exact-slice tensor-core BCGS-PIP (GMRES_ARITH_TC): parity of
ortho_gram_chol_tc + ortho_update_tc with the CPU oracle's BCGS-PIP (§IV-C,
Fig. 4a), and the properties that pin the slicing itself.

Tolerances.  The slicing keeps 55 bits of every column's largest entry per
64-row chunk (16-row group for V in the streaming narrow Gram) and sums the digit products exactly, so a Gram entry differs
from the exact X^T Y by a few units of 2^-53 of ||x_i|| ||y_j|| per chunk
(normwise, as FP64's own dot-product bound).  The parity bars are those of
the FP64 kernels (1e-12 of the column norm of R, widened by kappa(T)/100);
the exactness test holds the Gram entries to 2^-48 ||x_i|| ||y_j|| against
rational arithmetic.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import blockortho as bo
from oracle import checks

pytestmark = pytest.mark.gpu


def run_pip_tc(capi, Q, V, ld_pad=0, update=True, tc_update=True):
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
    capi.ortho_gram_chol_tc(Qd, Vd, R, work, st, k=k)
    if update:
        capi.ortho_update(Qd, Vd, R, st, k=k, tc=tc_update)
    torch.cuda.synchronize()
    return Vd.cpu().numpy(), R[: k + nb].cpu().numpy(), int(st.item())


def assert_parity(Q, V, Vg, Rg, st):
    k = 0 if Q is None else Q.shape[1]
    Qh, P, T = bo.bcgs_pip(np.zeros((V.shape[0], 0)) if Q is None else Q, V)
    Rref = np.concatenate([P, T], 0)
    assert st == 0
    scale = np.linalg.norm(Rref, axis=0)
    kap = np.linalg.cond(T)
    tol = 1e-12 * max(1.0, kap / 100.0)
    assert np.all(np.abs(Rg - Rref) <= tol * scale[None, :]), np.max(np.abs(Rg - Rref) / scale)
    assert np.all(np.tril(Rg[k:], -1) == 0.0)
    err = np.linalg.norm(Vg - Qh, axis=0)
    assert np.all(err <= 1e-12 * max(1.0, kap)), (err.max(), kap)


@pytest.mark.parametrize("n,k,nb", [
    (1, 0, 1), (37, 0, 5), (128, 0, 5), (129, 1, 5), (4099, 6, 5), (5000, 56, 5), (70001, 59, 5),
    (12345, 11, 10), (3001, 30, 16), (777, 3, 1), (61, 0, 61), (2000, 0, 61), (70001, 0, 61),
    (3333, 20, 21), (9000, 0, 17), (5000, 0, 64), (20011, 1, 57), (8191, 16, 48), (300, 40, 24)])
def test_tc_gram_matches_oracle(lib, n, k, nb):
    from paper_2402_15033_gb300 import capi
    if n < k + nb:
        pytest.skip("needs n >= k + nb")
    g = synth.rng(900 + n + k + nb)
    Q = bo.hhqr(g.standard_normal((n, k)))[0] if k else None
    V = g.standard_normal((n, nb)) / np.sqrt(n) + (Q @ g.standard_normal((k, nb)) / 4 if k else 0.0)
    Vg, Rg, st = run_pip_tc(capi, Q, V, ld_pad=n % 2)
    assert_parity(Q, V, Vg, Rg, st)


@pytest.mark.parametrize("n,k,nb", [(4099, 6, 5), (2000, 0, 61), (3001, 30, 16)])
def test_tc_gram_with_fp64_update(lib, n, k, nb):
    """The tensor-core Gram paired with the FP64 update: same bars."""
    from paper_2402_15033_gb300 import capi
    g = synth.rng(700 + n + k)
    Q = bo.hhqr(g.standard_normal((n, k)))[0] if k else None
    V = g.standard_normal((n, nb)) / np.sqrt(n) + (Q @ g.standard_normal((k, nb)) / 4 if k else 0.0)
    Vg, Rg, st = run_pip_tc(capi, Q, V, ld_pad=n % 2, tc_update=False)
    assert_parity(Q, V, Vg, Rg, st)


@pytest.mark.parametrize("scales", [(-40, 30), (25, -25), (-300, 0)])
def test_tc_update_equilibrates_column_scales(lib, scales):
    """V columns scaled by very different powers of two next to unit Q columns:
    the update slices V_j 2^(-g_j) against W rows scaled by 2^(g_j), so Q^
    keeps the FP64 parity bar (without equilibration the small entries of a
    row would lose their low digits)."""
    from paper_2402_15033_gb300 import capi
    g = synth.rng(808)
    n, k, nb = 30011, 12, 6
    Q = bo.hhqr(g.standard_normal((n, k)))[0]
    V = g.standard_normal((n, nb)) / np.sqrt(n) + Q @ g.standard_normal((k, nb)) / 3
    V[:, ::2] *= 2.0 ** scales[0]
    V[:, 1::2] *= 2.0 ** scales[1]
    Vg, Rg, st = run_pip_tc(capi, Q, V, ld_pad=1)
    assert_parity(Q, V, Vg, Rg, st)


def test_tc_wider_than_one_tile_uses_fp64(lib):
    """k + nb > 64 runs the FP64 kernel: same bars."""
    from paper_2402_15033_gb300 import capi
    g = synth.rng(31)
    n, k, nb = 4000, 70, 40
    Q = bo.hhqr(g.standard_normal((n, k)))[0]
    V = g.standard_normal((n, nb)) / np.sqrt(n)
    Vg, Rg, st = run_pip_tc(capi, Q, V)
    assert_parity(Q, V, Vg, Rg, st)


def _hard_digits(g, n, c):
    """Entries whose 8-bit digits take extreme and mixed values: +-(2 - 2^-52)
    scaled by random powers of two within +-3 binades, mixed signs, some
    exact zeros, and integers with long carry chains."""
    X = g.standard_normal((n, c))
    X[g.random((n, c)) < 0.3] = 2.0 - 2.0 ** -52
    X *= np.where(g.random((n, c)) < 0.5, -1.0, 1.0)
    X *= np.exp2(g.integers(-3, 4, size=(n, c)))
    X[g.random((n, c)) < 0.05] = 0.0
    X[g.random((n, c)) < 0.05] = 1.0 + 2.0 ** -52 * 0x7F7F7F
    return X


@pytest.mark.parametrize("n,k,nb", [(300, 6, 3), (257, 9, 5), (130, 2, 7)])
def test_tc_gram_entries_against_exact_rationals(lib, n, k, nb):
    """P = Q^T V (the first k rows of R) and G = T^T T + P^T P against X^T Y
    summed in exact rationals: every entry within 2^-48 ||x_i|| ||y_j||.  A
    tensor core that dropped low bits of an FP32 accumulation, a wrong digit
    weight or a lost carry would miss this by many orders of magnitude."""
    from paper_2402_15033_gb300 import capi
    g = synth.rng(4242 + n)
    Q = _hard_digits(g, n, k)
    # a power-of-two scale (digits unchanged) with ||Q||_2 <= 1/2 keeps
    # G - P^T P = V^T (I - Q Q^T) V positive definite, so T exists
    Q *= 2.0 ** -(np.ceil(np.log2(np.linalg.norm(Q))) + 1)
    V = _hard_digits(g, n, nb)
    _, Rg, st = run_pip_tc(capi, Q, V, ld_pad=n % 2, update=False)
    P_exact = checks.exact_gram(Q, V)
    nq = np.linalg.norm(Q, axis=0)
    nv = np.linalg.norm(V, axis=0)
    err = np.abs(Rg[:k] - P_exact) / np.outer(nq, nv)
    assert err.max() <= 2.0 ** -48, err.max()
    assert st == 0
    T = Rg[k:]
    G_exact = checks.exact_gram(V, V)
    G_rec = T.T @ T + Rg[:k].T @ Rg[:k]
    assert np.max(np.abs(G_rec - G_exact) / np.outer(nv, nv)) <= 1e-13


@pytest.mark.parametrize("scale_exp", [-400, -37, 29, 400])
def test_tc_power_of_two_scaling_is_exact(lib, scale_exp):
    """Scaling V by 2^e shifts the chunk exponents and nothing else: R scales
    by exactly 2^e bit for bit and Q^ is bit-identical (no FP32 range limit,
    unlike double-float)."""
    from paper_2402_15033_gb300 import capi
    g = synth.rng(55)
    n, k, nb = 20011, 7, 5
    Q = bo.hhqr(g.standard_normal((n, k)))[0]
    V = g.standard_normal((n, nb))
    V0, R0, s0 = run_pip_tc(capi, Q, V, ld_pad=1)
    V1, R1, s1 = run_pip_tc(capi, Q, V * 2.0 ** scale_exp, ld_pad=1)
    assert s0 == 0 and s1 == 0
    assert np.array_equal(R1, R0 * 2.0 ** scale_exp)
    assert np.array_equal(V1, V0)


def test_tc_breakdown_nan_and_repeatability(lib):
    from paper_2402_15033_gb300 import capi
    g = synth.rng(12)
    n = 500
    V = g.standard_normal((n, 5))
    V[:, 3] = 0.0
    Vg, _, st = run_pip_tc(capi, None, V)
    assert st == 4 and np.array_equal(Vg, V)
    V = g.standard_normal((300, 4))
    V[17, 2] = np.nan
    _, _, st = run_pip_tc(capi, None, V)
    assert st == 3
    n, k, nb = 100003, 20, 5
    Q = bo.hhqr(g.standard_normal((n, k)))[0]
    V = g.standard_normal((n, nb))
    a = run_pip_tc(capi, Q, V, ld_pad=1)
    b = run_pip_tc(capi, Q, V, ld_pad=1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_tc_unaligned_columns_run_fp64(lib):
    """An odd leading dimension leaves every other column off a 16-byte
    boundary: the call runs the FP64 kernels (bit-identical to
    ortho_gram_chol + ortho_update) instead of the 16-byte staged ones."""
    from paper_2402_15033_gb300 import capi
    g = synth.rng(13)
    n, k, nb = 10001, 10, 5      # V's base stays aligned (k even), its odd columns do not
    Q = bo.hhqr(g.standard_normal((n, k)))[0]
    V = g.standard_normal((n, nb))
    Vt, Rt, st = run_pip_tc(capi, Q, V, ld_pad=0)
    assert st == 0
    from test_gpu_ortho import run_pip
    Vf, Rf, sf = run_pip(capi, Q, V, stage=1, ld_pad=0)
    assert np.array_equal(Vt, Vf) and np.array_equal(Rt, Rf)


def test_tc_two_stage_on_ill_conditioned_panels(lib):
    """The glued matrix (panel kappa 1e5) through stage 1 per block and stage 2
    on the big panel with the tensor-core Gram: O(eps) orthogonality after
    stage 2 (Theorem 3) and the oracle's R at the kappa^2 eps level."""
    from paper_2402_15033_gb300 import capi
    n, s, nblk = 20000, 5, 6
    V = synth.glued(n, s, nblk, 1e5, seed=9)
    _, _, Rd, _ = bo.two_stage_panel(np.zeros((n, 0)), [V[:, i * s:(i + 1) * s] for i in range(nblk)])
    ncol = s * nblk
    B = torch.tensor(V.T.copy(), device="cuda").T
    Rh = torch.zeros(ncol, ncol, dtype=torch.float64, device="cuda").T
    work = torch.empty(capi.workspace_bytes(n, ncol, ncol), dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    for j in range(nblk):
        c0 = j * s
        Qd = B[:, :c0] if c0 else None
        capi.ortho_gram_chol_tc(Qd, B[:, c0:c0 + s], Rh[:c0 + s, c0:c0 + s], work, st, k=c0)
        capi.ortho_update(Qd, B[:, c0:c0 + s], Rh[:c0 + s, c0:c0 + s], st, k=c0, tc=True)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
    R2 = torch.zeros(ncol, ncol, dtype=torch.float64, device="cuda").T
    capi.ortho_gram_chol_tc(None, B, R2, work, st, k=0)
    capi.ortho_update(None, B, R2, st, k=0, tc=True)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Qg = B.cpu().numpy()
    assert checks.orth_error(Qg)[0] < 100 * np.finfo(float).eps
    Rfin = R2.cpu().numpy() @ Rh.cpu().numpy()
    assert np.allclose(Rfin, Rd, rtol=0, atol=1e-9 * np.abs(Rd).max())
    assert np.allclose(Qg @ Rfin, V, atol=1e-12 * np.abs(V).max())


# ---------------------------------------------------------------- digit basis
def _cols(n, c, ld_pad, g):
    """n x c column-major CUDA view with ld = n + ld_pad, N(0,1)/sqrt(n) entries."""
    buf = torch.zeros(c, n + ld_pad, dtype=torch.float64, device="cuda")
    buf[:, :n] = torch.tensor(g.standard_normal((c, n)) / np.sqrt(n))
    return buf.T[:n]


@pytest.mark.parametrize("n,k,nb", [(4099, 6, 5), (3001, 30, 16), (20000, 0, 61), (130, 56, 5), (64, 1, 5)])
def test_digit_basis_gram_is_bit_identical(lib, n, k, nb):
    """The Gram that reads Q's and V's digits from the digit basis equals the
    one that slices them, bit for bit (the digits are the same).  With only Q
    cached and nb <= 8 the streaming kernel runs instead: V's digits are taken
    against 16-row groups, so it agrees to rounding (2^-46 of the column norms);
    so does the tcgen05 kernel that takes every column from the basis when
    nb >= 9 and k + nb <= 64 (exact sums per CTA, rounded once)."""
    from paper_2402_15033_gb300 import capi
    g = synth.rng(1300 + n + k)
    pad = n % 2
    X = _cols(n, k + nb, pad, g)
    Q, V = (X[:, :k] if k else None), X[:, k:]
    capc = 64
    dig = torch.zeros(capi.digits_bytes(n, capc), dtype=torch.uint8, device="cuda")
    capi.digits_fill(X, 0, dig, capc)
    work = torch.empty(capi.workspace_bytes(n, k, nb), dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    outs = []
    for kc in (None, k, k + nb):
        R = torch.full((nb, k + nb), np.nan, dtype=torch.float64, device="cuda").T
        if kc is None:
            capi.ortho_gram_chol_tc(Q, V, R, work, st, k=k)
        else:
            capi.ortho_gram_chol_tcd(Q, V, R, work, st, dig, capc, kc, k=k)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        outs.append(R.cpu().numpy())
    scale = np.linalg.norm(outs[0], axis=0)
    if nb >= 9 and k + nb <= 64:
        assert np.all(np.abs(outs[2] - outs[0]) <= 2.0 ** -46 * scale[None, :])
    else:
        assert np.array_equal(outs[0], outs[2])
    if nb <= 8:
        scale = np.linalg.norm(outs[0], axis=0)
        assert np.all(np.abs(outs[1] - outs[0]) <= 2.0 ** -46 * scale[None, :])
    else:
        assert np.array_equal(outs[0], outs[1])


def run_gram_stream(capi, Q, V, ld_pad=0, update=True, capc=64, cached_v=False):
    """Gram through the streaming kernel (Q from the digit basis, nb <= 8) and
    the FP64 update.  cached_v: V's digits are in the basis too (every column
    cached, as for the stage-2 panel)."""
    n, nb = V.shape
    k = 0 if Q is None else Q.shape[1]
    buf = torch.zeros(k + nb, n + ld_pad, dtype=torch.float64, device="cuda")
    if k:
        buf[:k, :n] = torch.tensor(Q.T)
    buf[k:, :n] = torch.tensor(V.T)
    Qd = buf[:k].T[:n] if k else None
    Vd = buf[k:].T[:n]
    dig = torch.zeros(capi.digits_bytes(n, capc), dtype=torch.uint8, device="cuda")
    if cached_v:
        capi.digits_fill(buf.T[:n], 0, dig, capc)
    elif k:
        capi.digits_fill(Qd, 0, dig, capc)
    R = torch.full((nb, k + nb + 3), np.nan, dtype=torch.float64, device="cuda").T
    work = torch.empty(capi.workspace_bytes(n, k, nb), dtype=torch.uint8, device="cuda")
    st = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    capi.ortho_gram_chol_tcd(Qd, Vd, R, work, st, dig, capc, k + nb if cached_v else k, k=k)
    if update:
        capi.ortho_update(Qd, Vd, R, st, k=k)
    torch.cuda.synchronize()
    return Vd.cpu().numpy(), R[: k + nb].cpu().numpy(), int(st.item())


@pytest.mark.parametrize("n,k,nb", [(64, 0, 5), (65, 1, 1), (127, 6, 5), (4099, 15, 1), (4099, 16, 8),
                                    (4099, 17, 3), (20001, 31, 5), (20001, 32, 8), (3001, 47, 5), (3001, 48, 5),
                                    (100003, 56, 5), (777, 59, 5), (5000, 56, 8), (130, 2, 7), (300, 24, 8)])
def test_streaming_digit_gram_matches_oracle(lib, n, k, nb):
    """The narrow Gram that streams Q's digit units per warp (every M-tile
    layout: Q only, Q and V mixed, V only; ragged last chunks) meets the FP64
    parity bars against the oracle's BCGS-PIP."""
    from paper_2402_15033_gb300 import capi
    if n < k + nb:
        pytest.skip("needs n >= k + nb")
    g = synth.rng(2100 + n + k + nb)
    Q = bo.hhqr(g.standard_normal((n, k)))[0] if k else None
    V = g.standard_normal((n, nb)) / np.sqrt(n) + (Q @ g.standard_normal((k, nb)) / 4 if k else 0.0)
    Vg, Rg, st = run_gram_stream(capi, Q, V, ld_pad=n % 2)
    assert_parity(Q, V, Vg, Rg, st)


@pytest.mark.parametrize("n,k,nb", [(300, 6, 3), (257, 9, 5), (130, 2, 7), (1000, 40, 8)])
def test_streaming_digit_gram_against_exact_rationals(lib, n, k, nb):
    """P = Q^T V of the streaming kernel against exact rational sums on hard
    digits: every entry within 2^-48 ||q_i|| ||v_j||."""
    from paper_2402_15033_gb300 import capi
    g = synth.rng(4343 + n)
    Q = _hard_digits(g, n, k)
    Q *= 2.0 ** -(np.ceil(np.log2(np.linalg.norm(Q))) + 1)
    V = _hard_digits(g, n, nb)
    _, Rg, st = run_gram_stream(capi, Q, V, ld_pad=n % 2, update=False)
    P_exact = checks.exact_gram(Q, V)
    err = np.abs(Rg[:k] - P_exact) / np.outer(np.linalg.norm(Q, axis=0), np.linalg.norm(V, axis=0))
    assert err.max() <= 2.0 ** -48, err.max()
    assert st == 0
    T = Rg[k:]
    nv = np.linalg.norm(V, axis=0)
    G_rec = T.T @ T + Rg[:k].T @ Rg[:k]
    assert np.max(np.abs(G_rec - checks.exact_gram(V, V)) / np.outer(nv, nv)) <= 1e-13


@pytest.mark.parametrize("scale_exp", [-400, -37, 29, 400])
def test_streaming_digit_gram_power_of_two_scaling_is_exact(lib, scale_exp):
    from paper_2402_15033_gb300 import capi
    g = synth.rng(56)
    n, k, nb = 20011, 27, 5
    Q = bo.hhqr(g.standard_normal((n, k)))[0]
    V = g.standard_normal((n, nb))
    _, R0, s0 = run_gram_stream(capi, Q, V, ld_pad=1, update=False)
    _, R1, s1 = run_gram_stream(capi, Q, V * 2.0 ** scale_exp, ld_pad=1, update=False)
    assert s0 == 0 and s1 == 0
    assert np.array_equal(R1, R0 * 2.0 ** scale_exp)


def test_streaming_digit_gram_nan_zero_and_repeatability(lib):
    from paper_2402_15033_gb300 import capi
    g = synth.rng(57)
    n, k, nb = 30012, 20, 5
    Q = bo.hhqr(g.standard_normal((n, k)))[0]
    V = g.standard_normal((n, nb))
    a = run_gram_stream(capi, Q, V, update=False)
    b = run_gram_stream(capi, Q, V, update=False)
    assert a[2] == 0 and np.array_equal(a[1], b[1])
    Vz = V.copy()
    Vz[:, 3] = 0.0
    assert run_gram_stream(capi, Q, Vz, update=False)[2] == 4
    Vn = V.copy()
    Vn[29000, 2] = np.nan
    assert run_gram_stream(capi, Q, Vn, update=False)[2] == 3
    Qn = Q.copy()
    Qn[12345, 7] = np.inf    # row 7 of P is NaN, so is every entry of G - P^T P: the first pivot fails
    assert run_gram_stream(capi, Qn, V, update=False)[2] == 1


@pytest.mark.parametrize("n,k,nb", [(64, 0, 9), (65, 0, 16), (127, 3, 9), (4099, 0, 61), (4099, 15, 17),
                                    (20001, 16, 48), (3001, 40, 24), (100003, 0, 64), (777, 31, 33), (5000, 55, 9)])
def test_all_cached_digit_gram_matches_oracle(lib, n, k, nb):
    """The Gram over columns that are all in the digit basis (the stage-2
    panel; output tiles on and off the diagonal, ragged tile columns and last
    chunks) meets the FP64 parity bars against the oracle."""
    from paper_2402_15033_gb300 import capi
    g = synth.rng(2600 + n + k + nb)
    Q = bo.hhqr(g.standard_normal((n, k)))[0] if k else None
    V = g.standard_normal((n, nb)) / np.sqrt(n) + (Q @ g.standard_normal((k, nb)) / 4 if k else 0.0)
    Vg, Rg, st = run_gram_stream(capi, Q, V, ld_pad=n % 2, cached_v=True)
    assert_parity(Q, V, Vg, Rg, st)


def test_all_cached_digit_gram_zero_chunks_far_from_unit_scale(lib):
    """Columns that vanish over whole 64-row chunks, next to entries near 2^-300
    and 2^280: a zero chunk column carries the digit basis's zero marker, so it
    never sets the scale of the per-CTA exact sums (a zero chunk taken at
    exponent 0 would truncate every 2^-300 product); entries within 2^-48 of
    the exact rational sums."""
    from paper_2402_15033_gb300 import capi
    g = synth.rng(4412)
    n, k, nb = 8000, 3, 10
    Q = bo.hhqr(g.standard_normal((n, k)))[0]
    V = g.standard_normal((n, nb)) / np.sqrt(n) + Q @ g.standard_normal((k, nb)) / 4
    V[:640, 0::2] = 0.0
    V[64 * 50:64 * 60, 1] = 0.0
    V[:, 0::3] *= 2.0 ** -300
    V[:, 1::3] *= 2.0 ** 280
    _, Rg, st = run_gram_stream(capi, Q, V, ld_pad=0, update=False, cached_v=True)
    assert st == 0
    nq, nv = np.linalg.norm(Q, axis=0), np.linalg.norm(V, axis=0)
    err = np.abs(Rg[:k] - checks.exact_gram(Q, V)) / np.outer(nq, nv)
    assert err.max() <= 2.0 ** -48, err.max()
    G_rec = Rg[k:].T @ Rg[k:] + Rg[:k].T @ Rg[:k]
    assert np.max(np.abs(G_rec - checks.exact_gram(V, V)) / np.outer(nv, nv)) <= 1e-13


def test_all_cached_digit_gram_large_digit_sums(lib):
    """Rows whose digits 1..6 all equal -128 (x = -0x808080808080 2^-53 under a
    chunk maximum of 1, whose own digits are 32, 0, ..., 0): the weight-6 digit
    sum of that column with itself reaches 63 x 5 x 2^14 > 2^22, beyond the
    exact range of a single FP32-to-integer addition; the Gram still meets the
    1e-13 bar against exact rational sums."""
    from paper_2402_15033_gb300 import capi
    g = synth.rng(4413)
    n, nb = 2560, 10
    V = g.standard_normal((n, nb)) / np.sqrt(n)
    col = np.full(n, -float(0x808080808080) * 2.0 ** -53)
    col[::64] = 1.0
    V[:, 0] = col
    _, Rg, st = run_gram_stream(capi, None, V, ld_pad=0, update=False, cached_v=True)
    assert st == 0
    nv = np.linalg.norm(V, axis=0)
    G_rec = Rg.T @ Rg
    assert np.max(np.abs(G_rec - checks.exact_gram(V, V)) / np.outer(nv, nv)) <= 1e-13


def test_all_cached_digit_gram_exact_rationals_scaling_nan(lib):
    """Gram entries within 2^-48 of exact rational sums on hard digits; a
    power-of-two scale of V scales R exactly; a NaN in V fails its pivot; two
    runs agree bit for bit."""
    from paper_2402_15033_gb300 import capi
    g = synth.rng(4411)
    n, k, nb = 1000, 12, 20
    Q = _hard_digits(g, n, k)
    Q *= 2.0 ** -(np.ceil(np.log2(np.linalg.norm(Q))) + 1)
    V = _hard_digits(g, n, nb)
    _, Rg, st = run_gram_stream(capi, Q, V, ld_pad=0, update=False, cached_v=True)
    assert st == 0
    err = np.abs(Rg[:k] - checks.exact_gram(Q, V)) / np.outer(np.linalg.norm(Q, axis=0), np.linalg.norm(V, axis=0))
    assert err.max() <= 2.0 ** -48, err.max()
    nv = np.linalg.norm(V, axis=0)
    G_rec = Rg[k:].T @ Rg[k:] + Rg[:k].T @ Rg[:k]
    assert np.max(np.abs(G_rec - checks.exact_gram(V, V)) / np.outer(nv, nv)) <= 1e-13
    n, k, nb = 20011, 27, 17
    Qo = bo.hhqr(g.standard_normal((n, k)))[0]
    Vn = g.standard_normal((n, nb))
    _, R0, s0 = run_gram_stream(capi, Qo, Vn, ld_pad=1, update=False, cached_v=True)
    _, R1, s1 = run_gram_stream(capi, Qo, Vn * 2.0 ** -300, ld_pad=1, update=False, cached_v=True)
    _, R2, s2 = run_gram_stream(capi, Qo, Vn, ld_pad=1, update=False, cached_v=True)
    assert s0 == s1 == s2 == 0
    assert np.array_equal(R1, R0 * 2.0 ** -300) and np.array_equal(R2, R0)
    Vn[17000, 11] = np.nan
    assert run_gram_stream(capi, Qo, Vn, ld_pad=1, update=False, cached_v=True)[2] == 12


@pytest.mark.parametrize("n,k,nb", [(4099, 6, 5), (777, 20, 21), (20001, 56, 5), (1000, 0, 8), (131, 3, 1)])
def test_digit_basis_update_matches_oracle_and_writes_digits(lib, n, k, nb):
    """ortho_update_tcd (Q's digits read from the digit basis for nb <= 8) meets
    the FP64 parity bars against the oracle's BCGS-PIP, and the digits it writes
    for the new V equal those of ortho_digits_fill on the result."""
    from paper_2402_15033_gb300 import capi
    g = synth.rng(1400 + n + k)
    pad = n % 2
    Qh = bo.hhqr(g.standard_normal((n, k)))[0] if k else np.zeros((n, 0))
    Vh = g.standard_normal((n, nb)) / np.sqrt(n) + (Qh @ g.standard_normal((k, nb)) / 3 if k else 0.0)
    X = _cols(n, k + nb, pad, g)
    X[:, :k] = torch.tensor(Qh, device="cuda")
    X[:, k:] = torch.tensor(Vh, device="cuda")
    capc = 64
    dig = torch.zeros(capi.digits_bytes(n, capc), dtype=torch.uint8, device="cuda")
    if k:
        capi.digits_fill(X[:, :k], 0, dig, capc)
    work = torch.empty(capi.workspace_bytes(n, k, nb), dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    R = torch.zeros(nb, k + nb, dtype=torch.float64, device="cuda").T
    Qd = X[:, :k] if k else None
    capi.ortho_gram_chol_tcd(Qd, X[:, k:], R, work, st, dig, capc, k, k=k)
    capi.ortho_update_tcd(Qd, X[:, k:], R, st, dig, capc, k=k)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert_parity(Qh if k else None, Vh, X[:, k:].cpu().numpy(), R.cpu().numpy(), 0)
    ref = torch.zeros_like(dig)
    capi.digits_fill(X[:, k:], k, ref, capc)
    torch.cuda.synchronize()
    nch = (n + 63) // 64
    units = dig[: nch * capc * 448].view(nch, capc, 448)     # 7 digit bytes per value, 64 rows
    runits = ref[: nch * capc * 448].view(nch, capc, 448)
    assert torch.equal(units[:, k:k + nb], runits[:, k:k + nb])
    capx = (capc + 3) // 4 * 4      # a chunk's exponent row starts on a 16-byte boundary
    ex = dig[nch * capc * 448: nch * capc * 448 + nch * capx * 4].view(torch.int32).view(nch, capx)
    rex = ref[nch * capc * 448: nch * capc * 448 + nch * capx * 4].view(torch.int32).view(nch, capx)
    assert torch.equal(ex[:, k:k + nb], rex[:, k:k + nb])


@pytest.mark.parametrize("scales", [(-40, 30), (25, -25)])
def test_digit_basis_update_with_unbalanced_columns(lib, scales):
    """V columns scaled by very different powers of two: the per-chunk column
    exponents of the digit basis balance them (W'' = D W), so Q^ keeps the FP64
    parity bar."""
    from paper_2402_15033_gb300 import capi
    g = synth.rng(909)
    n, k, nb = 30011, 12, 6
    Qh = bo.hhqr(g.standard_normal((n, k)))[0]
    Vh = g.standard_normal((n, nb)) / np.sqrt(n) + Qh @ g.standard_normal((k, nb)) / 3
    Vh[:, ::2] *= 2.0 ** scales[0]
    Vh[:, 1::2] *= 2.0 ** scales[1]
    X = _cols(n, k + nb, 1, g)
    X[:, :k] = torch.tensor(Qh, device="cuda")
    X[:, k:] = torch.tensor(Vh, device="cuda")
    capc = 64
    dig = torch.zeros(capi.digits_bytes(n, capc), dtype=torch.uint8, device="cuda")
    capi.digits_fill(X[:, :k], 0, dig, capc)
    work = torch.empty(capi.workspace_bytes(n, k, nb), dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    R = torch.zeros(nb, k + nb, dtype=torch.float64, device="cuda").T
    capi.ortho_gram_chol_tcd(X[:, :k], X[:, k:], R, work, st, dig, capc, k, k=k)
    capi.ortho_update_tcd(X[:, :k], X[:, k:], R, st, dig, capc, k=k)
    torch.cuda.synchronize()
    assert_parity(Qh, Vh, X[:, k:].cpu().numpy(), R.cpu().numpy(), int(st.item()))


def test_digit_basis_two_stage_sequence_matches_oracle(lib):
    """The benchmark's sequence (column 0, blocks of 5 through stage 1, stage 2 on
    the panel) with the digit basis, against the oracle: R of every block and of
    stage 2, and the final Q, within the FP64 bars; O(eps) orthogonality."""
    from paper_2402_15033_gb300 import capi
    g = synth.rng(1500)
    n, s, nblk = 30001, 5, 6
    ncol = 1 + s * nblk
    B = _cols(n, ncol, 1, g)
    B[:, 0] /= torch.linalg.norm(B[:, 0])
    X = B.cpu().numpy().copy()
    capc = 64
    Rh = torch.zeros(ncol, ncol, dtype=torch.float64, device="cuda").T
    R2 = torch.zeros(ncol, ncol, dtype=torch.float64, device="cuda").T
    work = torch.empty(capi.workspace_bytes(n, ncol, ncol), dtype=torch.uint8, device="cuda")
    st = torch.zeros(nblk + 1, dtype=torch.int32, device="cuda")
    dig = torch.zeros(capi.digits_bytes(n, capc), dtype=torch.uint8, device="cuda")
    capi.digits_fill(B[:, :1], 0, dig, capc)
    for j in range(nblk):
        k = 1 + s * j
        Q, V, Rb = B[:, :k], B[:, k:k + s], Rh[:k + s, k:k + s]
        capi.ortho_gram_chol_tcd(Q, V, Rb, work, st[j:j + 1], dig, capc, k, k=k)
        capi.ortho_update_tcd(Q, V, Rb, st[j:j + 1], dig, capc, k=k)
    capi.ortho_gram_chol_tcd(None, B, R2, work, st[nblk:], dig, capc, ncol, k=0)
    capi.ortho_update(None, B, R2, st[nblk:], k=0, tc=True)
    torch.cuda.synchronize()
    assert int(st.abs().sum().item()) == 0
    Rh_ref = np.zeros((ncol, ncol))
    for j in range(nblk):
        k = 1 + s * j
        Qh, P, T = bo.stage1(X[:, :k], X[:, k:k + s])
        X[:, k:k + s] = Qh
        Rh_ref[:k, k:k + s] = P
        Rh_ref[k:k + s, k:k + s] = T
    Qf, _, T2 = bo.stage2(np.zeros((n, 0)), X)
    Rhg, R2g, Qg = Rh.cpu().numpy(), R2.cpu().numpy(), B.cpu().numpy()
    msk = np.triu(np.ones((ncol, ncol), bool), 1)
    msk[:, 0] = False
    scale = np.maximum(np.linalg.norm(Rh_ref, axis=0), 1e-300)
    assert np.all(np.abs(Rhg - Rh_ref)[msk] <= (1e-12 * scale[None, :].repeat(ncol, 0))[msk])
    sc = np.linalg.norm(T2, axis=0)
    assert np.all(np.abs(R2g - T2) <= 1e-12 * sc[None, :])
    assert np.max(np.abs(Qg - Qf)) <= 1e-12
    assert checks.orth_error(Qg)[0] < 100 * np.finfo(float).eps


@pytest.mark.slow
def test_full_size_digit_basis_sequence_sampled(lib):
    """The benchmark's headline sequence at its own size (n = 4,194,304 x 61:
    column 0 into the digit basis, 12 blocks of 5 through the digit-basis
    stage-1 Gram and update, k up to 56, then the all-cached stage-2 Gram and
    the tensor-core stage-2 update), launched as the benchmark launches it,
    against the oracle's stage 1 and stage 2 on the same input: every R entry
    within 1e-12 of its column's norm and 4096 sampled rows of Q within 1e-12."""
    from paper_2402_15033_gb300 import capi
    n, s, nblk = 4194304, 5, 12
    ncol = 1 + s * nblk
    B0 = synth.tall_basis(n, ncol, seed=1)
    buf = torch.tensor(B0.T.copy(), device="cuda")
    B = buf.T
    B[:, 0] /= torch.linalg.norm(B[:, 0])
    capc = 64
    Rh = torch.zeros(ncol, ncol, dtype=torch.float64, device="cuda").T
    R2 = torch.zeros(ncol, ncol, dtype=torch.float64, device="cuda").T
    work = torch.empty(capi.workspace_bytes(n, ncol, ncol), dtype=torch.uint8, device="cuda")
    st = torch.zeros(nblk + 1, dtype=torch.int32, device="cuda")
    dig = torch.empty(capi.digits_bytes(n, capc), dtype=torch.uint8, device="cuda")
    capi.digits_fill(B[:, :1], 0, dig, capc)
    for j in range(nblk):
        k = 1 + s * j
        Q, V, Rb = B[:, :k], B[:, k:k + s], Rh[:k + s, k:k + s]
        capi.ortho_gram_chol_tcd(Q, V, Rb, work, st[j:j + 1], dig, capc, k, k=k)
        capi.ortho_update_tcd(Q, V, Rb, st[j:j + 1], dig, capc, k=k)
    capi.ortho_gram_chol_tcd(None, B, R2, work, st[nblk:], dig, capc, ncol, k=0)
    capi.ortho_update(None, B, R2, st[nblk:], k=0, tc=True)
    torch.cuda.synchronize()
    assert int(st.abs().sum().item()) == 0
    del dig, work
    X = np.array(B0, copy=True)
    X[:, 0] /= np.linalg.norm(X[:, 0])
    Rh_ref = np.zeros((ncol, ncol))
    for j in range(nblk):
        k = 1 + s * j
        Qh, P, T = bo.stage1(X[:, :k], X[:, k:k + s])
        X[:, k:k + s] = Qh
        Rh_ref[:k, k:k + s] = P
        Rh_ref[k:k + s, k:k + s] = T
    Qf, _, T2 = bo.stage2(np.zeros((n, 0)), X)
    R2g, Rhg = R2.cpu().numpy(), Rh.cpu().numpy()
    sc = np.linalg.norm(T2, axis=0)
    assert np.all(np.abs(R2g - T2) <= 1e-12 * sc[None, :])
    msk = np.triu(np.ones((ncol, ncol), bool), 1)
    msk[:, 0] = False
    scale = np.maximum(np.linalg.norm(Rh_ref, axis=0), 1e-300)
    assert np.all(np.abs(Rhg - Rh_ref)[msk] <= (1e-12 * scale[None, :].repeat(ncol, 0))[msk])
    rows = synth.rng(3).choice(n, 4096, replace=False)
    Qs = B[torch.tensor(rows, device="cuda")].cpu().numpy()
    assert np.max(np.abs(Qs - Qf[rows])) <= 1e-12
