"""gmres_newton_shifts (host code in the library, no device work) against the
oracle's newton_shifts / newton_sigma and against closed forms: the Ritz
values' real parts in Leja order and the capacity scale that
GMRES_BASIS_NEWTON_AUTO takes after its first cycle.  CPU only."""
import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import krylov as kr


@pytest.fixture(scope="module")
def capi():
    from paper_2402_15033_gb300 import build, capi as cap
    build.build()
    cap.load()
    return cap


def similar_hessenberg(d, seed):
    """Upper Hessenberg matrix orthogonally similar to diag(d) (scipy's
    Householder reduction), so its eigenvalues are d."""
    g = synth.rng(seed)
    k = len(d)
    Q, _ = np.linalg.qr(g.standard_normal((k, k)))
    return sla.hessenberg(Q @ np.diag(d) @ Q.T)


@pytest.mark.parametrize("k,s", [(1, 1), (2, 2), (3, 5), (7, 7), (20, 10), (60, 16), (63, 5)])
def test_real_spectrum_matches_the_oracle(capi, k, s):
    g = synth.rng(100 + k)
    d = np.sort(g.uniform(0.05, 8.0, k))
    d[0] = 0.05          # distinct, well separated products
    H = similar_hessenberg(d, k)
    th, sg = capi.newton_shifts(H, s, sigma=8.0)
    ref = kr.newton_shifts(H, s)
    assert np.allclose(th, ref, rtol=0, atol=1e-10 * d.max())
    assert np.allclose(th, kr.leja_order(d)[[i % k for i in range(s)]], atol=1e-9 * d.max())
    assert sg == kr.newton_sigma(ref, 8.0)


def test_nonsymmetric_hessenberg_gives_real_parts_in_leja_order(capi):
    """A nonsymmetric Hessenberg matrix with complex pairs: every shift is the
    real part of an eigenvalue (numpy/LAPACK), the first two shifts (largest
    modulus, then farthest) equal the oracle's, and the whole sequence is a
    valid Leja order of the computed real parts (each pick maximizes the
    distance product among the points left, to rounding)."""
    g = synth.rng(7)
    k = 30
    H = np.triu(g.standard_normal((k, k)), -1)
    ev = np.linalg.eigvals(H)
    assert np.count_nonzero(np.abs(ev.imag) > 1e-8) >= 4
    th, _ = capi.newton_shifts(H, 16)
    ref = kr.newton_shifts(H, 16)
    for t in th:
        assert np.min(np.abs(ev.real - t)) <= 1e-10 * np.abs(ev).max()
    assert np.allclose(th[:2], ref[:2], atol=1e-10 * np.abs(ev).max())
    pts = list(np.sort(ev.real))
    taken = []
    for t in th:
        j = int(np.argmin(np.abs(np.array(pts) - t)))
        if taken:
            prods = [np.prod([abs(p - q) for q in taken]) for p in pts]
            assert np.prod([abs(pts[j] - q) for q in taken]) >= max(prods) * (1 - 1e-8) - 1e-12
        taken.append(pts.pop(j))


def test_closed_forms(capi):
    # rotation generator: eigenvalues +-i, real parts 0 and 0; no interval
    th, sg = capi.newton_shifts([[0.0, -1.0], [1.0, 0.0]], 3, sigma=4.0)
    assert th.tolist() == [0.0, 0.0, 0.0] and sg == 4.0
    # already triangular: the diagonal, Leja order from the largest modulus
    H = np.array([[3.0, 1.0, 2.0], [0.0, -5.0, 1.0], [0.0, 0.0, 1.0]])
    th, sg = capi.newton_shifts(H, 3, sigma=1.0)
    assert th.tolist() == [-5.0, 3.0, 1.0]
    assert sg == 2.0          # capacity (3 + 5) / 4 = 2
    # 2 x 2 with a real pair: eigenvalues of [[a, b], [c, d]] by the quadratic formula
    a, b, c, d = 1.0, 2.0, 3.0, 4.0
    mid, rad = (a + d) / 2, np.sqrt(((a - d) / 2) ** 2 + b * c)
    th, _ = capi.newton_shifts([[a, b], [c, d]], 2)
    assert np.allclose(th, [mid + rad, mid - rad], rtol=1e-15)
    # k = 0: zero shifts
    th, sg = capi.newton_shifts(np.zeros((0, 0)), 4, sigma=8.0)
    assert th.tolist() == [0.0] * 4 and sg == 8.0


def test_scale_free_at_extreme_magnitudes(capi):
    d = np.array([0.5, 1.0, 2.0, 3.5, 7.0])
    H = similar_hessenberg(d, 3)
    base, _ = capi.newton_shifts(H, 5)
    for e in (-600, 600):
        th, sg = capi.newton_shifts(H * 2.0 ** e, 5, sigma=1.0)
        assert np.allclose(th, base * 2.0 ** e, rtol=1e-12, atol=0)
        assert sg == kr.newton_sigma(base * 2.0 ** e, 1.0)


def test_bad_arguments_fail_cleanly(capi):
    lib = capi.load()
    H = np.eye(4)
    with pytest.raises(capi.GmresError) as e:
        capi.newton_shifts(H, 17)
    assert e.value.code == capi.GMRES_ERR_ARG
    with pytest.raises(capi.GmresError) as e:
        capi.newton_shifts(H, 0)
    assert e.value.code == capi.GMRES_ERR_ARG
    th = (capi.C.c_double * 4)()
    assert lib.gmres_newton_shifts(None, 4, 4, 4, th, None) == capi.GMRES_ERR_ARG
    assert lib.gmres_newton_shifts(H.ctypes.data, 3, 4, 4, th, None) == capi.GMRES_ERR_ARG
    Hn = H.copy()
    Hn[1, 0] = np.nan
    with pytest.raises(capi.GmresError) as e:
        capi.newton_shifts(Hn, 4)
    assert e.value.code == capi.GMRES_ERR_EIG
