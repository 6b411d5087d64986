"""The C-ABI library builds, loads and exports every symbol include/gmres.h
declares; argument checks fail cleanly without launching anything (CPU only)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gmres.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|size_t|const\s+char\s*\*)\s+(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def capi():
    from paper_2402_15033_gb300 import build, capi as cap
    build.build()
    cap.load()
    return cap


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("gmres_create", "gmres_solve", "gmres_destroy", "ortho_stage1", "ortho_stage2",
              "ortho_workspace_bytes", "gmres_last_error", "gmres_default_opts", "gmres_mpk"):
        assert n in names


def test_library_exports_every_declared_symbol(capi):
    lib = capi.load()
    for name in declared_functions():
        assert name in capi.SIGNATURES, f"binding lacks {name}"
        assert getattr(lib, name) is not None


def test_struct_layouts_match_the_header(capi):
    assert C.sizeof(capi.gmres_opts) == 216
    assert C.sizeof(capi.gmres_result) == 216      # 6 int32, 8 doubles, theta[16]
    assert capi.gmres_result.sigma.offset == 80 and capi.gmres_result.theta.offset == 88
    assert capi.gmres_opts.tol.offset == 16
    assert capi.gmres_opts.theta.offset == 48
    assert capi.gmres_result.relres_implicit.offset == 24
    assert capi.gmres_opts.shift.offset == capi.gmres_opts.arith.offset + 4


def test_default_opts(capi):
    o = capi.default_opts()
    assert (o.m, o.s, o.panel, o.tol, o.ortho, o.precision, o.shift) == (60, 5, 60, 1e-8, 0, 0, 0)


def test_workspace_size_is_positive_and_monotone(capi):
    a = capi.workspace_bytes(4096, 1, 5)
    b = capi.workspace_bytes(4194304, 56, 5)
    c = capi.workspace_bytes(4194304, 0, 61)
    assert 0 < a <= b
    assert c > 0
    assert capi.workspace_bytes(0, 1, 5) == 0


def test_bad_arguments_are_rejected_before_any_launch(capi):
    lib = capi.load()
    st = C.c_void_p(16)  # never dereferenced: validation fails first
    # nb = 0
    rc = lib.ortho_stage1(None, 100, None, 100, 0, C.c_void_p(256), 100, 0, C.c_void_p(256), 1,
                          C.c_void_p(256), 1 << 20, st)
    assert rc == capi.GMRES_ERR_ARG and "nb" in capi.last_error()
    # misaligned V
    rc = lib.ortho_stage1(None, 100, None, 100, 0, C.c_void_p(8), 100, 5, C.c_void_p(256), 5,
                          C.c_void_p(256), 1 << 20, st)
    assert rc == capi.GMRES_ERR_ARG and "aligned" in capi.last_error()
    # size limits: nb <= 64, k + nb <= 256 (dummy pointers, never read)
    for k, nb in ((0, 65), (192, 65), (200, 57), (256, 1)):
        rc = lib.ortho_stage2(None, 1000, C.c_void_p(256), 1000, k, C.c_void_p(256), 1000, nb, C.c_void_p(256),
                              k + nb, C.c_void_p(256), 1 << 30, st)
        assert rc == capi.GMRES_ERR_ARG and "k + nb <= 256" in capi.last_error(), (k, nb)
    # too small workspace
    rc = lib.ortho_stage2(None, 100, None, 100, 0, C.c_void_p(256), 100, 5, C.c_void_p(256), 5,
                          C.c_void_p(256), 8, st)
    assert rc == capi.GMRES_ERR_WORKSPACE
    # bad options at create
    o = capi.default_opts(panel=7)
    h = C.c_void_p()
    import numpy as np
    rp = np.array([0, 1], dtype=np.int64)
    ci = np.array([0], dtype=np.int32)
    vv = np.array([1.0])
    rc = lib.gmres_create(C.byref(h), 1, 1, rp.ctypes.data_as(C.c_void_p), ci.ctypes.data_as(C.c_void_p),
                          vv.ctypes.data_as(C.c_void_p), 0, C.byref(o), None)
    assert rc == capi.GMRES_ERR_ARG and "panel" in capi.last_error()
    # shifted CholQR: a known shift, FP64 basis, not the five-reduction scheme
    for bad in (dict(shift=2), dict(shift=1, precision=capi.GMRES_PREC_MIXED),
                dict(shift=1, ortho=capi.GMRES_ORTHO_BCGS2_CHOLQR2, panel=5)):
        o = capi.default_opts(**bad)
        rc = lib.gmres_create(C.byref(h), 1, 1, rp.ctypes.data_as(C.c_void_p), ci.ctypes.data_as(C.c_void_p),
                              vv.ctypes.data_as(C.c_void_p), 0, C.byref(o), None)
        assert rc == capi.GMRES_ERR_ARG and "shift" in capi.last_error(), bad
    assert lib.gmres_destroy(None) == capi.GMRES_OK


def test_digit_basis_size_formula(capi):
    """ortho_digits_bytes (host code): per 64-row chunk, capc columns of 448
    digit bytes (seven per row), then each chunk's row of int32 exponents padded
    to a multiple of four columns (16-byte aligned rows), plus 256 bytes."""
    for n, capc in [(1, 1), (64, 5), (65, 61), (4194304, 64), (1000, 63), (129, 62)]:
        chunks = (n + 63) // 64
        expect = chunks * capc * 64 * 7 + chunks * ((capc + 3) // 4 * 4) * 4 + 256
        assert capi.digits_bytes(n, capc) == expect, (n, capc)


def test_footprint_covers_the_resident_state(capi):
    """gmres_footprint (host code; the serving loop admits requests by it): at
    least the basis (m+1) x n in the basis precision plus the CSR, as the
    admission rule states; the tensor-core arithmetic adds the digit basis
    (7 bytes per basis entry); monotone in n and nnz; 0 for invalid input."""
    n, nnz = 1 << 20, 5 << 20
    ldq = (n + 31) // 32 * 32
    csr = (n + 1) * 4 + nnz * 4 + nnz * 8
    f64 = capi.footprint(n, nnz, capi.default_opts(m=60, s=5, panel=60))
    mix = capi.footprint(n, nnz, capi.default_opts(m=60, s=5, panel=60, precision=capi.GMRES_PREC_MIXED))
    tc = capi.footprint(n, nnz, capi.default_opts(m=60, s=5, panel=60, arith=capi.GMRES_ARITH_TC))
    assert f64 >= 61 * ldq * 8 + csr
    assert mix >= 61 * ldq * 4 + csr + nnz * 4     # FP32 basis, plus the FP32 copy of the values
    assert mix < f64 - 61 * ldq * 3                 # the basis takes half the bytes
    assert tc - f64 >= 61 * n * 7                   # seven digit bytes per entry
    assert tc - f64 < 61 * n * 8                    # and no more than the FP64 basis itself
    assert f64 - csr < 61 * ldq * 8 * 1.25          # and not much else
    assert capi.footprint(2 * n, nnz, capi.default_opts(m=60, s=5, panel=60)) > f64
    assert capi.footprint(n, 2 * nnz, capi.default_opts(m=60, s=5, panel=60)) > f64
    assert capi.footprint(0, nnz, capi.default_opts()) == 0
    assert capi.footprint(n, nnz, capi.default_opts(m=60, s=7, panel=60)) == 0


def test_batch_footprint_covers_the_resident_state(capi):
    """gmres_batch_footprint (host code): at least every system's basis rows
    (padded to 32) x (m+1) in the basis precision plus the concatenated CSR;
    0 for options a batch rejects and for empty systems."""
    import ctypes as C2
    ns = [1000, 4097, 250001]
    nz = [5 * v for v in ns]
    N = (C2.c_int64 * 3)(*ns)
    Z = (C2.c_int64 * 3)(*nz)
    lib = capi.load()
    rows = sum((v + 31) // 32 * 32 for v in ns)
    csr = (rows + 3) * 4 + sum(nz) * 12
    f64 = lib.gmres_batch_footprint(3, N, Z, C2.byref(capi.default_opts(m=40, s=5, panel=40)))
    mix = lib.gmres_batch_footprint(3, N, Z, C2.byref(capi.default_opts(m=40, s=5, panel=40,
                                                                          precision=capi.GMRES_PREC_MIXED)))
    assert f64 >= rows * 41 * 8 + csr
    assert mix >= rows * 41 * 4 + csr + sum(nz) * 4
    assert mix < f64
    for bad in (dict(m=40, s=5, panel=15), dict(m=64, s=8, panel=64), dict(arith=capi.GMRES_ARITH_TC),
                dict(ortho=2), dict(basis=capi.GMRES_BASIS_NEWTON_AUTO)):
        o = capi.default_opts(**{**dict(m=40, s=5, panel=40), **bad})
        assert lib.gmres_batch_footprint(3, N, Z, C2.byref(o)) == 0, bad
    N0 = (C2.c_int64 * 3)(1000, 0, 5)
    assert lib.gmres_batch_footprint(3, N0, Z, C2.byref(capi.default_opts(m=40, s=5, panel=40))) == 0


def test_binding_rejects_bad_host_vectors(capi):
    """The binding checks solver vectors before their pointers reach the
    library: float64, contiguous, the system's length, x writable."""
    import numpy as np
    ok = np.zeros(10)
    p, dev = capi._vec(ok, 10, "b")
    assert dev is False and p.value == ok.ctypes.data
    for bad in (np.zeros(9), np.zeros(10, dtype=np.float32), np.zeros(20)[::2], [0.0] * 10):
        with pytest.raises(ValueError):
            capi._vec(bad, 10, "b")
    ro = np.zeros(10)
    ro.flags.writeable = False
    capi._vec(ro, 10, "b")
    with pytest.raises(ValueError):
        capi._vec(ro, 10, "x", writable=True)
