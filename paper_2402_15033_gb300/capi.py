"""Thin ctypes binding of ``libgmres.so`` (the C ABI in ``include/gmres.h``).

Argument marshalling only: every step of the solver and of the block
orthogonalization runs in the library's CUDA kernels.  Device buffers are
passed as raw pointers (``tensor.data_ptr()``); PyTorch is used by callers only
to own device memory and streams.  ``load()`` raises if the library is missing
or was built without a symbol the header declares; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgmres.so")

GMRES_OK = 0
GMRES_WARN_MAXIT = 1
GMRES_ERR_ARG = -1
GMRES_ERR_CUDA = -2
GMRES_ERR_OOM = -3
GMRES_ERR_BREAKDOWN = -4
GMRES_ERR_NAN = -5
GMRES_ERR_TIMEOUT = -6
GMRES_ERR_WORKSPACE = -7
GMRES_ERR_EIG = -8

GMRES_ORTHO_TWO_STAGE = 0
GMRES_ORTHO_BCGS_PIP2 = 1
GMRES_ORTHO_BCGS2_CHOLQR2 = 2
GMRES_PREC_FP64 = 0
GMRES_PREC_MIXED = 1
GMRES_BASIS_MONOMIAL = 0
GMRES_BASIS_NEWTON = 1
GMRES_BASIS_NEWTON_AUTO = 2
GMRES_BASIS_CHEBYSHEV = 3
GMRES_BASIS_CHEBYSHEV_AUTO = 4
GMRES_ARITH_FP64 = 0
GMRES_ARITH_DD = 1
GMRES_ARITH_TC = 2
GMRES_SHIFT_NONE = 0
GMRES_SHIFT_CHOLQR3 = 1
GMRES_PRECOND_NONE = 0
GMRES_PRECOND_MCGS = 1


class gmres_opts(C.Structure):
    _fields_ = [("m", C.c_int32), ("s", C.c_int32), ("panel", C.c_int32), ("max_restarts", C.c_int32),
                ("tol", C.c_double), ("sigma", C.c_double),
                ("ortho", C.c_int32), ("precision", C.c_int32), ("basis", C.c_int32), ("timing", C.c_int32),
                ("theta", C.c_double * 16), ("inner_tol", C.c_double), ("max_ir", C.c_int32),
                ("arith", C.c_int32), ("shift", C.c_int32), ("precond", C.c_int32), ("reserved", C.c_int32 * 4)]


class gmres_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("rejected", C.c_int64), ("failed", C.c_int64), ("active", C.c_int64), ("pending", C.c_int64),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double),
                ("solves_per_s", C.c_double), ("busy_s", C.c_double),
                ("mem_budget", C.c_size_t), ("mem_in_use", C.c_size_t)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class gmres_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("restarts", C.c_int32), ("ir_steps", C.c_int32),
                ("breakdown_block", C.c_int32), ("breakdown_pivot", C.c_int32),
                ("relres_implicit", C.c_double), ("relres_true", C.c_double),
                ("t_mpk_ms", C.c_double), ("t_stage1_ms", C.c_double), ("t_stage2_ms", C.c_double),
                ("t_ls_ms", C.c_double), ("t_total_ms", C.c_double),
                ("sigma", C.c_double), ("theta", C.c_double * 16)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["theta"] = list(self.theta)
        return d


_vp, _i32, _i64, _sz, _dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t, C.c_double

# name -> (restype, argtypes); every symbol the header declares
SIGNATURES = {
    "gmres_default_opts": (_i32, [C.POINTER(gmres_opts)]),
    "gmres_create": (_i32, [C.POINTER(_vp), _i64, _i64, _vp, _vp, _vp, _i32, C.POINTER(gmres_opts), _vp]),
    "gmres_solve": (_i32, [_vp, _vp, _vp, _i32, C.POINTER(gmres_result)]),
    "gmres_destroy": (_i32, [_vp]),
    "gmres_last_error": (C.c_char_p, []),
    "ortho_workspace_bytes": (_sz, [_i64, _i32, _i32]),
    "ortho_stage1": (_i32, [_vp, _i64, _vp, _i64, _i32, _vp, _i64, _i32, _vp, _i32, _vp, _sz, _vp]),
    "ortho_stage1_shifted": (_i32, [_vp, _i64, _vp, _i64, _i32, _vp, _i64, _i32, _vp, _i32, _vp, _sz, _vp]),
    "gmres_precond_apply": (_i32, [_vp, _vp, _vp]),
    "ortho_plan_create": (_i32, [_vp, _i64, _i32, _i32, _i32, _vp]),
    "ortho_plan_run": (_i32, [_vp, _vp, _i64, _vp, _i64, _vp, _vp, _i32, _i32, _vp]),
    "ortho_plan_destroy": (_i32, [_vp]),
    "ortho_stage2": (_i32, [_vp, _i64, _vp, _i64, _i32, _vp, _i64, _i32, _vp, _i32, _vp, _sz, _vp]),
    "gmres_mpk": (_i32, [_vp, _vp, _vp, _i64, _i32, _dbl, C.POINTER(_dbl)]),
    "ortho_gram_chol": (_i32, [_vp, _i64, _vp, _i64, _i32, _vp, _i64, _i32, _vp, _i32, _vp, _sz, _vp]),
    "ortho_update": (_i32, [_vp, _i64, _vp, _i64, _i32, _vp, _i64, _i32, _vp, _i32, _vp]),
    "ortho_gram_chol_dd": (_i32, [_vp, _i64, _vp, _i64, _i32, _vp, _i64, _i32, _vp, _i32, _vp, _sz, _vp]),
    "ortho_gram_chol_tc": (_i32, [_vp, _i64, _vp, _i64, _i32, _vp, _i64, _i32, _vp, _i32, _vp, _sz, _vp]),
    "ortho_update_tc": (_i32, [_vp, _i64, _vp, _i64, _i32, _vp, _i64, _i32, _vp, _i32, _vp]),
    "ortho_digits_bytes": (_sz, [_i64, _i32]),
    "ortho_digits_fill": (_i32, [_vp, _i64, _vp, _i64, _i32, _i32, _vp, _i32]),
    "ortho_gram_chol_tcd": (_i32, [_vp, _i64, _vp, _i64, _i32, _vp, _i64, _i32, _vp, _i32, _vp, _sz, _vp,
                                   _vp, _i32, _i32]),
    "ortho_update_tcd": (_i32, [_vp, _i64, _vp, _i64, _i32, _vp, _i64, _i32, _vp, _i32, _vp, _vp, _i32]),
    "ortho_update_dd": (_i32, [_vp, _i64, _vp, _i64, _i32, _vp, _i64, _i32, _vp, _i32, _vp]),
    "ortho_stage1_f32": (_i32, [_vp, _i64, _vp, _i64, _i32, _vp, _i64, _i32, _vp, _i32, _vp, _sz, _vp]),
    "ortho_stage2_f32": (_i32, [_vp, _i64, _vp, _i64, _i32, _vp, _i64, _i32, _vp, _i32, _vp, _sz, _vp]),
    "gmres_batch_footprint": (_sz, [_i32, _vp, _vp, C.POINTER(gmres_opts)]),
    "gmres_batch_create": (_i32, [C.POINTER(_vp), _i32, _vp, _vp, _vp, _vp, C.POINTER(gmres_opts), _vp]),
    "gmres_batch_solve": (_i32, [_vp, _vp, _vp, _vp]),
    "gmres_batch_autotune": (_i32, [_vp, C.POINTER(_dbl)]),
    "gmres_batch_destroy": (_i32, [_vp]),
    "gmres_footprint": (_sz, [_i64, _i64, C.POINTER(gmres_opts)]),
    "gmres_server_start": (_i32, [C.POINTER(_vp), _sz, _i32]),
    "gmres_server_submit": (_i32, [_vp, _i64, _vp, _vp, _vp, _vp, _vp, C.POINTER(gmres_opts), C.POINTER(_i64)]),
    "gmres_server_wait": (_i32, [_vp, _i64, _vp, C.POINTER(gmres_result), _dbl]),
    "gmres_server_poll": (_i32, [_vp, _i64, _vp, C.POINTER(gmres_result)]),
    "gmres_server_get_stats": (_i32, [_vp, C.POINTER(gmres_server_stats)]),
    "gmres_server_stop": (_i32, [_vp]),
    "gmres_newton_shifts": (_i32, [_vp, _i32, _i32, _i32, C.POINTER(_dbl), C.POINTER(_dbl)]),
    "ortho_stage1_noalloc": (_i32, [_vp, _i64, _vp, _i64, _i32, _vp, _i64, _i32, _vp, _i32, _vp]),
}

_lib = None


class GmresError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libgmres error {code}: {msg}")
        self.code = code


def load(path: str = LIB_PATH):
    """Load the library once and declare every signature.  Raises if the shared
    object is missing (build it with ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first (python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def last_error() -> str:
    return load().gmres_last_error().decode()


def check(rc: int, allow=(GMRES_OK,)) -> int:
    if rc not in allow:
        raise GmresError(rc, last_error())
    return rc


def default_opts(**kw) -> gmres_opts:
    o = gmres_opts()
    check(load().gmres_default_opts(C.byref(o)))
    for k, v in kw.items():
        if k == "theta":
            for i, t in enumerate(v):
                o.theta[i] = t
        else:
            setattr(o, k, v)
    return o


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _vec(a, n, name, writable=False):
    """Checks a solver vector before its pointer goes to the library: a
    contiguous float64 numpy array (host) or CUDA tensor (device) of n entries.
    Returns (pointer, on_device)."""
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float64 or not a.is_cuda or not a.is_contiguous() or a.numel() != n:
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor of {n} entries")
        return C.c_void_p(a.data_ptr()), True
    import numpy as np
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous or a.size != n:
        raise ValueError(f"{name} must be a contiguous float64 numpy array of {n} entries")
    if writable and not a.flags.writeable:
        raise ValueError(f"{name} must be writable")
    return a.ctypes.data_as(C.c_void_p), False


class Solver:
    """gmres_create / gmres_solve / gmres_destroy around one CSR matrix.

    ``rowptr`` (int64), ``colind`` (int32) and ``vals`` (float64) are numpy
    arrays (host) or torch CUDA tensors (device)."""

    def __init__(self, n, rowptr, colind, vals, opts: gmres_opts | None = None, stream=None):
        lib = load()
        on_dev = hasattr(rowptr, "data_ptr")
        if on_dev:
            ptrs = [C.c_void_p(a.data_ptr()) for a in (rowptr, colind, vals)]
        else:
            ptrs = [a.ctypes.data_as(C.c_void_p) for a in (rowptr, colind, vals)]
            self._keep = (rowptr, colind, vals)
        o = opts if opts is not None else default_opts()
        h = C.c_void_p()
        nnz = int(rowptr[-1])
        check(lib.gmres_create(C.byref(h), int(n), nnz, *ptrs, int(on_dev), C.byref(o), C.c_void_p(stream or 0)))
        self.h = h
        self.n = int(n)
        self.opts = o

    @classmethod
    def from_csr(cls, A, opts=None, stream=None):
        return cls(A.n, A.rowptr, A.colind, A.vals, opts, stream)

    def solve(self, b, x):
        """b, x: numpy float64 arrays (host) or torch float64 CUDA tensors.
        x holds x0 and receives the solution.  Returns (status, result dict)."""
        lib = load()
        res = gmres_result()
        bp, b_dev = _vec(b, self.n, "b")
        xp, x_dev = _vec(x, self.n, "x", writable=True)
        if b_dev != x_dev:
            raise ValueError("b and x must both be on the host or both on the device")
        rc = lib.gmres_solve(self.h, bp, xp, int(b_dev), C.byref(res))
        out = res.as_dict()
        out["error"] = last_error() if rc < 0 else ""
        return rc, out

    def precond_apply(self, r, z):
        """z = M^{-1} r (device tensors of n FP64 values) for the context's preconditioner."""
        return check(load().gmres_precond_apply(self.h, _ptr(r), _ptr(z)))

    def mpk(self, v, W, s, sigma, theta=None):
        lib = load()
        th = (C.c_double * s)(*theta) if theta is not None else None
        check(lib.gmres_mpk(self.h, _ptr(v), _ptr(W), W.stride(1), int(s), float(sigma), th))

    def close(self):
        if getattr(self, "h", None):
            load().gmres_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr_array(arrs):
    return (C.c_void_p * len(arrs))(*[a.ctypes.data_as(C.c_void_p) for a in arrs])


class Batch:
    """gmres_batch_create / _solve / _autotune / _destroy over a list of CSR
    matrices (objects with n, rowptr, colind, vals as numpy arrays)."""

    def __init__(self, mats, opts: gmres_opts | None = None, stream=None):
        lib = load()
        self.mats = list(mats)
        self.n = [int(A.n) for A in self.mats]
        ns = len(self.mats)
        nn = (C.c_int64 * ns)(*self.n)
        o = opts if opts is not None else default_opts()
        h = C.c_void_p()
        check(lib.gmres_batch_create(C.byref(h), ns, nn, _ptr_array([A.rowptr for A in self.mats]),
                                     _ptr_array([A.colind for A in self.mats]), _ptr_array([A.vals for A in self.mats]),
                                     C.byref(o), C.c_void_p(stream or 0)))
        self.h = h
        self.opts = o

    @staticmethod
    def footprint(mats, opts=None) -> int:
        ns = len(mats)
        nn = (C.c_int64 * ns)(*[int(A.n) for A in mats])
        nz = (C.c_int64 * ns)(*[int(A.rowptr[-1]) for A in mats])
        o = opts if opts is not None else default_opts()
        return int(load().gmres_batch_footprint(ns, nn, nz, C.byref(o)))

    def solve(self, bs, xs):
        """bs, xs: lists of float64 numpy arrays (x holds x0, receives x).
        Returns (worst status, list of result dicts)."""
        ns = len(self.mats)
        if len(bs) != ns or len(xs) != ns:
            raise ValueError(f"need {ns} right-hand sides and {ns} solution vectors")
        for i, (b, x) in enumerate(zip(bs, xs)):
            if _vec(b, self.n[i], f"b[{i}]")[1] or _vec(x, self.n[i], f"x[{i}]", writable=True)[1]:
                raise ValueError("batch vectors are host numpy arrays")
        res = (gmres_result * ns)()
        rc = load().gmres_batch_solve(self.h, _ptr_array(bs), _ptr_array(xs), res)
        if rc in (GMRES_ERR_ARG, GMRES_ERR_CUDA, GMRES_ERR_OOM):
            raise GmresError(rc, last_error())
        return rc, [r.as_dict() for r in res]

    def autotune(self):
        out = (C.c_double * 4)()
        check(load().gmres_batch_autotune(self.h, out))
        return {"gram_ms": out[0], "update_ms": out[1], "gram_grid": int(out[2]), "row_grid": int(out[3])}

    def close(self):
        if getattr(self, "h", None):
            load().gmres_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def footprint(n, nnz, opts=None) -> int:
    o = opts if opts is not None else default_opts()
    return int(load().gmres_footprint(int(n), int(nnz), C.byref(o)))


class Server:
    """gmres_server_start / submit / wait / stats / stop."""

    def __init__(self, mem_budget=0, max_active=16):
        h = C.c_void_p()
        check(load().gmres_server_start(C.byref(h), int(mem_budget), int(max_active)))
        self.h = h
        self._n = {}

    def submit(self, A, b, x0=None, opts=None):
        rid = C.c_int64()
        o = opts if opts is not None else default_opts()
        for v, name in ((b, "b"), (x0, "x0")):
            if v is not None and _vec(v, int(A.n), name)[1]:
                raise ValueError(f"{name} must be a host numpy array")
        check(load().gmres_server_submit(self.h, int(A.n), A.rowptr.ctypes.data_as(C.c_void_p),
                                         A.colind.ctypes.data_as(C.c_void_p), A.vals.ctypes.data_as(C.c_void_p),
                                         b.ctypes.data_as(C.c_void_p),
                                         None if x0 is None else x0.ctypes.data_as(C.c_void_p), C.byref(o),
                                         C.byref(rid)))
        self._n[rid.value] = int(A.n)
        return rid.value

    def wait(self, rid, timeout=-1.0):
        """Returns (x, result dict) once finished, or None on timeout."""
        n = self._n[rid]
        x = __import__("numpy").zeros(n)
        res = gmres_result()
        got = load().gmres_server_wait(self.h, int(rid), x.ctypes.data_as(C.c_void_p), C.byref(res), float(timeout))
        if got < 0:
            raise GmresError(got, last_error())
        if got == 0:
            return None
        del self._n[rid]
        return x, res.as_dict()

    def stats(self):
        st = gmres_server_stats()
        check(load().gmres_server_get_stats(self.h, C.byref(st)))
        return st.as_dict()

    def stop(self):
        if getattr(self, "h", None):
            load().gmres_server_stop(self.h)
            self.h = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


def workspace_bytes(n, k, nb) -> int:
    return int(load().ortho_workspace_bytes(int(n), int(k), int(nb)))


def _ortho(fn, Q, V, R, work, status, k, stream):
    """Q: (>=n, >=k) column-major view or None; V: column-major (ld, nb) view."""
    n = V.shape[0]
    nb = V.shape[1]
    ldv = V.stride(1)
    ldq = Q.stride(1) if (Q is not None and k > 0) else n
    qp = C.c_void_p(Q.data_ptr()) if (Q is not None and k > 0) else None
    return fn(C.c_void_p(stream or 0), int(n), qp, int(ldq), int(k), C.c_void_p(V.data_ptr()), int(ldv), int(nb),
              C.c_void_p(R.data_ptr()), int(R.stride(1)), C.c_void_p(work.data_ptr()),
              int(work.numel() * work.element_size()), C.c_void_p(status.data_ptr()))


def ortho_gram_chol(Q, V, R, work, status, k=None, stream=None):
    """First half of BCGS-PIP: [P; G] = [Q, V]^T V and T = Chol(G - P^T P) into R."""
    k = (Q.shape[1] if Q is not None else 0) if k is None else k
    return check(_ortho(load().ortho_gram_chol, Q, V, R, work, status, k, stream))


def ortho_gram_chol_dd(Q, V, R, work, status, k=None, stream=None):
    """ortho_gram_chol in double-float arithmetic (~2^-48 relative)."""
    k = (Q.shape[1] if Q is not None else 0) if k is None else k
    return check(_ortho(load().ortho_gram_chol_dd, Q, V, R, work, status, k, stream))


def ortho_gram_chol_tc(Q, V, R, work, status, k=None, stream=None):
    """ortho_gram_chol with the Gram on the tensor cores by exact slicing (k + nb <= 64)."""
    k = (Q.shape[1] if Q is not None else 0) if k is None else k
    return check(_ortho(load().ortho_gram_chol_tc, Q, V, R, work, status, k, stream))


def ortho_update(Q, V, R, status, k=None, stream=None, dd=False, tc=False):
    """Second half of BCGS-PIP: V <- (V - Q P) T^{-1} (dd: double-float arithmetic;
    tc: tensor cores by exact slicing)."""
    k = (Q.shape[1] if Q is not None else 0) if k is None else k
    n, nb = V.shape
    ldq = Q.stride(1) if (Q is not None and k > 0) else n
    qp = C.c_void_p(Q.data_ptr()) if (Q is not None and k > 0) else None
    fn = load().ortho_update_dd if dd else (load().ortho_update_tc if tc else load().ortho_update)
    return check(fn(C.c_void_p(stream or 0), int(n), qp, int(ldq), int(k),
                                     C.c_void_p(V.data_ptr()), int(V.stride(1)), int(nb),
                                     C.c_void_p(R.data_ptr()), int(R.stride(1)), C.c_void_p(status.data_ptr())))


def digits_bytes(n, capc):
    """Bytes of a digit basis of capc columns for n rows: 7 per value (seven
    biased 8-bit digits) plus an int32 exponent per 64-row chunk and column."""
    return int(load().ortho_digits_bytes(int(n), int(capc)))


def digits_fill(X, c0, digits, capc, stream=None):
    """Slice the columns of X (column-major CUDA tensor view) into digit columns c0 ..."""
    n, nc = X.shape
    return check(load().ortho_digits_fill(C.c_void_p(stream or 0), int(n), C.c_void_p(X.data_ptr()),
                                          int(X.stride(1)), int(c0), int(nc), C.c_void_p(digits.data_ptr()),
                                          int(capc)))


def ortho_gram_chol_tcd(Q, V, R, work, status, digits, capc, kc, k=None, stream=None):
    """ortho_gram_chol_tc reading the first kc columns of [Q, V] from the digit basis."""
    k = (Q.shape[1] if Q is not None else 0) if k is None else k
    n, nb = V.shape
    ldq = Q.stride(1) if (Q is not None and k > 0) else n
    qp = C.c_void_p(Q.data_ptr()) if (Q is not None and k > 0) else None
    return check(load().ortho_gram_chol_tcd(C.c_void_p(stream or 0), int(n), qp, int(ldq), int(k),
                                            C.c_void_p(V.data_ptr()), int(V.stride(1)), int(nb),
                                            C.c_void_p(R.data_ptr()), int(R.stride(1)), C.c_void_p(work.data_ptr()),
                                            int(work.numel() * work.element_size()), C.c_void_p(status.data_ptr()),
                                            C.c_void_p(digits.data_ptr()), int(capc), int(kc)))


def ortho_update_tcd(Q, V, R, status, digits, capc, k=None, stream=None):
    """ortho_update_tc that also writes the new V's digits into digit columns k .. k+nb-1."""
    k = (Q.shape[1] if Q is not None else 0) if k is None else k
    n, nb = V.shape
    ldq = Q.stride(1) if (Q is not None and k > 0) else n
    qp = C.c_void_p(Q.data_ptr()) if (Q is not None and k > 0) else None
    return check(load().ortho_update_tcd(C.c_void_p(stream or 0), int(n), qp, int(ldq), int(k),
                                         C.c_void_p(V.data_ptr()), int(V.stride(1)), int(nb),
                                         C.c_void_p(R.data_ptr()), int(R.stride(1)), C.c_void_p(status.data_ptr()),
                                         C.c_void_p(digits.data_ptr()), int(capc)))


def ortho_stage1_noalloc(Q, V, R, status, k=None, stream=None):
    """Stage 1 without a caller workspace, for callers that cannot allocate
    device memory: the scratch is a fixed array inside the library (nb <= 16,
    k + nb <= 64).  Calls that overlap on the GPU share that array and race."""
    k = (Q.shape[1] if Q is not None else 0) if k is None else k
    n, nb = V.shape
    ldq = Q.stride(1) if (Q is not None and k > 0) else n
    qp = C.c_void_p(Q.data_ptr()) if (Q is not None and k > 0) else None
    return check(load().ortho_stage1_noalloc(C.c_void_p(stream or 0), int(n), qp, int(ldq), int(k),
                                             C.c_void_p(V.data_ptr()), int(V.stride(1)), int(nb),
                                             C.c_void_p(R.data_ptr()), int(R.stride(1)),
                                             C.c_void_p(status.data_ptr())))


class OrthoPlan:
    """ortho_plan_create / _run / _destroy: the two-stage orthogonalization of
    an n x (1 + s nblk) panel in one call, on host (numpy or pinned torch CPU
    tensors) or device (torch CUDA tensors) buffers."""

    def __init__(self, n, s, nblk, arith=GMRES_ARITH_TC, stream=None):
        h = C.c_void_p()
        check(load().ortho_plan_create(C.byref(h), int(n), int(s), int(nblk), int(arith), C.c_void_p(stream or 0)))
        self.h, self.n, self.ncol = h, int(n), 1 + int(s) * int(nblk)
        self.nblk = int(nblk)

    @staticmethod
    def _addr(t):
        return C.c_void_p(t.data_ptr()) if hasattr(t, "data_ptr") else t.ctypes.data_as(C.c_void_p)

    def run(self, X, Q, Rhat=None, R2=None, on_device=None):
        """X, Q: column-major (n x ncol) views (``t.T`` of a (ncol, ld) tensor, or
        Fortran-ordered numpy arrays); Rhat, R2: (ncol x ncol) column-major or
        None.  Returns (status, block statuses)."""
        if on_device is None:
            on_device = bool(getattr(X, "is_cuda", False))
        ld = lambda a: (a.stride(1) if hasattr(a, "stride") and callable(a.stride) else a.strides[1] // 8)
        st = (C.c_int32 * (self.nblk + 1))()
        ldr = ld(Rhat) if Rhat is not None else (ld(R2) if R2 is not None else self.ncol)
        rc = load().ortho_plan_run(self.h, self._addr(X), int(ld(X)), self._addr(Q), int(ld(Q)),
                                   self._addr(Rhat) if Rhat is not None else None,
                                   self._addr(R2) if R2 is not None else None, int(ldr), int(on_device), st)
        if rc < 0 and rc != GMRES_ERR_BREAKDOWN:
            raise GmresError(rc, last_error())
        return rc, list(st)

    def close(self):
        if getattr(self, "h", None):
            load().ortho_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ortho_stage1(Q, V, R, work, status, k=None, stream=None):
    """BCGS-PIP of V against the first k columns of Q (stage 1 of §V).
    Tensors are column-major views (``t.T`` of a row-major (cols, ld) tensor)."""
    k = (Q.shape[1] if Q is not None else 0) if k is None else k
    return check(_ortho(load().ortho_stage1, Q, V, R, work, status, k, stream))


def ortho_stage1_shifted(Q, V, R, work, status, k=None, stream=None):
    """Stage 1 with the shifted Cholesky of shifted CholQR: T = Chol(G - P^T P +
    sigma I), sigma = 11 (n nb + nb (nb + 1)) u trace(G); FP64 arithmetic."""
    k = (Q.shape[1] if Q is not None else 0) if k is None else k
    return check(_ortho(load().ortho_stage1_shifted, Q, V, R, work, status, k, stream))


def ortho_stage1_f32(Q, V, R, work, status, k=None, stream=None):
    """Stage 1 on an FP32 basis (FP64 products and sums, FP64 R, FP32 result)."""
    k = (Q.shape[1] if Q is not None else 0) if k is None else k
    return check(_ortho(load().ortho_stage1_f32, Q, V, R, work, status, k, stream))


def ortho_stage2_f32(Q, V, R, work, status, k=None, stream=None):
    """Stage 2 on an FP32 basis (FP64 products and sums, FP64 R, FP32 result)."""
    k = (Q.shape[1] if Q is not None else 0) if k is None else k
    return check(_ortho(load().ortho_stage2_f32, Q, V, R, work, status, k, stream))


def ortho_stage2(Q, V, R, work, status, k=None, stream=None):
    """BCGS-PIP of the big panel V against the first k columns of Q (stage 2 of §V)."""
    k = (Q.shape[1] if Q is not None else 0) if k is None else k
    return check(_ortho(load().ortho_stage2, Q, V, R, work, status, k, stream))


def newton_shifts(H, s, sigma=None):
    """gmres_newton_shifts: the Newton-basis shifts from the k x k upper
    Hessenberg matrix H (host array-like) and, when ``sigma`` is given, the
    capacity scale (``sigma`` returned unchanged when the shifts span no
    interval).  Returns (theta[s] as a numpy array, sigma or None)."""
    import numpy as np
    Hh = np.asfortranarray(np.asarray(H, dtype=np.float64))
    k = Hh.shape[0]
    if Hh.ndim != 2 or Hh.shape[1] != k:
        raise ValueError("H must be square")
    th = (C.c_double * int(s))()
    sg = C.c_double(float(sigma)) if sigma is not None else None
    hp = Hh.ctypes.data if k else None
    check(load().gmres_newton_shifts(hp, max(k, 1), int(k), int(s), th, C.byref(sg) if sg is not None else None))
    return np.array(th[:], dtype=np.float64), (sg.value if sg is not None else None)
