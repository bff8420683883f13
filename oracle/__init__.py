"""CPU oracle for DD/TD/QD arithmetic and GEMM -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It is the plain, slow reference the CUDA library
is checked against and shares no code with it.

Numbers are structure-of-arrays planes: a P-component array is a numpy array
of shape (P, ...) of float64, component 0 the most significant (Sec. 2.5).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
P_OF = {"dd": 2, "td": 3, "qd": 4}


def lib(path=None):
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if path is not None:
        return _load(path)
    if _lib is None:
        _lib = _load(_build.build())
    return _lib


def _load(path):
    L = ctypes.CDLL(path)
    d = ctypes.c_double
    pd = ctypes.POINTER(ctypes.c_double)
    for name in ("or_quick_two_sum", "or_two_sum", "or_two_prod"):
        f = getattr(L, name)
        f.argtypes = [d, d, pd, pd]
        f.restype = None
    for name in ("or_three_sum", "or_three_sum2"):
        getattr(L, name).argtypes = [pd, pd, pd]
    L.or_renorm5.argtypes = [pd, pd]
    L.or_vec_sum.argtypes = [ctypes.c_int, pd, pd]
    L.or_vseb.argtypes = [ctypes.c_int, pd, ctypes.c_int, pd]
    for name in ("or_dd_add", "or_dd_mul", "or_td_add", "or_td_addq", "or_td_mul",
                 "or_td_mulq", "or_td_mul_acc", "or_qd_add", "or_qd_mul", "or_qd_add_acc"):
        getattr(L, name).argtypes = [pd, pd, pd]
    vp = ctypes.c_void_p
    L.or_vec_op.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, vp, vp, vp]
    L.or_vec_op.restype = ctypes.c_int
    L.or_vec_eft.argtypes = [ctypes.c_int, ctypes.c_int64, vp, vp, vp, vp]
    L.or_vec_eft.restype = ctypes.c_int
    L.or_gemm.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                          vp, ctypes.c_int64, vp, ctypes.c_int64, vp, ctypes.c_int64,
                          ctypes.c_int]
    L.or_gemm.restype = ctypes.c_int
    L.or_dgemm.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                           vp, ctypes.c_int64, vp, ctypes.c_int64, vp, ctypes.c_int64,
                           ctypes.c_int]
    L.or_dgemm.restype = ctypes.c_int
    return L


# ------------------------------------------------------------ scalar calls

def _eft(name, a, b, L=None):
    L = L or lib()
    s, e = ctypes.c_double(), ctypes.c_double()
    getattr(L, name)(float(a), float(b), ctypes.byref(s), ctypes.byref(e))
    return s.value, e.value


def quick_two_sum(a, b, L=None):
    return _eft("or_quick_two_sum", a, b, L)


def two_sum(a, b, L=None):
    return _eft("or_two_sum", a, b, L)


def two_prod(a, b, L=None):
    return _eft("or_two_prod", a, b, L)


def _arr(vals, n=None):
    vals = list(vals)
    if n is not None:
        vals = vals + [0.0] * (n - len(vals))
    return (ctypes.c_double * len(vals))(*[float(v) for v in vals])


def three_sum(a, b, c, L=None):
    L = L or lib()
    x, y, z = ctypes.c_double(a), ctypes.c_double(b), ctypes.c_double(c)
    L.or_three_sum(ctypes.byref(x), ctypes.byref(y), ctypes.byref(z))
    return x.value, y.value, z.value


def three_sum2(a, b, c, L=None):
    L = L or lib()
    x, y, z = ctypes.c_double(a), ctypes.c_double(b), ctypes.c_double(c)
    L.or_three_sum2(ctypes.byref(x), ctypes.byref(y), ctypes.byref(z))
    return x.value, y.value


def renorm5(c, L=None):
    L = L or lib()
    cin, r = _arr(c), _arr([], 4)
    L.or_renorm5(cin, r)
    return tuple(r)


def vec_sum(x, L=None):
    L = L or lib()
    xin, e = _arr(x), _arr([], len(x))
    L.or_vec_sum(len(x), xin, e)
    return tuple(e)


def vseb(e, k, L=None):
    L = L or lib()
    ein, r = _arr(e), _arr([], k)
    L.or_vseb(len(e), ein, k, r)
    return tuple(r)


_SCALAR = {("dd", "add"): "or_dd_add", ("dd", "mul"): "or_dd_mul",
           ("td", "add"): "or_td_addq", ("td", "addm"): "or_td_add",
           ("td", "mul"): "or_td_mul",
           ("td", "mulq"): "or_td_mulq", ("td", "mula"): "or_td_mul_acc",
           ("qd", "add"): "or_qd_add", ("qd", "mul"): "or_qd_mul", ("qd", "adda"): "or_qd_add_acc"}
# elementwise op codes of or_vec_op
VEC_OPS = {"add": 0, "mul": 1, "addm": 2, "mulq": 3, "mula": 4, "adda": 5}


def op(prec, name, x, y, L=None):
    """Scalar multi-component op; ``name`` in add/mul, or a variant: ``addm``
    (TDadd, Alg. 3), ``mulq`` (TDmulq), ``mula`` (accurate TD product),
    ``adda`` (accurate QD addition)."""
    L = L or lib()
    P = P_OF[prec]
    r = _arr([], P)
    getattr(L, _SCALAR[(prec, name)])(_arr(x), _arr(y), r)
    return tuple(r)


# ------------------------------------------------------------ array calls

def _planes_ptrs(arr):
    arr = np.asarray(arr)
    assert arr.dtype == np.float64 and arr.flags.c_contiguous
    P = arr.shape[0]
    return (ctypes.c_void_p * P)(*[arr[c].ctypes.data for c in range(P)])


def vec_op(prec, name, x, y, L=None):
    """Elementwise r = x op y over SoA vectors of shape (P, n); op names as
    in ``op``."""
    L = L or lib()
    P = P_OF[prec]
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    assert x.shape == y.shape and x.shape[0] == P
    r = np.empty_like(x)
    n = x[0].size
    rc = L.or_vec_op(P, VEC_OPS[name], n, _planes_ptrs(x), _planes_ptrs(y),
                     _planes_ptrs(r))
    assert rc == 0
    return r


def vec_eft(which, a, b, L=None):
    L = L or lib()
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    s, e = np.empty_like(a), np.empty_like(a)
    idx = {"quick_two_sum": 0, "two_sum": 1, "two_prod": 2}[which]
    rc = L.or_vec_eft(idx, a.size, a.ctypes.data, b.ctypes.data, s.ctypes.data, e.ctypes.data)
    assert rc == 0
    return s, e


def gemm(prec, A, B, nthreads=1, L=None):
    """C = A B (Eq. 1, k-sequential) for planes A (P,m,k) and B (P,k,n)."""
    L = L or lib()
    P = P_OF[prec]
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    assert A.shape[0] == P and B.shape[0] == P and A.shape[2] == B.shape[1]
    m, k = A.shape[1], A.shape[2]
    n = B.shape[2]
    C = np.zeros((P, m, n), dtype=np.float64)
    rc = L.or_gemm(P, m, n, k, _planes_ptrs(A), k, _planes_ptrs(B), n, _planes_ptrs(C), n,
                   int(nthreads))
    assert rc == 0
    return C


def dgemm(A, B, nthreads=1, L=None):
    """C = A B in plain binary64 (Eq. 1, k-sequential, one fma per term) for
    single planes A (m, k) and B (k, n)."""
    L = L or lib()
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    assert A.ndim == 2 and B.ndim == 2 and A.shape[1] == B.shape[0]
    m, k = A.shape
    n = B.shape[1]
    C = np.zeros((m, n), dtype=np.float64)
    rc = L.or_dgemm(m, n, k, A.ctypes.data, k, B.ctypes.data, n, C.ctypes.data, n, int(nthreads))
    assert rc == 0
    return C


def gemm_entries(prec, A, B, rows, cols, nthreads=1, L=None):
    """Entries C[rows[t], cols[t]] of the k-sequential product, one by one."""
    A = np.asarray(A)
    B = np.asarray(B)
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    Asub = np.ascontiguousarray(A[:, rows, :])              # (P, s, k)
    Bsub = np.ascontiguousarray(B[:, :, cols].transpose(0, 2, 1))  # (P, s, k)
    out = np.empty((A.shape[0], len(rows)))
    for t in range(len(rows)):
        c = gemm(prec, Asub[:, t:t + 1, :], Bsub[:, t:t + 1, :].transpose(0, 2, 1),
                 nthreads=1, L=L)
        out[:, t] = c[:, 0, 0]
    return out


def num_cpus():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1
