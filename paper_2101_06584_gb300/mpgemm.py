"""Thin Python binding of libmpgemm.so (include/mpgemm.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Tensors are torch float64 CUDA tensors of shape (P, rows, cols)
(structure-of-arrays planes, row-major, plane 0 most significant) or, for
vectors, (P, n).  Calls are enqueued on torch's current CUDA stream.  There is
no CPU fallback: if the library is missing or a tensor is not on a CUDA
device, the call raises.
"""
import ctypes
import os

import torch

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libmpgemm.so")
P_OF = {"d": 1, "dd": 2, "td": 3, "qd": 4}   # "d": the binary64-only product
ALGO = {"auto": 0, "fp64": 1, "int8": 2, "bf16": 3, "crt": 4, "crt_bf16": 5, "crt2": 6, "crt2_bf16": 7}

_lib = None


class MPGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("mpgemm error %d: %s" % (code, msg))
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("trans_a", ctypes.c_int), ("trans_b", ctypes.c_int), ("algo", ctypes.c_int),
                ("split_k", ctypes.c_int), ("slices", ctypes.c_int), ("tile", ctypes.c_int),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t),
                ("strassen", ctypes.c_int)]


class Problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("A", ctypes.c_void_p * 4), ("lda", ctypes.c_int64),
                ("B", ctypes.c_void_p * 4), ("ldb", ctypes.c_int64),
                ("C", ctypes.c_void_p * 4), ("ldc", ctypes.c_int64),
                ("trans_a", ctypes.c_int), ("trans_b", ctypes.c_int)]


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmpgemm.so is not built (run paper_2101_06584_gb300.build.build())")
        _lib = _declare(ctypes.CDLL(LIB_PATH))
    return _lib


def _declare(L):
    i64, vp, i = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
    L.mpgemm_last_error.restype = ctypes.c_char_p
    L.mpgemm_set_stream.argtypes = [vp]
    L.mpgemm_get_stream.restype = vp
    for f in ("mp_quick_two_sum", "mp_two_sum", "mp_two_prod"):
        getattr(L, f).argtypes = [i64, vp, vp, vp, vp]
    L.mp_eft_int.argtypes = [i, i64, vp, vp, vp, vp]
    for f in ("mp_dd_add", "mp_dd_mul", "mp_td_add", "mp_td_add_merge", "mp_td_mul", "mp_td_mul_q",
              "mp_td_mul_accurate", "mp_qd_add", "mp_qd_mul", "mp_qd_add_accurate"):
        getattr(L, f).argtypes = [i64, vp, vp, vp]
    for f in ("mpgemm_d", "mpgemm_dd", "mpgemm_td", "mpgemm_qd"):
        getattr(L, f).argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64]
    L.mpgemm_ex.argtypes = [i, ctypes.POINTER(Opts), i64, i64, i64, vp, i64, vp, i64, vp, i64]
    L.mpgemm_workspace_size.argtypes = [i, ctypes.POINTER(Opts), i64, i64, i64]
    L.mpgemm_workspace_size.restype = ctypes.c_size_t
    L.mpgemm_dd_int8_static.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64, i]
    PP = ctypes.POINTER(Problem)
    L.mpgemm_batch_workspace_size.argtypes = [i, i, PP]
    L.mpgemm_batch_workspace_size.restype = ctypes.c_size_t
    L.mpgemm_batch_plan_create.argtypes = [i, i, PP, i, vp, ctypes.c_size_t, ctypes.POINTER(vp)]
    L.mpgemm_batch_run.argtypes = [vp]
    L.mpgemm_batch_plan_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int64 * 4)]
    L.mpgemm_batch_plan_destroy.argtypes = [vp]
    L.mpgemm_batch_autotune.argtypes = [i, i, PP, vp, ctypes.c_size_t, i, ctypes.POINTER(i),
                                        ctypes.POINTER(ctypes.c_float)]
    L.mpgemm_crt_beta.argtypes = [i, i64]
    L.mpgemm_crt_split_beta.argtypes = [i, i64]
    L.mpgemm_autotune.argtypes = [i, i64, i64, i64, vp, i64, vp, i64, vp, i64, i, ctypes.POINTER(i),
                                  ctypes.POINTER(ctypes.c_float)]
    L.mpgemm_tuned_tile.argtypes = [i, i64, i64, i64]
    L.mpgemm_tune_cache_reset.restype = None
    L.mpgemm_num_tiles.argtypes = [i]
    L.mpgemm_default_tile.argtypes = [i, i64, i64, i64]
    L.mpgemm_tc_status.argtypes = [vp]
    L.mpgemm_tile_info.argtypes = [i, i, ctypes.POINTER(ctypes.c_int * 6)]
    L.mpgemm_tile_int_ops.argtypes = [i, i]
    return L


def check(rc):
    if rc != 0:
        raise MPGError(rc, lib().mpgemm_last_error().decode())


def _bind_stream():
    lib().mpgemm_set_stream(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _require(t, name, P=None, ndim=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor (the library has no CPU path)" % name)
    if t.dtype != torch.float64:
        raise ValueError("%s must be float64" % name)
    if P is not None and t.shape[0] != P:
        raise ValueError("%s must have %d component planes, got %d" % (name, P, t.shape[0]))
    if ndim is not None and t.dim() != ndim:
        raise ValueError("%s must have %d dimensions" % (name, ndim))
    if t.numel() > 0 and t.stride(-1) != 1:
        raise ValueError("%s planes must be row-major with unit column stride" % name)


def planes(t):
    """Host array of the device pointers of the component planes of t."""
    P = t.shape[0]
    return (ctypes.c_void_p * P)(*[t[c].data_ptr() for c in range(P)])


def _ld(t):
    """Leading dimension of the planes of t (rows apart, in elements)."""
    if t.numel() == 0 or t.shape[1] <= 1:
        return max(t.shape[2], 1)
    return t.stride(1)


def gemm(prec, A, B, out=None, trans_a=False, trans_b=False, algo="auto", split_k=0, tile=0,
         slices=0, workspace=None, strassen=0):
    """C = op(A) op(B) for (P, rows, cols) planes; op = transpose when trans_*.

    A is (P, m, k) or, with trans_a, (P, k, m); B is (P, k, n) or, with
    trans_b, (P, n, k).  Returns C (P, m, n) (``out`` if given)."""
    P = P_OF[prec]
    _require(A, "A", P, 3)
    _require(B, "B", P, 3)
    m, k = (A.shape[2], A.shape[1]) if trans_a else (A.shape[1], A.shape[2])
    kb, n = (B.shape[2], B.shape[1]) if trans_b else (B.shape[1], B.shape[2])
    if kb != k:
        raise ValueError("inner dimensions differ: %d vs %d" % (k, kb))
    if out is None:
        out = torch.empty((P, m, n), dtype=torch.float64, device=A.device)
    _require(out, "out", P, 3)
    if tuple(out.shape[1:]) != (m, n):
        raise ValueError("out must be (P, %d, %d)" % (m, n))
    o = Opts(int(trans_a), int(trans_b), ALGO[algo], int(split_k), int(slices), int(tile),
             None, 0, int(strassen))
    if workspace is not None:
        _require_ws(workspace)
        o.workspace = workspace.data_ptr()
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    _bind_stream()
    check(lib().mpgemm_ex(P, ctypes.byref(o), m, n, k, planes(A), _ld(A), planes(B), _ld(B),
                          planes(out), _ld(out)))
    return out


def _require_ws(w):
    if not isinstance(w, torch.Tensor) or not w.is_cuda or not w.is_contiguous():
        raise ValueError("workspace must be a contiguous CUDA tensor")


def workspace_size(prec, m, n, k, algo="auto", slices=0, split_k=0, trans_a=False, trans_b=False,
                   strassen=0):
    o = Opts(int(trans_a), int(trans_b), ALGO[algo], int(split_k), int(slices), 0, None, 0, int(strassen))
    return int(lib().mpgemm_workspace_size(P_OF[prec], ctypes.byref(o), m, n, k))


def gemm_plain(prec, A, B, out=None):
    """C = A B through mpgemm_dd/td/qd (the paper's call, k-sequential)."""
    P = P_OF[prec]
    _require(A, "A", P, 3)
    _require(B, "B", P, 3)
    m, k = A.shape[1], A.shape[2]
    n = B.shape[2]
    if B.shape[1] != k:
        raise ValueError("inner dimensions differ")
    if out is None:
        out = torch.empty((P, m, n), dtype=torch.float64, device=A.device)
    _require(out, "out", P, 3)
    _bind_stream()
    fn = getattr(lib(), "mpgemm_" + prec)
    check(fn(m, n, k, planes(A), _ld(A), planes(B), _ld(B), planes(out), _ld(out)))
    return out


def _ld2(t):
    """Leading dimension of a 2-D row-major plane."""
    if t.numel() == 0 or t.shape[0] <= 1:
        return max(t.shape[1], 1)
    return t.stride(0)


def gemm_fp64(A, B, out=None, trans_a=False, trans_b=False, tile=0):
    """The binary64-only product C = op(A) op(B) of single planes (2-D float64
    CUDA tensors, e.g. the leading plane A[0] of a DD/TD/QD operand): one fma
    per term, k-sequential (mpgemm_d, or mpgemm_ex with P = 1 for transposes
    and a tile choice).  Returns C (m, n)."""
    for t, name in ((A, "A"), (B, "B")):
        _require(t, name, None, 2)
    m, k = (A.shape[1], A.shape[0]) if trans_a else (A.shape[0], A.shape[1])
    kb, n = (B.shape[1], B.shape[0]) if trans_b else (B.shape[0], B.shape[1])
    if kb != k:
        raise ValueError("inner dimensions differ: %d vs %d" % (k, kb))
    if out is None:
        out = torch.empty((m, n), dtype=torch.float64, device=A.device)
    _require(out, "out", None, 2)
    if tuple(out.shape) != (m, n):
        raise ValueError("out must be (%d, %d)" % (m, n))
    _bind_stream()
    if not trans_a and not trans_b and not tile:
        check(lib().mpgemm_d(m, n, k, A.data_ptr(), _ld2(A), B.data_ptr(), _ld2(B),
                             out.data_ptr(), _ld2(out)))
    else:
        o = Opts(int(trans_a), int(trans_b), ALGO["auto"], 0, 0, int(tile), None, 0, 0)
        one = lambda t: (ctypes.c_void_p * 1)(t.data_ptr())
        check(lib().mpgemm_ex(1, ctypes.byref(o), m, n, k, one(A), _ld2(A), one(B), _ld2(B),
                              one(out), _ld2(out)))
    return out


_VEC = {("dd", "add"): "mp_dd_add", ("dd", "mul"): "mp_dd_mul", ("td", "add"): "mp_td_add",
        ("td", "addm"): "mp_td_add_merge", ("td", "mul"): "mp_td_mul",
        ("td", "mulq"): "mp_td_mul_q", ("td", "mula"): "mp_td_mul_accurate",
        ("qd", "add"): "mp_qd_add", ("qd", "mul"): "mp_qd_mul", ("qd", "adda"): "mp_qd_add_accurate"}


def vec(prec, op, x, y, out=None):
    """Elementwise r = x op y over (P, n) SoA vectors: ``add``, ``mul``, or a
    variant -- ``addm`` (TDadd, Alg. 3), ``mulq`` (TDmulq), ``mula`` (accurate
    TD product), ``adda`` (accurate QD addition)."""
    P = P_OF[prec]
    _require(x, "x", P, 2)
    _require(y, "y", P, 2)
    if x.shape != y.shape:
        raise ValueError("x and y differ in shape")
    if out is None:
        out = torch.empty_like(x)
    _require(out, "out", P, 2)
    _bind_stream()
    check(getattr(lib(), _VEC[(prec, op)])(x.shape[1], planes(x), planes(y), planes(out)))
    return out


EFT_WHICH = {"quick_two_sum": 0, "two_sum": 1, "two_prod": 2}


def eft(which, a, b, int_pipes=False):
    """Elementwise EFT (quick_two_sum | two_sum | two_prod) of 1-D tensors; returns (s, e).

    With int_pipes the transformations run in their integer-pipe form
    (mp_eft_int), which returns the same bits."""
    for t, nm in ((a, "a"), (b, "b")):
        _require(t, nm)
    if a.shape != b.shape or a.dim() != 1:
        raise ValueError("a and b must be 1-D of equal length")
    s, e = torch.empty_like(a), torch.empty_like(a)
    _bind_stream()
    if int_pipes:
        check(lib().mp_eft_int(EFT_WHICH[which], a.numel(), a.data_ptr(), b.data_ptr(), s.data_ptr(),
                               e.data_ptr()))
    else:
        check(getattr(lib(), "mp_" + which)(a.numel(), a.data_ptr(), b.data_ptr(), s.data_ptr(),
                                            e.data_ptr()))
    return s, e


def crt_beta(moduli, k, split=False):
    """Bits per scaled entry of the CRT form with this many moduli at inner
    dimension k (split=True: with split integers)."""
    f = lib().mpgemm_crt_split_beta if split else lib().mpgemm_crt_beta
    b = f(int(moduli), int(k))
    check(b if b < 0 else 0)
    return b


def num_tiles(prec):
    return lib().mpgemm_num_tiles(P_OF[prec])


def tc_status(workspace):
    """The tcgen05 engine's status after a call with ``workspace`` (waits for
    the stream): 0, or the code of the role whose bounded wait gave up."""
    _require_ws(workspace)
    _bind_stream()
    code = lib().mpgemm_tc_status(ctypes.c_void_p(workspace.data_ptr()))
    check(code if code < 0 else 0)
    return code


def default_tile(prec, m, n, k):
    """The tile id (1-based) the library picks for an m x n x k FP64-EFT GEMM."""
    t = lib().mpgemm_default_tile(P_OF[prec], m, n, k)
    check(t if t < 0 else 0)
    return t


def autotune(prec, A, B, out=None, reps=3):
    """Time every FP64-EFT tile on C = A B (A (P, m, k), B (P, k, n), no
    transposes), remember the fastest for the shape's bucket (and in the file
    MPGEMM_TUNE_CACHE names) and return (tile id, ms per call)."""
    P = P_OF[prec]
    _require(A, "A", P, 3)
    _require(B, "B", P, 3)
    m, k, n = A.shape[1], A.shape[2], B.shape[2]
    if B.shape[1] != k:
        raise ValueError("inner dimensions differ: %d vs %d" % (k, B.shape[1]))
    if out is None:
        out = torch.empty((P, m, n), dtype=torch.float64, device=A.device)
    _require(out, "out", P, 3)
    tile, ms = ctypes.c_int(0), ctypes.c_float(0.0)
    _bind_stream()
    check(lib().mpgemm_autotune(P, m, n, k, planes(A), _ld(A), planes(B), _ld(B), planes(out), _ld(out),
                                int(reps), ctypes.byref(tile), ctypes.byref(ms)))
    return tile.value, ms.value


def tuned_tile(prec, m, n, k):
    """The remembered tile id of the bucket of (m, n, k), or 0."""
    return lib().mpgemm_tuned_tile(P_OF[prec], m, n, k)


def tune_cache_reset():
    """Forget remembered choices; the next lookup reads MPGEMM_TUNE_CACHE again."""
    lib().mpgemm_tune_cache_reset()


def tile_info(prec, tile):
    info = (ctypes.c_int * 6)()
    check(lib().mpgemm_tile_info(P_OF[prec], tile, ctypes.byref(info)))
    d = dict(zip(("bm", "bn", "bk", "tm", "tn", "threads"), list(info)))
    ints = lib().mpgemm_tile_int_ops(P_OF[prec], tile)
    if ints < 0:
        check(ints)
    d["int_ops"] = ints
    return d


def peak_probe(kind, blocks, iters, out):
    """Launch a throughput probe (kind 0 FP64 add, 1 mul, 2 fma, 3 mma.sync s8,
    4/5/6 TwoSum/FastTwoSum/TwoProd on the integer pipes) writing to ``out``
    (a CUDA float64 tensor of blocks*256 elements)."""
    if out.numel() < blocks * 256 or not out.is_cuda or out.dtype != torch.float64:
        raise ValueError("out must be a CUDA float64 tensor of at least blocks*256 elements")
    lib().mpgemm_peak_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    _bind_stream()
    check(lib().mpgemm_peak_probe(int(kind), int(blocks), int(iters), out.data_ptr()))


def _problem(prec, A, B, C, trans_a=False, trans_b=False):
    P = P_OF[prec]
    for t, nm in ((A, "A"), (B, "B"), (C, "C")):
        _require(t, nm, P, 3)
    m, k = (A.shape[2], A.shape[1]) if trans_a else (A.shape[1], A.shape[2])
    kb, n = (B.shape[2], B.shape[1]) if trans_b else (B.shape[1], B.shape[2])
    if kb != k or tuple(C.shape[1:]) != (m, n):
        raise ValueError("inconsistent problem shapes")
    q = Problem()
    q.m, q.n, q.k = m, n, k
    for c in range(P):
        q.A[c] = A[c].data_ptr()
        q.B[c] = B[c].data_ptr()
        q.C[c] = C[c].data_ptr()
    q.lda, q.ldb, q.ldc = _ld(A), _ld(B), _ld(C)
    q.trans_a, q.trans_b = int(trans_a), int(trans_b)
    return q


# Batch policies: 0-4 split problems into 16 x 16 or 32 x 32 tiles by an m*n
# threshold on the FP64-pipe arithmetic; BATCH_INT_POLICY puts every problem
# in 16 x 16 tiles with TwoSum (and for DD FastTwoSum) on the integer pipes.
BATCH_POLICIES = 6
BATCH_INT_POLICY = 5


def batch_int_ops(prec, policy):
    """The mpgemm_tile_int_ops-style mask a batch policy runs with."""
    return (3 if P_OF[prec] == 2 else 1) if policy == BATCH_INT_POLICY else 0


class BatchPlan:
    """A batch of independent products (A_i, B_i, C_i) in precision ``prec``,
    run as one persistent kernel replayed from a CUDA graph.  ``policy`` None
    runs the library's autotuner first.  The tensors must stay alive while the
    plan is used (the plan keeps references)."""

    def __init__(self, prec, triples, policy=None, reps=3):
        P = P_OF[prec]
        self.P = P
        self._keep = list(triples)
        self._probs = (Problem * max(1, len(triples)))(*[_problem(prec, *t) for t in triples])
        n = len(triples)
        nbytes = lib().mpgemm_batch_workspace_size(P, n, self._probs)
        dev = triples[0][0].device if triples else torch.device("cuda")
        self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
        self.tune_ms = None
        _bind_stream()
        if policy is None:
            best = ctypes.c_int()
            ms = ctypes.c_float()
            check(lib().mpgemm_batch_autotune(P, n, self._probs, self.workspace.data_ptr(),
                                              self.workspace.numel(), int(reps), ctypes.byref(best),
                                              ctypes.byref(ms)))
            policy = best.value
            self.tune_ms = ms.value
        self.policy = policy
        h = ctypes.c_void_p()
        check(lib().mpgemm_batch_plan_create(P, n, self._probs, int(policy),
                                             self.workspace.data_ptr(), self.workspace.numel(),
                                             ctypes.byref(h)))
        self._h = h

    def run(self):
        _bind_stream()
        check(lib().mpgemm_batch_run(self._h))

    def info(self):
        v = (ctypes.c_int64 * 4)()
        check(lib().mpgemm_batch_plan_info(self._h, ctypes.byref(v)))
        return dict(zip(("tiles", "grid", "policy", "count"), list(v)))

    def close(self):
        if getattr(self, "_h", None):
            lib().mpgemm_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
