"""The C-ABI library builds, loads and exports every function that
include/*.h declares; host-side argument validation rejects bad calls with
MPG_EINVAL and a message, without launching anything (no GPU needed: the
plane addresses below are never dereferenced)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2101_06584_gb300 import build, mpgemm
    build.build()
    return mpgemm.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b([A-Za-z_]\w*)\s*\(", text, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "return", "sizeof", "defined"):
                names.add(name)
    return sorted(names)


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for f in ("mpgemm_dd", "mpgemm_td", "mpgemm_qd", "mp_two_sum", "mp_two_prod",
              "mp_quick_two_sum", "mp_dd_add", "mp_qd_mul", "mpgemm_ex"):
        assert f in names


def test_every_declared_symbol_is_exported(L):
    missing = [f for f in declared_functions() if not hasattr(L, f)]
    assert not missing, missing


FAKE = 1 << 40       # plausible-looking device addresses, never dereferenced


def ptrs(*addrs):
    return (ctypes.c_void_p * len(addrs))(*addrs)


def planes(base, P, stride=1 << 30):
    return ptrs(*[base + c * stride for c in range(P)])


def err(L):
    return L.mpgemm_last_error().decode()


def test_gemm_rejects_negative_dims(L):
    A, B, C = planes(FAKE, 2), planes(2 * FAKE, 2), planes(3 * FAKE, 2)
    assert L.mpgemm_dd(-1, 4, 4, A, 4, B, 4, C, 4) == -1
    assert "m, n, k" in err(L)
    assert L.mpgemm_dd(4, 4, -2, A, 4, B, 4, C, 4) == -1


def test_gemm_rejects_small_leading_dims(L):
    A, B, C = planes(FAKE, 3), planes(2 * FAKE, 3), planes(3 * FAKE, 3)
    assert L.mpgemm_td(8, 9, 10, A, 9, B, 9, C, 9) == -1
    assert "lda" in err(L)
    assert L.mpgemm_td(8, 9, 10, A, 10, B, 8, C, 9) == -1
    assert "ldb" in err(L)
    assert L.mpgemm_td(8, 9, 10, A, 10, B, 9, C, 8) == -1
    assert "ldc" in err(L)


def test_gemm_rejects_null_planes(L):
    A, B, C = planes(FAKE, 4), planes(2 * FAKE, 4), planes(3 * FAKE, 4)
    A[2] = None
    assert L.mpgemm_qd(8, 8, 8, A, 8, B, 8, C, 8) == -1
    assert "A plane 2" in err(L)
    assert L.mpgemm_qd(8, 8, 8, None, 8, B, 8, C, 8) == -1


def test_gemm_rejects_overlap(L):
    A, B = planes(FAKE, 2), planes(2 * FAKE, 2)
    C = ptrs(FAKE + 64, 3 * FAKE)                       # C[0] inside A[0]
    assert L.mpgemm_dd(8, 8, 8, A, 8, B, 8, C, 8) == -1
    assert "overlaps A" in err(L)
    C = ptrs(3 * FAKE, 3 * FAKE + 8 * 8)                # C planes overlap each other
    assert L.mpgemm_dd(8, 8, 8, A, 8, B, 8, C, 8) == -1
    assert "C planes" in err(L)


def test_gemm_empty_is_a_noop(L):
    A, B, C = planes(FAKE, 2), planes(2 * FAKE, 2), planes(3 * FAKE, 2)
    assert L.mpgemm_dd(0, 8, 8, A, 8, B, 8, C, 8) == 0
    assert L.mpgemm_dd(8, 0, 8, A, 8, B, 1, C, 1) == 0


def test_ex_rejects_bad_options(L):
    from paper_2101_06584_gb300.mpgemm import Opts
    A, B, C = planes(FAKE, 2), planes(2 * FAKE, 2), planes(3 * FAKE, 2)
    o = Opts(0, 0, 0, 3, 0, 0, None, 0)
    assert L.mpgemm_ex(2, ctypes.byref(o), 8, 8, 8, A, 8, B, 8, C, 8) == -1
    assert "split_k" in err(L)
    o = Opts(0, 0, 0, 0, 0, 99, None, 0)
    assert L.mpgemm_ex(2, ctypes.byref(o), 8, 8, 8, A, 8, B, 8, C, 8) == -1
    assert "tile" in err(L)
    assert L.mpgemm_ex(5, None, 8, 8, 8, A, 8, B, 8, C, 8) == -1
    o = Opts(1, 0, 0, 0, 0, 0, None, 0)                  # trans_a: A stored k x m
    assert L.mpgemm_ex(2, ctypes.byref(o), 8, 8, 16, A, 4, B, 8, C, 8) == -1
    assert "lda" in err(L)


def test_strassen_options(L):
    """Workspace of the Strassen form and the argument errors it reports
    before any launch."""
    from paper_2101_06584_gb300.mpgemm import Opts
    size = L.mpgemm_workspace_size
    size.restype = ctypes.c_size_t
    o = Opts(0, 0, 0, 0, 0, 0, None, 0, 1)
    # one level: P (m/2 k/2 + k/2 n/2 + 7 m/2 n/2) doubles
    assert size(2, ctypes.byref(o), 8, 6, 4) == 2 * (4 * 2 + 2 * 3 + 7 * 4 * 3) * 8
    o = Opts(0, 0, 0, 0, 0, 0, None, 0, 2)
    # two levels: the outer level's blocks plus the inner level's, once
    assert size(4, ctypes.byref(o), 8, 8, 8) == 4 * ((16 + 16 + 7 * 16) + (4 + 4 + 7 * 4)) * 8
    assert size(2, ctypes.byref(o), 7, 8, 8) == 0              # odd m: the plain GEMM
    o = Opts(0, 0, 0, 0, 0, 0, None, 0, 0)
    assert size(2, ctypes.byref(o), 8, 8, 8) == 0
    A, B, C = planes(FAKE, 2), planes(2 * FAKE, 2), planes(3 * FAKE, 2)
    o = Opts(0, 0, 0, 0, 0, 0, None, 0, -1)
    assert L.mpgemm_ex(2, ctypes.byref(o), 8, 8, 8, A, 8, B, 8, C, 8) == -1
    assert "strassen" in err(L)
    o = Opts(1, 0, 0, 0, 0, 0, None, 0, 1)
    assert L.mpgemm_ex(2, ctypes.byref(o), 8, 8, 8, A, 8, B, 8, C, 8) == -4
    o = Opts(0, 0, 0, 2, 0, 0, None, 0, 1)
    assert L.mpgemm_ex(2, ctypes.byref(o), 8, 8, 8, A, 8, B, 8, C, 8) == -1
    o = Opts(0, 0, 0, 0, 0, 0, None, 0, 1)
    assert L.mpgemm_ex(2, ctypes.byref(o), 8, 8, 8, A, 8, B, 8, C, 8) == -3
    assert "workspace" in err(L)
    o = Opts(0, 0, 2, 0, 0, 0, None, 0, 1)                  # with a slicing form
    assert L.mpgemm_ex(2, ctypes.byref(o), 8, 8, 8, A, 8, B, 8, C, 8) == -1


def test_slicing_options(L):
    """Host-side limits of the slicing forms, each reported before any launch:
    the slice count, k beyond the exact int32 weight sums (S k 4096 < 2^31),
    the workspace (missing, misaligned, too small, overlapping an operand),
    the int8 tiling id and the grid's row limit."""
    from paper_2101_06584_gb300.mpgemm import Opts
    A, B, C = planes(FAKE, 4), planes(2 * FAKE, 4), planes(3 * FAKE, 4)
    W = 4 * FAKE                                        # 256-byte aligned, far from the operands
    big = 1 << 40
    for algo in (2, 3):                                 # int8, bf16
        o = Opts(0, 0, algo, 0, 17, 0, W, big)
        assert L.mpgemm_ex(2, ctypes.byref(o), 8, 8, 8, A, 8, B, 8, C, 8) == -1 and "slices" in err(L)
        o = Opts(0, 0, algo, 0, 41, 0, W, big)
        assert L.mpgemm_ex(4, ctypes.byref(o), 8, 8, 8, A, 8, B, 8, C, 8) == -1 and "slices" in err(L)
        # S = 14: k <= (2^31 - 1) // (14 * 4096) = 37449
        k = (2 ** 31 - 1) // (14 * 4096)
        o = Opts(0, 0, algo, 0, 14, 0, None, 0)
        assert L.mpgemm_ex(2, ctypes.byref(o), 8, 8, k + 1, A, k + 1, B, 8, C, 8) == -4
        assert "exceeds" in err(L)
        assert L.mpgemm_ex(2, ctypes.byref(o), 8, 8, k, A, k, B, 8, C, 8) == -3   # no workspace
        o = Opts(0, 0, algo, 0, 0, 0, W + 8, big)
        assert L.mpgemm_ex(2, ctypes.byref(o), 8, 8, 8, A, 8, B, 8, C, 8) == -3 and "aligned" in err(L)
        o = Opts(0, 0, algo, 0, 0, 0, W, 1024)
        assert L.mpgemm_ex(2, ctypes.byref(o), 8, 8, 8, A, 8, B, 8, C, 8) == -3 and "smaller" in err(L)
        o = Opts(0, 0, algo, 0, 0, 0, FAKE, big)        # on top of A
        assert L.mpgemm_ex(2, ctypes.byref(o), 8, 8, 8, A, 8, B, 8, C, 8) == -3 and "overlaps" in err(L)
    o = Opts(0, 0, 2, 0, 0, 4, W, big)                  # int8 tilings are 1..3
    assert L.mpgemm_ex(2, ctypes.byref(o), 8, 8, 8, A, 8, B, 8, C, 8) == -1 and "tile" in err(L)
    m = 64 * 65536                                      # 65536 row blocks of 64
    o = Opts(0, 0, 2, 0, 0, 0, W, big)
    assert L.mpgemm_ex(2, ctypes.byref(o), m, 8, 8, A, 8, B, 8, C, 8) == -1 and "too large" in err(L)


def test_version(L):
    assert L.mpgemm_version() == 106


def test_tc_status_validation(L):
    assert L.mpgemm_tc_status(None) == -1 and "NULL" in err(L)


def test_vector_validation(L):
    x, y, r = planes(FAKE, 2), planes(2 * FAKE, 2), planes(3 * FAKE, 2)
    assert L.mp_dd_add(-5, x, y, r) == -1
    assert L.mp_dd_add(0, None, None, None) == 0
    bad = ptrs(FAKE + 8, 3 * FAKE)                       # partial overlap with x[0]
    assert L.mp_dd_mul(100, x, y, bad) == -1
    assert "overlap" in err(L)
    assert L.mp_two_sum(10, FAKE, 2 * FAKE, 3 * FAKE, 3 * FAKE + 8) == -1
    # the integer-pipe form validates the same way, and its selector
    assert L.mp_eft_int(1, 0, None, None, None, None) == 0
    assert L.mp_eft_int(3, 4, FAKE, 2 * FAKE, 3 * FAKE, 4 * FAKE) == -1 and "which" in err(L)
    assert L.mp_eft_int(-1, 4, FAKE, 2 * FAKE, 3 * FAKE, 4 * FAKE) == -1
    assert L.mp_eft_int(2, -1, FAKE, 2 * FAKE, 3 * FAKE, 4 * FAKE) == -1
    assert L.mp_eft_int(0, 10, FAKE, 2 * FAKE, 3 * FAKE, 3 * FAKE + 8) == -1 and "overlap" in err(L)
    assert L.mp_eft_int(2, 4, None, 2 * FAKE, 3 * FAKE, 4 * FAKE) == -1


def test_tile_table(L):
    for P in (2, 3, 4):
        nt = L.mpgemm_num_tiles(P)
        assert nt >= 3
        for t in range(1, nt + 1):
            info = (ctypes.c_int * 6)()
            assert L.mpgemm_tile_info(P, t, ctypes.byref(info)) == 0
            bm, bn, bk, tm, tn, threads = list(info)
            assert bk > 0 and bm % tm == 0 and bn % tn == 0 and (bm // tm) * (bn // tn) == threads
            assert 0 <= L.mpgemm_tile_int_ops(P, t) <= 7
        info = (ctypes.c_int * 6)()
        assert L.mpgemm_tile_info(P, nt + 1, ctypes.byref(info)) == -1
        assert L.mpgemm_tile_int_ops(P, nt + 1) == -1 and L.mpgemm_tile_int_ops(P, 0) == -1
        # both forms are there: tiles on the FP64 pipe alone and tiles with
        # TwoSum on the integer pipes
        masks = [L.mpgemm_tile_int_ops(P, t) for t in range(1, nt + 1)]
        assert 0 in masks and any(m & 1 for m in masks)
    assert all(L.mpgemm_tile_int_ops(1, t) == 0 for t in range(1, L.mpgemm_num_tiles(1) + 1))


def _tile(L, P, t):
    info = (ctypes.c_int * 6)()
    assert L.mpgemm_tile_info(P, t, ctypes.byref(info)) == 0
    return tuple(info)[:2]


def test_default_tile_rule(L):
    """Without a device the library assumes 152 SMs: the largest candidate
    tile whose CTAs keep >= 90% of the SMs busy in the last wave, else the
    closest; from 256 outputs per SM (38912) the candidates are the tiles
    with TwoSum (DD: and FastTwoSum) on the integer pipes."""
    def pick(P, m, n):
        t = L.mpgemm_default_tile(P, m, n, 64)
        return _tile(L, P, t) + (L.mpgemm_tile_int_ops(P, t),)
    assert pick(4, 1024, 1024) == (16, 16, 1)       # 4096 CTAs: 27 per SM, 99.8%
    assert pick(3, 1024, 1024) == (16, 16, 1)
    assert pick(4, 256, 256) == (8, 8, 1)           # 16x16: 256 CTAs, 84%; 8x8: 1024 CTAs, 96%
    assert pick(3, 198, 198) == (8, 8, 1)           # 39204 outputs: 16x16 56%, 8x8 82% (closest)
    assert pick(3, 197, 197) == (8, 8, 0)           # 38809 outputs: below the threshold
    assert pick(2, 4096, 4096) == (16, 16, 3)
    assert pick(2, 2048, 2048) == (16, 16, 3)
    assert pick(2, 256, 256) == (8, 8, 3)           # 16x16: 84%, 8x8: 96%
    assert pick(2, 128, 128) == (8, 8, 0)           # 32x32: 11%, 16x16: 42%, 8x8 staging 128: 84%
    assert pick(2, 304, 128) == (16, 16, 3)         # 38912 outputs; 19 x 8 = 152 CTAs: one per SM
    assert pick(2, 303, 128) == (16, 16, 0)         # 38784 outputs; 32x32: 40 CTAs, 26%; 16x16: 100%
    assert pick(2, 640, 256) == (8, 8, 3)           # 16x16: 640 CTAs, 84%; 8x8: 2560 CTAs, 99%
    assert L.mpgemm_default_tile(5, 8, 8, 8) == -1 and "P must be" in err(L)
    assert L.mpgemm_default_tile(2, -1, 8, 8) == -1


def test_batch_plan_rejects_bad_problem(L):
    from paper_2101_06584_gb300.mpgemm import Problem
    probs = (Problem * 2)()
    for q in probs:
        q.m, q.n, q.k = 8, 8, 8
        q.lda, q.ldb, q.ldc = 8, 8, 8
        for c in range(2):
            q.A[c] = FAKE + c * (1 << 30)
            q.B[c] = 2 * FAKE + c * (1 << 30)
            q.C[c] = 3 * FAKE + c * (1 << 30)
    probs[1].ldb = 4                                   # too small
    h = ctypes.c_void_p()
    rc = L.mpgemm_batch_plan_create(2, 2, probs, 0, ctypes.c_void_p(4 * FAKE), 1 << 20, ctypes.byref(h))
    assert rc == -1 and "ldb" in err(L) and not h.value
    rc = L.mpgemm_batch_plan_create(2, 2, probs, 7, ctypes.c_void_p(4 * FAKE), 1 << 20, ctypes.byref(h))
    assert rc == -1 and "policy" in err(L)
    rc = L.mpgemm_batch_plan_create(2, 2, probs, 0, ctypes.c_void_p(4 * FAKE + 8), 1 << 20, ctypes.byref(h))
    assert rc == -3
    assert L.mpgemm_batch_workspace_size(2, 2, probs) > 256


def test_binary64_product_validation(L):
    """mpgemm_d (and mpgemm_ex with P = 1) check their arguments like the
    multi-component calls and take no slicing, split-K or Strassen option."""
    from paper_2101_06584_gb300.mpgemm import Opts
    A, B, C = FAKE, 2 * FAKE, 3 * FAKE
    assert L.mpgemm_d(-1, 4, 4, A, 4, B, 4, C, 4) == -1
    assert "m, n, k" in err(L)
    assert L.mpgemm_d(8, 9, 10, A, 9, B, 9, C, 9) == -1
    assert "lda" in err(L)
    assert L.mpgemm_d(8, 8, 8, FAKE, 8, B, 8, FAKE + 64, 8) == -1
    assert "overlaps A" in err(L)
    assert L.mpgemm_d(0, 8, 8, A, 8, B, 8, C, 8) == 0
    one = lambda a: ptrs(a)
    for opts in (Opts(0, 0, 2, 0, 0, 0, None, 0), Opts(0, 0, 0, 4, 0, 0, None, 0),
                 Opts(0, 0, 0, 0, 0, 0, None, 0, 1)):
        assert L.mpgemm_ex(1, ctypes.byref(opts), 8, 8, 8, one(A), 8, one(B), 8, one(C), 8) == -1
        assert "P = 1" in err(L)
    assert L.mpgemm_num_tiles(1) == 4
    info = (ctypes.c_int * 6)()
    assert L.mpgemm_tile_info(1, 1, ctypes.byref(info)) == 0 and list(info)[:2] == [64, 64]
    assert L.mpgemm_version() >= 102


def test_crt_form_host_checks(L):
    """The CRT form's bit count agrees with the oracle's definition for every
    moduli count and several k (which checks the library's moduli and their
    product), its workspace follows the stated layout, and bad requests are
    refused before any launch."""
    from oracle import crt as R
    from paper_2101_06584_gb300.mpgemm import Opts
    for N in range(1, 50):
        for k in (1, 2, 127, 1024, 4096, 37449, 131071):
            assert L.mpgemm_crt_beta(N, k) == R.beta_bits(N, k), (N, k)
    assert L.mpgemm_crt_beta(0, 8) == -1 and L.mpgemm_crt_beta(50, 8) == -1
    r = lambda x: (x + 127) // 128 * 128
    r256 = lambda x: (x + 255) // 256 * 256
    for (m, n, k, N) in ((100, 70, 300, 28), (4096, 4096, 4096, 26), (1, 1, 1, 49)):
        for algo, head, eb in ((4, 0, 1), (5, 256, 2)):           # int8; tcgen05: header, bf16 residues
            o = Opts(0, 0, algo, 0, N, 0, None, 0)
            mp = r(m)
            want = (head + r256(N * mp * r(k) * eb) + r256(N * r(n) * r(k) * eb) + r256(4 * mp) +
                    r256(4 * r(n)) + r256(N * mp * r(n)))
            assert L.mpgemm_workspace_size(2, ctypes.byref(o), m, n, k) == want, (algo, m, n, k, N)
    A, B, C = planes(FAKE, 2), planes(2 * FAKE, 2), planes(3 * FAKE, 2)
    for N, k, code, text in ((50, 8, -1, "moduli"), (1, 200, -4, "no bits"), (28, 8, -3, "workspace")):
        o = Opts(0, 0, 4, 0, N, 0, None, 0)
        assert L.mpgemm_ex(2, ctypes.byref(o), 8, 8, k, A, k, B, 8, C, 8) == code
        assert text in err(L)
    o = Opts(0, 0, 4, 0, 28, 0, None, 0)
    big = 131072
    assert L.mpgemm_ex(2, ctypes.byref(o), 8, 8, big, A, big, B, 8, C, 8) == -4
    assert "int32" in err(L)


def test_crt_split_host_checks(L):
    """Split integers: the bit count agrees with the oracle's definition
    (beta = 2w, the largest w with k 2^(2w) < M), the workspace holds 2N
    residue planes per operand and 3N product planes, and k above 65535, too
    few moduli and more than 316 bits are refused before any launch."""
    from oracle import crt as R
    from paper_2101_06584_gb300.mpgemm import Opts
    for N in range(1, 50):
        for k in (1, 2, 127, 1024, 4096, 37449, 65535):
            assert L.mpgemm_crt_split_beta(N, k) == R.beta_bits(N, k, halves=2), (N, k)
    assert L.mpgemm_crt_split_beta(0, 8) == -1 and L.mpgemm_crt_split_beta(50, 8) == -1
    assert R.k_limit(2) == 65535
    r = lambda x: (x + 127) // 128 * 128
    r256 = lambda x: (x + 255) // 256 * 256
    for (m, n, k, N) in ((100, 70, 300, 28), (1024, 1024, 1024, 30), (1, 1, 1, 40)):
        for algo, head, eb in ((6, 0, 1), (7, 256, 2)):
            o = Opts(0, 0, algo, 0, N, 0, None, 0)
            mp = r(m)
            want = (head + r256(2 * N * mp * r(k) * eb) + r256(2 * N * r(n) * r(k) * eb) + r256(4 * mp) +
                    r256(4 * r(n)) + r256(3 * N * mp * r(n)))
            assert L.mpgemm_workspace_size(4, ctypes.byref(o), m, n, k) == want, (algo, m, n, k, N)
    o = Opts(0, 0, 6, 0, 0, 0, None, 0)                       # default moduli: 16 / 22 / 30
    for P, N in ((2, 16), (3, 22), (4, 30)):
        want = r256(2 * N * 128 * 128) * 2 + 2 * 512 + r256(3 * N * 128 * 128)
        assert L.mpgemm_workspace_size(P, ctypes.byref(o), 64, 64, 64) == want
    A, B, C = planes(FAKE, 4), planes(2 * FAKE, 4), planes(3 * FAKE, 4)
    # N = 1: M = 256 leaves w = 0 at k = 200; 49 moduli at k = 8: 2w = 336 > 316
    for N, k, code, text in ((50, 8, -1, "moduli"), (1, 200, -4, "no bits"), (49, 8, -4, "316"),
                             (30, 8, -3, "workspace")):
        o = Opts(0, 0, 6, 0, N, 0, None, 0)
        assert L.mpgemm_ex(4, ctypes.byref(o), 8, 8, k, A, k, B, 8, C, 8) == code, (N, k)
        assert text in err(L)
    o = Opts(0, 0, 7, 0, 30, 0, None, 0)
    big = 65536
    assert L.mpgemm_ex(4, ctypes.byref(o), 8, 8, big, A, big, B, 8, C, 8) == -4
    assert "int32" in err(L)


def test_tune_cache_file(L, tmp_path, monkeypatch):
    """The autotuner's cache file: entries of this device ("none" without a
    GPU) are found by shape bucket (m, n, k rounded up to powers of two),
    lines that do not parse, other devices' entries and out-of-range tile ids
    are ignored, a missing file or no MPGEMM_TUNE_CACHE means no choice, and
    a reset re-reads the environment."""
    nt = L.mpgemm_num_tiles(2)
    path = tmp_path / "tune.json"
    path.write_text(
        '{\n "version": 1,\n "entries": {\n'
        '  "none|gemm:2:7:7:7": {"choice": 3, "ms": 0.25},\n'
        '  "none|gemm:2:12:12:12": {"choice": %d, "ms": 1.5},\n'
        '  this line is not an entry\n'
        '  "other GPU/99|gemm:3:10:10:10": {"choice": 1, "ms": 2},\n'
        '  "none|gemm:4:10:10:10": {"choice": 2, "ms": 9.5}\n'
        ' }\n}\n' % (nt + 1))
    monkeypatch.delenv("MPGEMM_TUNE_CACHE", raising=False)
    L.mpgemm_tune_cache_reset()
    assert L.mpgemm_tuned_tile(2, 128, 128, 128) == 0               # no file named
    monkeypatch.setenv("MPGEMM_TUNE_CACHE", str(path))
    L.mpgemm_tune_cache_reset()
    assert L.mpgemm_tuned_tile(2, 128, 128, 128) == 3
    assert L.mpgemm_tuned_tile(2, 65, 100, 127) == 3               # the same bucket: 2^7 each
    assert L.mpgemm_tuned_tile(2, 129, 128, 128) == 0              # the next bucket of m
    assert L.mpgemm_tuned_tile(2, 4096, 4096, 4096) == 0           # tile id out of range
    assert L.mpgemm_tuned_tile(3, 1024, 1024, 1024) == 0           # another device's entry
    assert L.mpgemm_tuned_tile(4, 1000, 600, 1024) == 2
    assert L.mpgemm_tuned_tile(4, -1, 600, 1024) == 0
    monkeypatch.setenv("MPGEMM_TUNE_CACHE", str(tmp_path / "missing.json"))
    assert L.mpgemm_tuned_tile(2, 128, 128, 128) == 3              # still the choices in memory
    L.mpgemm_tune_cache_reset()
    assert L.mpgemm_tuned_tile(2, 128, 128, 128) == 0
    monkeypatch.delenv("MPGEMM_TUNE_CACHE")
    L.mpgemm_tune_cache_reset()
