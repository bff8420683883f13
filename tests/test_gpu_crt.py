"""The CRT form (MPG_ALGO_INT8_CRT, and MPG_ALGO_BF16_CRT on tcgen05) on the
GPU against its oracle
(oracle/crt.py): the residues in the workspace equal the oracle's for every
modulus; the results are bit-identical to the oracle's steps for DD, TD and
QD, ragged shapes spanning several tiles, both transposes, cancelling inputs,
outputs down to the subnormal range, one modulus and all 49, and at the
largest k the form accepts; at the DD 4096^3 workload's full size a 16 x 16
grid of entries is bit-identical and two whole rows are within n 2^-100 of
the exact product.  The same for split integers (MPG_ALGO_INT8_CRT_SPLIT and
MPG_ALGO_BF16_CRT_SPLIT), with QD 1024^3 at full size within n 2^-200."""
import numpy as np
import pytest

from gpu_util import assert_bitwise, dev, host, torch_cuda
from oracle import crt as R
from oracle import exact as X
from paper_2101_06584_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


ENGINES = ["crt", "crt_bf16"]


def _run(torch, prec, A, B, N, trans_a=False, trans_b=False, algo="crt"):
    from paper_2101_06584_gb300 import mpgemm as mm
    Ad = dev(torch, A.transpose(0, 2, 1) if trans_a else A)
    Bd = dev(torch, B.transpose(0, 2, 1) if trans_b else B)
    m, k = A.shape[1], A.shape[2]
    n = B.shape[2]
    ws = torch.empty(mm.workspace_size(prec, m, n, k, algo=algo, slices=N), dtype=torch.uint8, device="cuda")
    C = mm.gemm(prec, Ad, Bd, trans_a=trans_a, trans_b=trans_b, algo=algo, slices=N, workspace=ws)
    if algo == "crt_bf16":
        assert mm.tc_status(ws) == 0, "tcgen05 kernel reported a timeout"
    return host(C), host(ws)


def _layout(N, m, n, k):
    r = lambda x, q: (max(x, 1) + q - 1) // q * q
    mp, np_, kp = r(m, 128), r(n, 128), r(k, 128)
    offB = r(N * mp * kp, 256)
    offSig = offB + r(N * np_ * kp, 256)
    offTau = offSig + r(mp * 4, 256)
    return mp, np_, kp, offB, offSig, offTau


@pytest.mark.parametrize("prec,N", [("dd", 1), ("dd", 28), ("td", 44), ("qd", 49)])
def test_residues_and_result_bitwise(torch, prec, N):
    P = I.P_OF[prec]
    rng = np.random.default_rng(800 + P + N)
    m, n, k = 37, 45, 53 if N > 1 else 3
    A, B = I.uniform(P, (m, k), rng), I.ill_scaled(P, (k, n), rng)
    C, ws = _run(torch, prec, A, B, N)
    beta = R.beta_bits(N, k)
    mp, np_, kp, offB, offSig, offTau = _layout(N, m, n, k)
    sig, RA = R.residues(A, N, beta)
    tau, RB = R.residues(np.ascontiguousarray(B.transpose(0, 2, 1)), N, beta)
    ga = ws[:N * mp * kp].view(np.int8).reshape(N, mp, kp)
    gb = ws[offB:offB + N * np_ * kp].view(np.int8).reshape(N, np_, kp)
    assert (ws[offSig:offSig + 4 * m].view(np.int32) == sig).all()
    assert (ws[offTau:offTau + 4 * n].view(np.int32) == tau).all()
    assert (ga[:, :m, :k] == RA).all() and not ga[:, m:, :].any() and not ga[:, :, k:].any()
    assert (gb[:, :n, :k] == RB).all() and not gb[:, n:, :].any() and not gb[:, :, k:].any()
    want, _, _, _ = R.gemm(A, B, N)
    assert_bitwise(C, want, "%s crt N=%d" % (prec, N))
    Ct, _ = _run(torch, prec, A, B, N, algo="crt_bf16")
    assert_bitwise(Ct, want, "%s crt on tcgen05 N=%d" % (prec, N))


@pytest.mark.parametrize("algo", ENGINES)
@pytest.mark.parametrize("prec", ["dd", "td"])
def test_transposes_tiles_and_cancellation(torch, prec, algo):
    """Several 128 x 128 tiles with ragged edges, every transpose, cancelling
    ill-scaled operands, k over several 1024-wide drains of the tcgen05
    engine's accumulators."""
    P = I.P_OF[prec]
    rng = np.random.default_rng(810 + P)
    A, B = I.cancelling_pair(P, 150, 270, 2300, rng)
    N = 28 if prec == "dd" else 44
    rows, cols = [0, 77, 127, 128, 149], [0, 100, 127, 128, 255, 256, 269]
    want, _, _, _ = R.gemm(A, B, N, rows=rows, cols=cols)
    first = None
    for ta, tb in ((False, False), (True, False), (False, True), (True, True)):
        C, _ = _run(torch, prec, A, B, N, trans_a=ta, trans_b=tb, algo=algo)
        assert_bitwise(C[:, rows][:, :, cols], want, "%s %s trans %s %s" % (prec, algo, ta, tb))
        if first is None:
            first = C
        assert_bitwise(C, first, "%s %s transposes agree" % (prec, algo))


@pytest.mark.parametrize("algo", ENGINES)
@pytest.mark.parametrize("prec", ["dd", "qd"])
def test_products_below_the_normal_range(torch, prec, algo):
    """Rows of A scaled by 1 .. 2^-1060 and columns of B by 1 .. 2^-530: the
    components of the recovered products run through the subnormal range and
    down to signed zeros; every entry bit-identical to the oracle."""
    P = I.P_OF[prec]
    rng = np.random.default_rng(820 + P)
    m, n, k = 40, 36, 64
    A, B = I.uniform(P, (m, k), rng), I.uniform(P, (k, n), rng)
    A *= np.array([1.0, 2.0 ** -500, 2.0 ** -530, 2.0 ** -1060])[np.arange(m) % 4][None, :, None]
    B *= np.array([1.0, 2.0 ** -500, 2.0 ** -530])[(np.arange(n) // 2) % 3][None, None, :]
    C, _ = _run(torch, prec, A, B, 30, algo=algo)
    want, _, _, _ = R.gemm(A, B, 30)
    assert ((np.abs(want) < 2.0 ** -1022) & (want != 0)).any() and np.isfinite(want).all()
    assert_bitwise(C, want, "%s crt tiny products" % prec)


def test_largest_k_and_refusal(torch):
    """k = 131071, the largest whose residue products sum exactly in int32:
    sampled entries bit-identical to the oracle; k + 1 is refused."""
    from paper_2101_06584_gb300 import mpgemm as mm
    k = R.k_limit()
    m = n = 16
    rng = np.random.default_rng(830)
    A, B = I.uniform(2, (m, k), rng), I.uniform(2, (k, n), rng)
    C, _ = _run(torch, "dd", A, B, 40)
    want, _, _, _ = R.gemm(A, B, 40, rows=[0, 15], cols=[3, 9])
    assert_bitwise(C[:, [0, 15]][:, :, [3, 9]], want, "crt at the largest k")
    Ct, _ = _run(torch, "dd", A, B, 40, algo="crt_bf16")
    assert_bitwise(Ct, C, "both engines at the largest k")
    A1 = np.concatenate([A, np.zeros((2, m, 1))], axis=2)
    B1 = np.concatenate([B, np.zeros((2, 1, n))], axis=1)
    with pytest.raises(mm.MPGError) as e:
        mm.gemm("dd", dev(torch, A1), dev(torch, B1), algo="crt", slices=40,
                workspace=torch.empty(1 << 20, dtype=torch.uint8, device="cuda"))
    assert e.value.code == -4


@pytest.mark.parametrize("N", [23, 28])          # 23: the count the benchmark chooses
def test_full_size_dd(torch, N):
    """DD 4096^3 on the uniform inputs of that workload's seed: the tcgen05
    engine equals the int8 engine on every entry (compared on the device), a
    16 x 16 grid of random rows and columns is bit-identical to the oracle,
    and two whole rows with the grid are within n 2^-100 of the exact
    product."""
    from paper_2101_06584_gb300 import mpgemm as mm
    n = 4096
    rng = I.rng_for(2)
    A, B = I.uniform(2, (n, n), rng), I.uniform(2, (n, n), rng)
    Ad, Bd = dev(torch, A), dev(torch, B)
    out = {}
    for algo in ENGINES:
        ws = torch.empty(mm.workspace_size("dd", n, n, n, algo=algo, slices=N), dtype=torch.uint8, device="cuda")
        out[algo] = mm.gemm("dd", Ad, Bd, algo=algo, slices=N, workspace=ws)
        if algo == "crt_bf16":
            assert mm.tc_status(ws) == 0
        del ws
    diff = int((out["crt"].view(torch.int64) != out["crt_bf16"].view(torch.int64)).sum())
    assert diff == 0, "%d values differ between the engines" % diff
    C = host(out["crt_bf16"])
    del out
    srng = np.random.default_rng(840)
    rows = sorted(int(x) for x in srng.choice(n, 16, replace=False))
    cols = sorted(int(x) for x in srng.choice(n, 16, replace=False))
    want, _, _, _ = R.gemm(A, B, N, rows=rows, cols=cols)
    assert_bitwise(C[:, rows][:, :, cols], want, "crt 4096 grid")
    full = sorted(int(x) for x in srng.choice(n, 2, replace=False))
    ent = sorted({(i, j) for i in full for j in range(n)} | {(i, j) for i in rows for j in cols})
    err = X.gemm_error(C, A, B, ent)
    assert err["err_abs"] <= n * 2.0 ** -100, err


def test_tcgen05_abort_path(torch):
    """The abort path of the tcgen05 CRT kernel: with MPGEMM_TEST_TC_ABORT=1 the
    producer gives up before any load; the call returns, the status names the
    producer, and the next call is bit-identical to the int8 engine."""
    import os
    from paper_2101_06584_gb300 import mpgemm as mm
    rng = np.random.default_rng(850)
    A, B = I.uniform(2, (200, 300), rng), I.uniform(2, (300, 150), rng)
    Ad, Bd = dev(torch, A), dev(torch, B)
    ws = torch.empty(mm.workspace_size("dd", 200, 150, 300, algo="crt_bf16", slices=28), dtype=torch.uint8,
                     device="cuda")
    os.environ["MPGEMM_TEST_TC_ABORT"] = "1"
    try:
        mm.gemm("dd", Ad, Bd, algo="crt_bf16", slices=28, workspace=ws)
        code = mm.tc_status(ws)
    finally:
        del os.environ["MPGEMM_TEST_TC_ABORT"]
    assert code == 1 and "producer" in mm.lib().mpgemm_last_error().decode()
    got = host(mm.gemm("dd", Ad, Bd, algo="crt_bf16", slices=28, workspace=ws))
    assert mm.tc_status(ws) == 0
    want, _ = _run(torch, "dd", A, B, 28)
    assert_bitwise(got, want, "after an aborted call")


def test_tcgen05_several_tiles(torch):
    """Several 128 x 128 tiles with ragged edges and a k over several drains
    on the tcgen05 engine: bit-identical to the int8 engine and, on sampled
    entries, to the oracle."""
    from paper_2101_06584_gb300 import mpgemm as mm
    rng = np.random.default_rng(861)
    m, n, k, N = 530, 300, 2200, 26
    A, B = I.uniform(2, (m, k), rng), I.ill_scaled(2, (k, n), rng)
    C, _ = _run(torch, "dd", A, B, N, algo="crt_bf16")
    want_all, _ = _run(torch, "dd", A, B, N)
    assert_bitwise(C, want_all, "tcgen05 vs int8")
    rows, cols = [0, 127, 128, 511, 512, 529], [0, 127, 128, 299]
    want, _, _, _ = R.gemm(A, B, N, rows=rows, cols=cols)
    assert_bitwise(C[:, rows][:, :, cols], want, "tcgen05 vs oracle")


# ---------------------------------------------------------------- split integers

SPLIT_ENGINES = ["crt2", "crt2_bf16"]


def _run2(torch, prec, A, B, N, trans_a=False, trans_b=False, algo="crt2"):
    from paper_2101_06584_gb300 import mpgemm as mm
    Ad = dev(torch, A.transpose(0, 2, 1) if trans_a else A)
    Bd = dev(torch, B.transpose(0, 2, 1) if trans_b else B)
    m, k = A.shape[1], A.shape[2]
    n = B.shape[2]
    ws = torch.empty(mm.workspace_size(prec, m, n, k, algo=algo, slices=N), dtype=torch.uint8, device="cuda")
    C = mm.gemm(prec, Ad, Bd, trans_a=trans_a, trans_b=trans_b, algo=algo, slices=N, workspace=ws)
    if algo.endswith("bf16"):
        assert mm.tc_status(ws) == 0, "tcgen05 kernel reported a timeout"
    return host(C), host(ws)


def _split_residues(planes, N, beta):
    """Exponents and the residues [2N][r][k] of the halves (A1's, then A0's)."""
    sig, rows = R.integer_rows(planes, beta)
    w = beta // 2
    hi = [[R.split(a, w)[0] for a in row] for row in rows]
    lo = [[R.split(a, w)[1] for a in row] for row in rows]
    return sig, np.concatenate([R._res(hi, N), R._res(lo, N)])


@pytest.mark.parametrize("prec,N", [("dd", 3), ("td", 20), ("qd", 30), ("qd", 44)])
def test_split_residues_and_result_bitwise(torch, prec, N):
    """Both operands' 2N residue planes in the workspace equal the oracle's
    (A1's then A0's), and the results of both engines are bit-identical to
    the oracle's split-integer steps."""
    from paper_2101_06584_gb300 import mpgemm as mm
    P = I.P_OF[prec]
    rng = np.random.default_rng(870 + P + N)
    m, n, k = 37, 45, 53
    A, B = I.uniform(P, (m, k), rng), I.ill_scaled(P, (k, n), rng)
    C, ws = _run2(torch, prec, A, B, N)
    beta = R.beta_bits(N, k, halves=2)
    assert mm.crt_beta(N, k, split=True) == beta
    mp, np_, kp = 128, 128, 128
    offB = 2 * N * mp * kp
    offSig = offB + 2 * N * np_ * kp
    offTau = offSig + 512
    sig, RA = _split_residues(A, N, beta)
    tau, RB = _split_residues(np.ascontiguousarray(B.transpose(0, 2, 1)), N, beta)
    ga = ws[:2 * N * mp * kp].view(np.int8).reshape(2 * N, mp, kp)
    gb = ws[offB:offB + 2 * N * np_ * kp].view(np.int8).reshape(2 * N, np_, kp)
    assert (ws[offSig:offSig + 4 * m].view(np.int32) == sig).all()
    assert (ws[offTau:offTau + 4 * n].view(np.int32) == tau).all()
    assert (ga[:, :m, :k] == RA).all() and not ga[:, m:, :].any() and not ga[:, :, k:].any()
    assert (gb[:, :n, :k] == RB).all() and not gb[:, n:, :].any() and not gb[:, :, k:].any()
    want, _, _, _ = R.gemm(A, B, N, halves=2)
    assert_bitwise(C, want, "%s split N=%d" % (prec, N))
    Ct, _ = _run2(torch, prec, A, B, N, algo="crt2_bf16")
    assert_bitwise(Ct, want, "%s split on tcgen05 N=%d" % (prec, N))


@pytest.mark.parametrize("algo", SPLIT_ENGINES)
def test_split_transposes_tiles_and_cancellation(torch, algo):
    """QD, several 128 x 128 tiles with ragged edges, every transpose,
    cancelling ill-scaled operands, k over several drains of the tcgen05
    accumulators (the middle product's two sub-products in one sum)."""
    rng = np.random.default_rng(880)
    A, B = I.cancelling_pair(4, 150, 270, 2300, rng)
    N = 30
    rows, cols = [0, 77, 127, 128, 149], [0, 100, 127, 128, 255, 256, 269]
    want, _, _, _ = R.gemm(A, B, N, rows=rows, cols=cols, halves=2)
    first = None
    for ta, tb in ((False, False), (True, False), (False, True), (True, True)):
        C, _ = _run2(torch, "qd", A, B, N, trans_a=ta, trans_b=tb, algo=algo)
        assert_bitwise(C[:, rows][:, :, cols], want, "qd %s trans %s %s" % (algo, ta, tb))
        if first is None:
            first = C
        assert_bitwise(C, first, "qd %s transposes agree" % algo)


@pytest.mark.parametrize("algo", SPLIT_ENGINES)
def test_split_products_below_the_normal_range(torch, algo):
    """Rows of A scaled by 1 .. 2^-1060 and columns of B by 1 .. 2^-530 with
    split integers: components through the subnormal range and down to signed
    zeros, every entry bit-identical to the oracle."""
    rng = np.random.default_rng(890)
    m, n, k = 40, 36, 64
    A, B = I.uniform(4, (m, k), rng), I.uniform(4, (k, n), rng)
    A *= np.array([1.0, 2.0 ** -500, 2.0 ** -530, 2.0 ** -1060])[np.arange(m) % 4][None, :, None]
    B *= np.array([1.0, 2.0 ** -500, 2.0 ** -530])[(np.arange(n) // 2) % 3][None, None, :]
    C, _ = _run2(torch, "qd", A, B, 36, algo=algo)
    want, _, _, _ = R.gemm(A, B, 36, halves=2)
    assert ((np.abs(want) < 2.0 ** -1022) & (want != 0)).any() and np.isfinite(want).all()
    assert_bitwise(C, want, "qd split tiny products")


def test_split_largest_k_and_refusal(torch):
    """k = 65535, the largest whose middle products sum exactly in int32:
    sampled entries bit-identical to the oracle on both engines; k + 1 is
    refused."""
    from paper_2101_06584_gb300 import mpgemm as mm
    k = R.k_limit(2)
    m = n = 16
    rng = np.random.default_rng(900)
    A, B = I.uniform(2, (m, k), rng), I.uniform(2, (k, n), rng)
    C, _ = _run2(torch, "dd", A, B, 10)
    want, _, _, _ = R.gemm(A, B, 10, rows=[0, 15], cols=[3, 9], halves=2)
    assert_bitwise(C[:, [0, 15]][:, :, [3, 9]], want, "split at the largest k")
    Ct, _ = _run2(torch, "dd", A, B, 10, algo="crt2_bf16")
    assert_bitwise(Ct, C, "both engines at the largest k")
    A1 = np.concatenate([A, np.zeros((2, m, 1))], axis=2)
    B1 = np.concatenate([B, np.zeros((2, 1, n))], axis=1)
    with pytest.raises(mm.MPGError) as e:
        mm.gemm("dd", dev(torch, A1), dev(torch, B1), algo="crt2", slices=10,
                workspace=torch.empty(1 << 20, dtype=torch.uint8, device="cuda"))
    assert e.value.code == -4


@pytest.mark.parametrize("N", [30])
def test_split_full_size_qd(torch, N):
    """QD 1024^3 on the inputs of the TD/QD workload (cancelling pairs): the
    tcgen05 engine equals the int8 engine on every entry, a 16 x 16 grid is
    bit-identical to the oracle, and two whole rows with the grid are within
    n 2^-200 of the exact product."""
    from paper_2101_06584_gb300 import mpgemm as mm
    n = 1024
    rng = I.rng_for(1)
    I.cancelling_pair(3, n, n, n, rng)
    A, B = I.cancelling_pair(4, n, n, n, rng)
    Ad, Bd = dev(torch, A), dev(torch, B)
    out = {}
    for algo in SPLIT_ENGINES:
        ws = torch.empty(mm.workspace_size("qd", n, n, n, algo=algo, slices=N), dtype=torch.uint8, device="cuda")
        out[algo] = mm.gemm("qd", Ad, Bd, algo=algo, slices=N, workspace=ws)
        if algo == "crt2_bf16":
            assert mm.tc_status(ws) == 0
        del ws
    diff = int((out["crt2"].view(torch.int64) != out["crt2_bf16"].view(torch.int64)).sum())
    assert diff == 0, "%d values differ between the engines" % diff
    C = host(out["crt2_bf16"])
    srng = np.random.default_rng(910)
    rows = sorted(int(x) for x in srng.choice(n, 16, replace=False))
    cols = sorted(int(x) for x in srng.choice(n, 16, replace=False))
    want, _, _, _ = R.gemm(A, B, N, rows=rows, cols=cols, halves=2)
    assert_bitwise(C[:, rows][:, :, cols], want, "split qd 1024 grid")
    full = sorted(int(x) for x in srng.choice(n, 2, replace=False))
    ent = sorted({(i, j) for i in full for j in range(n)} | {(i, j) for i in rows for j in cols})
    err = X.gemm_error(C, A, B, ent)
    assert err["err_abs"] <= n * 2.0 ** -200, err
