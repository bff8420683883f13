"""The INT8 error-free slicing form on the GPU against its oracle: the
slices and exponents in the workspace are bit-identical to the definition,
the DD result is bit-identical to the oracle's steps (small shapes, both
transposes, ragged tiles), and at the full 4096^3 size the sampled entries
are bit-identical and within n 2^-100 of the exact product."""
import numpy as np
import pytest

from gpu_util import assert_bitwise, dev, host, torch_cuda
from oracle import exact as X
from oracle import ozaki as OZ
from paper_2101_06584_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def _run(torch, A, B, S, trans_a=False, trans_b=False):
    from paper_2101_06584_gb300 import mpgemm as mm
    Ad = dev(torch, A.transpose(0, 2, 1) if trans_a else A)
    Bd = dev(torch, B.transpose(0, 2, 1) if trans_b else B)
    m, k = A.shape[1], A.shape[2]
    n = B.shape[2]
    nbytes = mm.workspace_size("dd", m, n, k, algo="int8", slices=S)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    C = mm.gemm("dd", Ad, Bd, trans_a=trans_a, trans_b=trans_b, algo="int8", slices=S, workspace=ws)
    return host(C), host(ws)


def _layout(S, m, n, k):
    r = lambda x, q: (max(x, 1) + q - 1) // q * q
    mp, np_, kp = r(m, 64), r(n, 64), r(k, 128)
    offB = r(S * mp * kp, 256)
    offSig = offB + r(S * np_ * kp, 256)
    offTau = offSig + r(mp * 4, 256)
    return mp, np_, kp, offB, offSig, offTau


@pytest.mark.parametrize("S", [1, 5, 14, 16])
def test_slices_and_result_bitwise(torch, S):
    rng = np.random.default_rng(600 + S)
    m, n, k = 37, 45, 53
    A, B = I.uniform(2, (m, k), rng), I.ill_scaled(2, (k, n), rng)
    C, ws = _run(torch, A, B, S)
    mp, np_, kp, offB, offSig, offTau = _layout(S, m, n, k)
    sig, DA = OZ.slice_rows(A, S)
    tau, DB = OZ.slice_cols(B, S)
    gsa = ws[:S * mp * kp].view(np.int8).reshape(S, mp, kp)
    gsb = ws[offB:offB + S * np_ * kp].view(np.int8).reshape(S, np_, kp)
    gsig = ws[offSig:offSig + 4 * mp].view(np.int32)
    gtau = ws[offTau:offTau + 4 * np_].view(np.int32)
    assert (gsig[:m] == sig).all() and (gsig[m:] == 0).all()
    assert (gtau[:n] == tau).all() and (gtau[n:] == 0).all()
    assert (gsa[:, :m, :k] == DA).all() and not gsa[:, m:, :].any() and not gsa[:, :, k:].any()
    assert (gsb[:, :n, :k] == DB).all() and not gsb[:, n:, :].any() and not gsb[:, :, k:].any()
    want, _, _ = OZ.gemm(A, B, S)
    assert_bitwise(C, want, "int8 S=%d" % S)


def test_transposes_and_cancellation(torch):
    rng = np.random.default_rng(610)
    A, B = I.cancelling_pair(2, 70, 66, 130, rng)
    want, _, _ = OZ.gemm(A, B, 9)
    for ta, tb in ((False, True), (True, False), (True, True)):
        C, _ = _run(torch, A, B, 9, trans_a=ta, trans_b=tb)
        assert_bitwise(C, want, "int8 trans %s %s" % (ta, tb))


def test_workspace_errors(torch):
    from paper_2101_06584_gb300 import mpgemm as mm
    A = torch.zeros((2, 8, 8), dtype=torch.float64, device="cuda")
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(mm.MPGError) as e:
        mm.gemm("dd", A, A, algo="int8", slices=4, workspace=small)
    assert e.value.code == -3
    with pytest.raises(mm.MPGError) as e:
        mm.gemm("dd", A, A, algo="int8", slices=4)
    assert e.value.code == -3
    Q = torch.zeros((4, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(mm.MPGError) as e:
        mm.gemm("qd", Q, Q, algo="int8")                  # supported, but needs a workspace
    assert e.value.code == -3
    with pytest.raises(mm.MPGError) as e:
        mm.gemm("qd", Q, Q, algo="bf16")                  # the tcgen05 path needs one too
    assert e.value.code == -3


def test_tile_variants_agree(torch):
    """Both CTA tilings of the slice-product kernel give the same bits."""
    from paper_2101_06584_gb300 import mpgemm as mm
    rng = np.random.default_rng(630)
    m, n, k = 150, 97, 200
    A, B = I.ill_scaled(2, (m, k), rng), I.uniform(2, (k, n), rng)
    Ad, Bd = dev(torch, A), dev(torch, B)
    ws = torch.empty(mm.workspace_size("dd", m, n, k, algo="int8", slices=11), dtype=torch.uint8,
                     device="cuda")
    C1 = host(mm.gemm("dd", Ad, Bd, algo="int8", slices=11, workspace=ws, tile=1))
    for tile in (2, 3):
        C2 = host(mm.gemm("dd", Ad, Bd, algo="int8", slices=11, workspace=ws, tile=tile))
        assert_bitwise(C1, C2, "tile variant %d" % tile)
    want, _, _ = OZ.gemm(A, B, 11)
    assert_bitwise(C1, want, "int8 vs oracle")


def test_bf16_path_matches_int8(torch):
    """The bf16 digits on tcgen05 (TMEM accumulators) compute the same integer
    weight sums: the result equals the int8 path's and the oracle's bit for
    bit (ragged shape, ill-scaled operands, transposed B)."""
    from paper_2101_06584_gb300 import mpgemm as mm
    rng = np.random.default_rng(640)
    m, n, k = 131, 70, 300
    A, B = I.ill_scaled(2, (m, k), rng), I.uniform(2, (k, n), rng)
    Ad, Bt = dev(torch, A), dev(torch, B.transpose(0, 2, 1))
    S = 12
    ws = torch.empty(mm.workspace_size("dd", m, n, k, algo="bf16", slices=S), dtype=torch.uint8,
                     device="cuda")
    Cb = host(mm.gemm("dd", Ad, Bt, trans_b=True, algo="bf16", slices=S, workspace=ws))
    assert host(ws[:4]).view(np.int32)[0] == 0, "tcgen05 kernel reported a timeout"
    ws8 = torch.empty(mm.workspace_size("dd", m, n, k, algo="int8", slices=S), dtype=torch.uint8,
                      device="cuda")
    Ci = host(mm.gemm("dd", Ad, Bt, trans_b=True, algo="int8", slices=S, workspace=ws8))
    assert_bitwise(Cb, Ci, "bf16 vs int8")
    want, _, _ = OZ.gemm(A, B, S)
    assert_bitwise(Cb, want, "bf16 vs oracle")


def test_bf16_partial_sums_at_the_drain_limit(torch):
    """Constant operands whose first digits are all 64: the (1, 1) slice pair
    sums 64 * 64 over 2048 values of k, exactly 2^23, between drains of the
    fp32 fragments; the result must still be the exact integer sums."""
    from paper_2101_06584_gb300 import mpgemm as mm
    m, n, k = 64, 32, 4096
    A = np.zeros((2, m, k))
    B = np.zeros((2, k, n))
    # a = (1 - 2^-20) / 2: sigma = ilogb(a) + 2 = 0, a 2^-sigma 2^7 = 64 (1 - 2^-20) -> digit 64
    A[0] = 2.0 ** -1 * (1 - 2.0 ** -20)
    B[0] = 2.0 ** -1 * (1 - 2.0 ** -20)
    S = 4
    sig, DA = OZ.slice_rows(A[:, :1, :8], S)
    assert DA[0, 0, 0] == 64                       # first digit at its maximum
    Ad, Bd = dev(torch, A), dev(torch, B)
    ws = torch.empty(mm.workspace_size("dd", m, n, k, algo="bf16", slices=S), dtype=torch.uint8,
                     device="cuda")
    Cb = host(mm.gemm("dd", Ad, Bd, algo="bf16", slices=S, workspace=ws))
    assert host(ws[:4]).view(np.int32)[0] == 0, "tcgen05 kernel reported a timeout"
    ws8 = torch.empty(mm.workspace_size("dd", m, n, k, algo="int8", slices=S), dtype=torch.uint8,
                      device="cuda")
    Ci = host(mm.gemm("dd", Ad, Bd, algo="int8", slices=S, workspace=ws8))
    assert_bitwise(Cb, Ci, "bf16 vs int8 at the limit")
    want, _, _ = OZ.gemm(A, B, S, rows=[0, 63], cols=[0, 31])
    assert_bitwise(Cb[:, [0, 63]][:, :, [0, 31]], want, "bf16 vs oracle at the limit")


def test_bf16_long_ragged_k(torch):
    """k = 2500 (segments of 2048 and of the rest for each pair, zero-padded
    last stage), three weight groups (S = 12), ragged m and n on the CTA-pair
    engine: equal to the int8 engine everywhere and to the oracle on sampled
    entries."""
    from paper_2101_06584_gb300 import mpgemm as mm
    rng = np.random.default_rng(660)
    m, n, k, S = 300, 200, 2500, 12
    A, B = I.ill_scaled(2, (m, k), rng), I.uniform(2, (k, n), rng)
    Ad, Bd = dev(torch, A), dev(torch, B)
    wsb = torch.empty(mm.workspace_size("dd", m, n, k, algo="bf16", slices=S), dtype=torch.uint8, device="cuda")
    Cb = host(mm.gemm("dd", Ad, Bd, algo="bf16", slices=S, workspace=wsb))
    assert host(wsb[:4]).view(np.int32)[0] == 0, "tcgen05 kernel reported a timeout"
    ws8 = torch.empty(mm.workspace_size("dd", m, n, k, algo="int8", slices=S), dtype=torch.uint8, device="cuda")
    Ci = host(mm.gemm("dd", Ad, Bd, algo="int8", slices=S, workspace=ws8))
    assert_bitwise(Cb, Ci, "bf16 vs int8, long k")
    rows, cols = [0, 131, 299], [0, 127, 128, 199]
    want, _, _ = OZ.gemm(A, B, S, rows=rows, cols=cols)
    assert_bitwise(Cb[:, rows][:, :, cols], want, "bf16 vs oracle, long k")


@pytest.mark.parametrize("prec,S", [("td", 1), ("td", 22), ("td", 40), ("qd", 5), ("qd", 29), ("qd", 40)])
def test_td_qd_bitwise(torch, prec, S):
    """TD/QD slicing forms: the result is bit-identical to the oracle's steps
    (ragged shape, ill-scaled A, transposed B), and the workspace slices match
    the oracle's digits."""
    from paper_2101_06584_gb300 import mpgemm as mm
    P = I.P_OF[prec]
    rng = np.random.default_rng(660 + P + S)
    m, n, k = 37, 21, 150
    A, B = I.ill_scaled(P, (m, k), rng), I.uniform(P, (k, n), rng)
    Ad, Bt = dev(torch, A), dev(torch, B.transpose(0, 2, 1))
    ws = torch.empty(mm.workspace_size(prec, m, n, k, algo="int8", slices=S), dtype=torch.uint8,
                     device="cuda")
    C = host(mm.gemm(prec, Ad, Bt, trans_b=True, algo="int8", slices=S, workspace=ws))
    want, sig, tau = OZ.gemm(A, B, S)
    assert_bitwise(C, want, "%s int8 S=%d" % (prec, S))
    w = host(ws)
    mp, np_, kp, offB, offSig, offTau = _layout(S, m, n, k)
    _, DA = OZ.slice_rows(A, S)
    gsa = w[:S * mp * kp].view(np.int8).reshape(S, mp, kp)
    assert (gsa[:, :m, :k] == DA).all()
    assert (w[offSig:offSig + 4 * m].view(np.int32) == sig).all()


@pytest.mark.parametrize("prec,S", [("td", 22), ("qd", 29), ("dd", 3)])
def test_tc_engine_matches_int8(torch, prec, S):
    """TD/QD (and a 3-slice DD) on the tcgen05 engine equal the int8 engine and
    the oracle bit for bit; several output tiles, ragged edges, both
    transposes."""
    from paper_2101_06584_gb300 import mpgemm as mm
    P = I.P_OF[prec]
    rng = np.random.default_rng(680 + P)
    m, n, k = 200, 150, 190
    A, B = I.ill_scaled(P, (m, k), rng), I.uniform(P, (k, n), rng)
    At, Bt = dev(torch, A.transpose(0, 2, 1)), dev(torch, B.transpose(0, 2, 1))
    wsb = torch.empty(mm.workspace_size(prec, m, n, k, algo="bf16", slices=S), dtype=torch.uint8,
                      device="cuda")
    wsi = torch.empty(mm.workspace_size(prec, m, n, k, algo="int8", slices=S), dtype=torch.uint8,
                      device="cuda")
    Cb = host(mm.gemm(prec, At, Bt, trans_a=True, trans_b=True, algo="bf16", slices=S, workspace=wsb))
    assert host(wsb[:4]).view(np.int32)[0] == 0, "tcgen05 kernel reported a timeout"
    Ci = host(mm.gemm(prec, At, Bt, trans_a=True, trans_b=True, algo="int8", slices=S, workspace=wsi))
    assert_bitwise(Cb, Ci, "%s tcgen05 vs int8" % prec)
    want, _, _ = OZ.gemm(A, B, S, rows=[0, 127, 128, 199], cols=[0, 127, 128, 149])
    assert_bitwise(Cb[:, [0, 127, 128, 199]][:, :, [0, 127, 128, 149]], want, "%s tcgen05 vs oracle" % prec)


def test_largest_exact_k(torch):
    """DD at the largest k the slicing form accepts with 14 slices,
    (2^31 - 1) // (14 * 4096) = 37449 (every int32 weight sum exact): both
    engines agree on all 64 x 64 entries, and four sampled entries are
    bit-identical to the oracle's steps; k + 1 is refused."""
    from paper_2101_06584_gb300 import mpgemm as mm
    S = 14
    k = OZ.k_limit(S)
    assert k == (2 ** 31 - 1) // (S * 4096)
    m = n = 64
    rng = np.random.default_rng(690)
    A, B = I.uniform(2, (m, k), rng), I.uniform(2, (k, n), rng)
    Ad, Bd = dev(torch, A), dev(torch, B)
    out = {}
    for algo in ("int8", "bf16"):
        ws = torch.empty(mm.workspace_size("dd", m, n, k, algo=algo, slices=S), dtype=torch.uint8,
                         device="cuda")
        out[algo] = host(mm.gemm("dd", Ad, Bd, algo=algo, slices=S, workspace=ws))
        if algo == "bf16":
            assert host(ws[:4]).view(np.int32)[0] == 0, "tcgen05 kernel reported a timeout"
    assert_bitwise(out["bf16"], out["int8"], "bf16 vs int8 at the largest k")
    rows, cols = [0, 40], [31, 63]
    want, _, _ = OZ.gemm(A, B, S, rows=rows, cols=cols)
    assert_bitwise(out["int8"][:, rows][:, :, cols], want, "largest k sampled")
    A1 = np.concatenate([A, np.zeros((2, m, 1))], axis=2)
    B1 = np.concatenate([B, np.zeros((2, 1, n))], axis=1)
    with pytest.raises(mm.MPGError):
        mm.gemm("dd", dev(torch, A1), dev(torch, B1), algo="int8", slices=S,
                workspace=torch.empty(1 << 20, dtype=torch.uint8, device="cuda"))


@pytest.mark.parametrize("algo", ["int8", "bf16"])
def test_slicing_form_in_a_cuda_graph(torch, algo):
    """A slicing-form call captured into a CUDA graph replays to the same bits
    as a direct call: the op(B) slicing runs on a second stream forked from
    the capturing stream and joined back to it, so it is captured too."""
    from paper_2101_06584_gb300 import mpgemm as mm
    rng = np.random.default_rng(695)
    m, n, k = 300, 200, 260
    A, B = I.uniform(2, (m, k), rng), I.uniform(2, (k, n), rng)
    Ad, Bd = dev(torch, A), dev(torch, B)
    ws = torch.empty(mm.workspace_size("dd", m, n, k, algo=algo), dtype=torch.uint8, device="cuda")
    want = host(mm.gemm("dd", Ad, Bd, algo=algo, workspace=ws))
    out = torch.empty((2, m, n), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):                       # a warm-up call on a side stream, outside the capture
        mm.gemm("dd", Ad, Bd, out=out, algo=algo, workspace=ws)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        mm.gemm("dd", Ad, Bd, out=out, algo=algo, workspace=ws)
    for _ in range(2):
        out.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert_bitwise(host(out), want, "%s graph replay" % algo)


@pytest.mark.parametrize("prec,S", [("dd", 14), ("qd", 29)])
@pytest.mark.parametrize("algo", ["int8", "bf16"])
def test_products_below_the_normal_range(torch, prec, S, algo):
    """Rows of A scaled by 1, 2^-500, 2^-530 or 2^-1060 (a subnormal leading
    component) and columns of B by 1, 2^-500 or 2^-530: outputs range from
    normal through 2^-1000 .. 2^-1060, where the group parts fall below the
    normal binary64 range and are rounded there (the first group then being
    added to zero instead of stored as it is), down to products that round
    to signed zeros.  Both engines are bit-identical to the oracle's steps on
    every entry."""
    from paper_2101_06584_gb300 import mpgemm as mm
    P = I.P_OF[prec]
    rng = np.random.default_rng(700 + P)
    m, n, k = 48, 40, 64
    A, B = I.uniform(P, (m, k), rng), I.uniform(P, (k, n), rng)
    rs = np.array([1.0, 2.0 ** -500, 2.0 ** -530, 2.0 ** -1060])[np.arange(m) % 4]
    cs = np.array([1.0, 2.0 ** -500, 2.0 ** -530])[(np.arange(n) // 2) % 3]
    A *= rs[None, :, None]
    B *= cs[None, None, :]
    ws = torch.empty(mm.workspace_size(prec, m, n, k, algo=algo, slices=S), dtype=torch.uint8, device="cuda")
    C = host(mm.gemm(prec, dev(torch, A), dev(torch, B), algo=algo, slices=S, workspace=ws))
    if algo == "bf16":
        assert host(ws[:4]).view(np.int32)[0] == 0, "tcgen05 kernel reported a timeout"
    want, _, _ = OZ.gemm(A, B, S)
    assert (np.abs(want[0]) < 2.0 ** -1022).sum() > 0 and np.isfinite(want).all()
    assert_bitwise(C, want, "%s %s tiny products" % (prec, algo))


def test_tc_status(torch):
    """The tcgen05 engine's status read through the C ABI: 0 after a normal
    call; a code planted in the workspace header on the host (the device-side
    timeout is not provoked) is returned with the role it names."""
    from paper_2101_06584_gb300 import mpgemm as mm
    rng = np.random.default_rng(710)
    A, B = I.uniform(2, (70, 90), rng), I.uniform(2, (90, 50), rng)
    ws = torch.empty(mm.workspace_size("dd", 70, 50, 90, algo="bf16"), dtype=torch.uint8, device="cuda")
    mm.gemm("dd", dev(torch, A), dev(torch, B), algo="bf16", workspace=ws)
    assert mm.tc_status(ws) == 0
    ws[:4].view(torch.int32).fill_(3)
    assert mm.tc_status(ws) == 3
    assert "loaded stage" in mm.lib().mpgemm_last_error().decode()
    mm.gemm("dd", dev(torch, A), dev(torch, B), algo="bf16", workspace=ws)
    assert mm.tc_status(ws) == 0                       # every call clears the header first


def _workload_inputs(prec, n):
    """The benchmark's inputs: DD from the 4096 workload's seed (uniform A
    then B); TD and QD from the main workload's seed, TD drawn first."""
    if prec == "dd":
        rng = I.rng_for(2)
        return I.uniform(2, (n, n), rng), I.uniform(2, (n, n), rng)
    rng = I.rng_for(1)
    pair = I.cancelling_pair(3, n, n, n, rng)
    return pair if prec == "td" else I.cancelling_pair(4, n, n, n, rng)


# the slice counts the benchmark chooses on these inputs (the smallest meeting n 2^-p)
@pytest.mark.parametrize("prec,n,S", [("dd", 4096, 13), ("td", 1024, 21), ("qd", 1024, 28)])
def test_full_size_both_engines(torch, prec, n, S):
    """The slicing form at the benchmark's full sizes and inputs, in its launch
    configuration, on both engines:
    - the tcgen05 engine (CTA pairs for DD) equals the int8 engine on every
      one of the n^2 entries, compared on the device;
    - a 16 x 16 grid of random rows and columns (256 entries) is bit-identical
      to the oracle's steps;
    - two whole rows and the grid are within n 2^-p of the exact product."""
    from paper_2101_06584_gb300 import mpgemm as mm
    P = I.P_OF[prec]
    A, B = _workload_inputs(prec, n)
    Ad, Bd = dev(torch, A), dev(torch, B)
    out = {}
    for algo in ("int8", "bf16"):
        ws = torch.empty(mm.workspace_size(prec, n, n, n, algo=algo, slices=S), dtype=torch.uint8, device="cuda")
        out[algo] = mm.gemm(prec, Ad, Bd, algo=algo, slices=S, workspace=ws)
        if algo == "bf16":
            assert mm.tc_status(ws) == 0, "tcgen05 kernel reported a timeout"
        del ws
    diff = int((out["int8"].view(torch.int64) != out["bf16"].view(torch.int64)).sum())
    assert diff == 0, "%d of %d values differ between the engines" % (diff, P * n * n)
    C = host(out["bf16"])
    srng = np.random.default_rng(620 + P)
    rows = sorted(int(x) for x in srng.choice(n, 16, replace=False))
    cols = sorted(int(x) for x in srng.choice(n, 16, replace=False))
    want, _, _ = OZ.gemm(A, B, S, rows=rows, cols=cols)
    assert_bitwise(C[:, rows][:, :, cols], want, "%s %d grid of 256 entries" % (prec, n))
    full = sorted(int(x) for x in srng.choice(n, 2, replace=False))
    ent = sorted({(i, j) for i in full for j in range(n)} | {(i, j) for i in rows for j in cols})
    err = X.gemm_error(C, A, B, ent)
    assert err["err_abs"] <= n * 2.0 ** -{"dd": 100, "td": 150, "qd": 200}[prec], err


@pytest.mark.parametrize("prec", ["dd", "td", "qd"])
def test_tc_abort_path(torch, prec):
    """The tcgen05 engines' abort path, run for real: with MPGEMM_TEST_TC_ABORT=1
    the producer gives up before issuing any load (as if its first bounded wait
    had run out), so every other role finds the abort flag with no load or MMA
    in flight.  The call returns at once, mpgemm_tc_status names the producer,
    and the next normal call on the same workspace is bit-identical to the int8
    engine (TMEM was released, the header is cleared)."""
    import os
    import time
    from paper_2101_06584_gb300 import mpgemm as mm
    P = I.P_OF[prec]
    rng = np.random.default_rng(720 + P)
    m, n, k = 300, 200, 260
    A, B = I.uniform(P, (m, k), rng), I.uniform(P, (k, n), rng)
    Ad, Bd = dev(torch, A), dev(torch, B)
    ws = torch.empty(mm.workspace_size(prec, m, n, k, algo="bf16"), dtype=torch.uint8, device="cuda")
    C = torch.zeros((P, m, n), dtype=torch.float64, device="cuda")
    os.environ["MPGEMM_TEST_TC_ABORT"] = "1"
    try:
        t0 = time.perf_counter()
        mm.gemm(prec, Ad, Bd, out=C, algo="bf16", workspace=ws)
        code = mm.tc_status(ws)
        elapsed = time.perf_counter() - t0
    finally:
        del os.environ["MPGEMM_TEST_TC_ABORT"]
    assert code == 1 and "producer" in mm.lib().mpgemm_last_error().decode()
    assert elapsed < 5.0, elapsed                     # no wait ran to its one-second limit
    got = mm.gemm(prec, Ad, Bd, algo="bf16", workspace=ws)
    assert mm.tc_status(ws) == 0
    ws8 = torch.empty(mm.workspace_size(prec, m, n, k, algo="int8"), dtype=torch.uint8, device="cuda")
    want = mm.gemm(prec, Ad, Bd, algo="int8", workspace=ws8)
    assert_bitwise(host(got), host(want), "%s after an aborted call" % prec)
