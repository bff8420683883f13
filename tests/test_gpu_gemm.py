"""GEMM on the GPU against the oracle.

The k-sequential FP64-EFT kernel is bit-identical to the oracle's Eq. 1 loop
for every tile configuration, both transposes, ragged shapes spanning several
tiles, the cancelling ill-scaled inputs and the paper's Sec. 3 matrices, and
on sampled rows at the full sizes of the TD/QD 1024^3 and DD 4096^3 workloads
in the launch configuration the benchmark times.  The split-K kernel is within
the normwise bound k 2^-p of the exact product."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_bitwise, dev, host, torch_cuda
from oracle import exact as X
from paper_2101_06584_gb300 import inputs as I

pytestmark = pytest.mark.gpu
PBITS = {"dd": 100, "td": 150, "qd": 200}


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def _mm():
    from paper_2101_06584_gb300 import mpgemm
    return mpgemm


SHAPES = [(1, 1, 1), (37, 45, 53), (64, 64, 64), (70, 33, 129), (5, 130, 17)]


@pytest.mark.parametrize("prec", ["dd", "td", "qd"])
def test_kseq_bitwise_all_tiles(torch, prec):
    mm = _mm()
    P = I.P_OF[prec]
    rng = np.random.default_rng(400 + P)
    for (m, n, k) in SHAPES:
        A = I.uniform(P, (m, k), rng)
        B = I.uniform(P, (k, n), rng)
        want = oracle.gemm(prec, A, B, nthreads=4)
        Ad, Bd = dev(torch, A), dev(torch, B)
        assert_bitwise(host(mm.gemm_plain(prec, Ad, Bd)), want, "%s %s plain" % (prec, (m, n, k)))
        for tile in range(1, mm.num_tiles(prec) + 1):
            C = mm.gemm(prec, Ad, Bd, tile=tile)
            assert_bitwise(host(C), want, "%s %s tile %d" % (prec, (m, n, k), tile))


@pytest.mark.parametrize("prec", ["dd", "td", "qd"])
def test_kseq_transposes(torch, prec):
    mm = _mm()
    P = I.P_OF[prec]
    rng = np.random.default_rng(410 + P)
    m, n, k = 33, 47, 61
    A = I.uniform(P, (m, k), rng)
    B = I.uniform(P, (k, n), rng)
    want = oracle.gemm(prec, A, B, nthreads=4)
    At = dev(torch, A.transpose(0, 2, 1))
    Bt = dev(torch, B.transpose(0, 2, 1))
    assert_bitwise(host(mm.gemm(prec, At, dev(torch, B), trans_a=True)), want, "A^T")
    assert_bitwise(host(mm.gemm(prec, dev(torch, A), Bt, trans_b=True)), want, "B^T")
    assert_bitwise(host(mm.gemm(prec, At, Bt, trans_a=True, trans_b=True)), want, "A^T B^T")


@pytest.mark.parametrize("prec", ["dd", "td", "qd"])
def test_kseq_cancelling_and_paper(torch, prec):
    mm = _mm()
    P = I.P_OF[prec]
    rng = np.random.default_rng(420 + P)
    A, B = I.cancelling_pair(P, 40, 36, 96, rng)
    want = oracle.gemm(prec, A, B, nthreads=4)
    assert_bitwise(host(mm.gemm_plain(prec, dev(torch, A), dev(torch, B))), want, "cancelling")
    A, B = I.paper_matrices(P, 65)
    want = oracle.gemm(prec, A, B, nthreads=4)
    assert_bitwise(host(mm.gemm_plain(prec, dev(torch, A), dev(torch, B))), want, "paper")


def test_k_zero_and_empty(torch):
    mm = _mm()
    A = torch.empty((2, 5, 0), dtype=torch.float64, device="cuda")
    B = torch.empty((2, 0, 7), dtype=torch.float64, device="cuda")
    C = torch.full((2, 5, 7), 3.0, dtype=torch.float64, device="cuda")
    mm.gemm("dd", A, B, out=C)
    assert (host(C) == 0).all()
    A = torch.empty((3, 0, 4), dtype=torch.float64, device="cuda")
    B = torch.zeros((3, 4, 6), dtype=torch.float64, device="cuda")
    assert mm.gemm("td", A, B).shape == (3, 0, 6)


def test_leading_dimension_views(torch):
    """Planes that are column slices of wider matrices (ld > cols)."""
    mm = _mm()
    rng = np.random.default_rng(430)
    A = I.uniform(2, (30, 50), rng)
    B = I.uniform(2, (40, 60), rng)
    want = oracle.gemm("dd", np.ascontiguousarray(A[:, :, :40]), np.ascontiguousarray(B[:, :, :25]))
    Ad, Bd = dev(torch, A), dev(torch, B)
    C = torch.zeros((2, 30, 64), dtype=torch.float64, device="cuda")
    mm.gemm("dd", Ad[:, :, :40], Bd[:, :, :25], out=C[:, :, :25])
    assert_bitwise(host(C[:, :, :25]), want, "ld views")
    assert (host(C[:, :, 25:]) == 0).all()


@pytest.mark.parametrize("prec", ["dd", "td", "qd"])
@pytest.mark.parametrize("split", [2, 8, 32])
def test_splitk_within_bound(torch, prec, split):
    mm = _mm()
    P = I.P_OF[prec]
    rng = np.random.default_rng(440 + P + split)
    m, n, k = 9, 11, 203
    for A, B in ((I.uniform(P, (m, k), rng), I.uniform(P, (k, n), rng)),
                 I.cancelling_pair(P, m, n, k, rng)):
        C1 = host(mm.gemm(prec, dev(torch, A), dev(torch, B), split_k=split))
        C2 = host(mm.gemm(prec, dev(torch, A), dev(torch, B), split_k=split))
        assert_bitwise(C1, C2, "split-k deterministic")
        ent = [(i, j) for i in range(m) for j in range(n)]
        err = X.gemm_error(C1, A, B, ent)
        assert err["err_abs"] <= k * 2.0 ** -PBITS[prec], err


def test_full_size_main_workload_sampled(torch):
    """The main workload at its full size and launch configuration: TD then QD
    at m = n = k = 1024 on the cancelling ill-scaled inputs of its seed (the
    same generator, in the same order, as the benchmark), through the plain
    entry points with the library's default tile (16 x 16).  Eight sampled
    rows of each product, all 1024 columns, are bit-identical to the oracle's
    Eq. 1 loop."""
    mm = _mm()
    n = 1024
    rng = I.rng_for(1)
    srng = np.random.default_rng(450)
    for prec in ("td", "qd"):
        P = I.P_OF[prec]
        A, B = I.cancelling_pair(P, n, n, n, rng)
        ti = mm.tile_info(prec, mm.default_tile(prec, n, n, n))
        assert (ti["bm"], ti["bn"]) == (16, 16)
        C = host(mm.gemm_plain(prec, dev(torch, A), dev(torch, B)))
        rows = sorted({0, n - 1} | set(int(r) for r in srng.integers(0, n, 6)))
        want = oracle.gemm(prec, np.ascontiguousarray(A[:, rows, :]), B, nthreads=8)
        assert_bitwise(C[:, rows, :], want, "%s %d sampled rows" % (prec, n))


def test_full_size_dd_4096_sampled(torch):
    """DD at m = n = k = 4096 on the uniform inputs of that workload's seed (the
    plain product the benchmark times beside the slicing forms): three sampled
    rows, all 4096 columns, bit-identical to the oracle."""
    mm = _mm()
    n = 4096
    rng = I.rng_for(2)
    A = I.uniform(2, (n, n), rng)
    B = I.uniform(2, (n, n), rng)
    C = host(mm.gemm_plain("dd", dev(torch, A), dev(torch, B)))
    rows = [0, 2047, n - 1]
    want = oracle.gemm("dd", np.ascontiguousarray(A[:, rows, :]), B, nthreads=8)
    assert_bitwise(C[:, rows, :], want, "dd 4096 sampled rows")


@pytest.mark.parametrize("prec", ["dd", "td", "qd"])
def test_kseq_subnormal_products(torch, prec):
    """Rows of A and columns of B scaled so that products and partial sums
    fall into and below the subnormal range (IEEE gradual underflow on both
    sides): bit-identical to the oracle for every tile."""
    mm = _mm()
    P = I.P_OF[prec]
    rng = np.random.default_rng(460 + P)
    m, n, k = 24, 20, 40
    A, B = I.uniform(P, (m, k), rng), I.uniform(P, (k, n), rng)
    A *= np.array([1.0, 2.0 ** -530, 2.0 ** -560, 2.0 ** -1060])[np.arange(m) % 4][None, :, None]
    B *= np.array([1.0, 2.0 ** -520])[np.arange(n) % 2][None, None, :]
    want = oracle.gemm(prec, A, B, nthreads=4)
    assert ((np.abs(want[0]) < 2.0 ** -1022) & (want[0] != 0)).any()
    Ad, Bd = dev(torch, A), dev(torch, B)
    for tile in range(1, mm.num_tiles(prec) + 1):
        assert_bitwise(host(mm.gemm(prec, Ad, Bd, tile=tile)), want, "%s subnormal tile %d" % (prec, tile))
