"""The binary64-only product (mpgemm_d, mpgemm_ex with P = 1) on the GPU
against the oracle's plain binary64 loop (Eq. 1 with one fma per term, k
increasing): bit-identical for every tile, both transposes, ragged shapes,
plane views of multi-component operands, products in the subnormal range, and
on two full rows plus sampled entries of the DD 4096^3 workload's leading
planes -- the FP64-only GEMM whose error the benchmark reports beside the DD,
TD and QD products."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_bitwise, dev, host, torch_cuda
from paper_2101_06584_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def _mm():
    from paper_2101_06584_gb300 import mpgemm
    return mpgemm


SHAPES = [(1, 1, 1), (37, 45, 53), (64, 64, 64), (70, 33, 129), (5, 130, 17), (130, 67, 300)]


def test_fp64_bitwise_all_tiles(torch):
    mm = _mm()
    rng = np.random.default_rng(600)
    for (m, n, k) in SHAPES:
        A = rng.uniform(-1, 1, (m, k)) * np.ldexp(1.0, rng.integers(-20, 20, (m, k)))
        B = rng.uniform(-1, 1, (k, n))
        want = oracle.dgemm(A, B, nthreads=4)
        Ad, Bd = dev(torch, A), dev(torch, B)
        assert_bitwise(host(mm.gemm_fp64(Ad, Bd)), want, "%s plain" % ((m, n, k),))
        for tile in range(1, mm.num_tiles("d") + 1):
            assert_bitwise(host(mm.gemm_fp64(Ad, Bd, tile=tile)), want, "%s tile %d" % ((m, n, k), tile))


def test_fp64_transposes_and_plane_views(torch):
    """op(A) op(B) with stored transposes, and the leading planes of DD
    operands passed as strided views (the FP64-only GEMM of a DD product)."""
    mm = _mm()
    rng = np.random.default_rng(601)
    m, n, k = 33, 47, 61
    A = I.uniform(2, (m, k), rng)
    B = I.uniform(2, (k, n), rng)
    want = oracle.dgemm(A[0], B[0], nthreads=4)
    Ad, Bd = dev(torch, A), dev(torch, B)
    assert_bitwise(host(mm.gemm_fp64(Ad[0], Bd[0])), want, "plane views")
    At, Bt = dev(torch, A[0].T), dev(torch, B[0].T)
    for ta, tb in ((1, 0), (0, 1), (1, 1)):
        C = mm.gemm_fp64(At if ta else Ad[0], Bt if tb else Bd[0], trans_a=bool(ta), trans_b=bool(tb))
        assert_bitwise(host(C), want, "trans %d%d" % (ta, tb))
    wide = torch.zeros((m, n + 9), dtype=torch.float64, device="cuda")
    mm.gemm_fp64(Ad[0], Bd[0], out=wide[:, :n])
    assert_bitwise(host(wide[:, :n]), want, "ld view of C")
    assert (host(wide[:, n:]) == 0).all()


def test_fp64_worked_and_edge_cases(torch):
    """The fused accumulation in increasing k ([a, a] . [a, -a] = -2^-60 for
    a = 1 + 2^-30), k = 0 (C set to zero) and products below the normal
    range."""
    mm = _mm()
    x = 1.0 + 2.0 ** -30
    C = host(mm.gemm_fp64(dev(torch, np.array([[x, x]])), dev(torch, np.array([[x], [-x]]))))
    assert C[0, 0] == -(2.0 ** -60)
    C = torch.full((3, 4), 7.0, dtype=torch.float64, device="cuda")
    mm.gemm_fp64(torch.empty((3, 0), dtype=torch.float64, device="cuda"),
                 torch.empty((0, 4), dtype=torch.float64, device="cuda"), out=C)
    assert (host(C) == 0).all()
    rng = np.random.default_rng(602)
    A = rng.uniform(-1, 1, (24, 40)) * np.ldexp(1.0, -540)
    B = rng.uniform(-1, 1, (40, 20)) * np.ldexp(1.0, -500)
    want = oracle.dgemm(A, B)
    assert ((np.abs(want) < 2.0 ** -1022) & (want != 0)).any()
    for tile in range(1, mm.num_tiles("d") + 1):
        assert_bitwise(host(mm.gemm_fp64(dev(torch, A), dev(torch, B), tile=tile)), want, "subnormal %d" % tile)


def test_fp64_full_size_sampled(torch):
    """The leading planes of the DD 4096^3 workload (its seed and generator
    order), through mpgemm_d with the library's default tile: two full rows
    and 256 sampled entries bit-identical to the oracle."""
    mm = _mm()
    n = 4096
    rng = I.rng_for(2)
    A = I.uniform(2, (n, n), rng)
    B = I.uniform(2, (n, n), rng)
    C = host(mm.gemm_fp64(dev(torch, A[0]), dev(torch, B[0])))
    srng = np.random.default_rng(603)
    rows = [int(r) for r in srng.choice(n, 2, replace=False)]
    want = oracle.dgemm(np.ascontiguousarray(A[0, rows, :]), B[0], nthreads=8)
    assert_bitwise(C[rows, :], want, "full rows")
    ii, jj = srng.integers(0, n, 256), srng.integers(0, n, 256)
    for i, j in zip(ii, jj):
        w = oracle.dgemm(A[0, i:i + 1, :], np.ascontiguousarray(B[0, :, j:j + 1]))
        assert_bitwise(C[i:i + 1, j:j + 1], w, "entry (%d, %d)" % (i, j))
