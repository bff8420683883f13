"""The Strassen form on the GPU against the oracle's Strassen (Sec. 3): bit for
bit for DD, TD and QD at one to three levels, on ragged and odd shapes (where
the recursion stops early) and on strided views; at 2048^3 within the error
bound of the exact product."""
import numpy as np
import pytest

from gpu_util import assert_bitwise, dev, host, torch_cuda
from oracle import exact as X
from oracle import strassen as ST
from paper_2101_06584_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def run(torch, prec, A, B, L, views=False):
    from paper_2101_06584_gb300 import mpgemm as mm
    P = I.P_OF[prec]
    m, k = A.shape[1], A.shape[2]
    n = B.shape[2]
    if views:
        # operands and result as windows of larger matrices (leading dimensions > width)
        Ab = dev(torch, np.zeros((P, m + 3, k + 5)))
        Bb = dev(torch, np.zeros((P, k + 2, n + 7)))
        Cb = torch.zeros((P, m + 4, n + 9), dtype=torch.float64, device="cuda")
        Ab[:, 1:1 + m, 2:2 + k] = dev(torch, A)
        Bb[:, 2:2 + k, 3:3 + n] = dev(torch, B)
        Ad, Bd, Cd = Ab[:, 1:1 + m, 2:2 + k], Bb[:, 2:2 + k, 3:3 + n], Cb[:, 3:3 + m, 1:1 + n]
    else:
        Ad, Bd, Cd = dev(torch, A), dev(torch, B), None
    nb = mm.workspace_size(prec, m, n, k, strassen=L)
    ws = torch.empty(max(nb, 1), dtype=torch.uint8, device="cuda")
    C = mm.gemm(prec, Ad, Bd, out=Cd, strassen=L, workspace=ws if nb else None)
    return host(C)


@pytest.mark.parametrize("prec,shape,L", [
    ("dd", (64, 64, 64), 1), ("dd", (64, 64, 64), 2), ("dd", (96, 80, 112), 3),
    ("td", (64, 48, 32), 2), ("qd", (48, 64, 32), 2), ("dd", (70, 66, 130), 2), ("qd", (18, 14, 10), 3),
])
def test_bitwise_against_oracle(torch, prec, shape, L):
    P = I.P_OF[prec]
    m, n, k = shape
    rng = np.random.default_rng(900 + m + n + k + L)
    A, B = I.ill_scaled(P, (m, k), rng), I.uniform(P, (k, n), rng)
    want = ST.strassen(prec, A, B, L)
    assert_bitwise(run(torch, prec, A, B, L), want, "%s %s L=%d" % (prec, shape, L))


def test_odd_shapes_are_the_plain_gemm(torch):
    import oracle
    rng = np.random.default_rng(950)
    for (m, n, k) in ((63, 64, 64), (64, 1, 64), (64, 64, 33)):
        A, B = I.uniform(2, (m, k), rng), I.uniform(2, (k, n), rng)
        assert_bitwise(run(torch, "dd", A, B, 2), oracle.gemm("dd", A, B), "odd %s" % ((m, n, k),))


def test_strided_views(torch):
    rng = np.random.default_rng(960)
    A, B = I.uniform(4, (40, 24), rng), I.uniform(4, (24, 56), rng)
    assert_bitwise(run(torch, "qd", A, B, 2, views=True), ST.strassen("qd", A, B, 2), "qd views")


def test_full_size_within_bound(torch):
    """DD 2048^3, two levels: sampled entries within 4^L n 2^-100 of the exact
    product, like the k-sequential result."""
    from paper_2101_06584_gb300 import mpgemm as mm
    n, L = 2048, 2
    rng = I.rng_for(4)
    A, B = I.uniform(2, (n, n), rng), I.uniform(2, (n, n), rng)
    C = run(torch, "dd", A, B, L)
    srng = np.random.default_rng(970)
    entries = [(int(i), int(j)) for i, j in zip(srng.integers(0, n, 6), srng.integers(0, n, 6))]
    err = X.gemm_error(C, A, B, entries)
    assert err["err_abs"] <= 4.0 ** L * n * 2.0 ** -100, err
    plain = host(mm.gemm_plain("dd", dev(torch, A), dev(torch, B)))
    err0 = X.gemm_error(plain, A, B, entries)
    assert err0["err_abs"] <= n * 2.0 ** -100, err0
