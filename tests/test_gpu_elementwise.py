"""Elementwise EFTs and DD/TD/QD add/mul on the GPU are bit-identical to the
oracle (Sec. 2.1-2.5) on a million seeded elements plus edge cases."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_bitwise, dev, host, torch_cuda
from paper_2101_06584_gb300 import inputs as I

pytestmark = pytest.mark.gpu
N = 1_000_003          # not a multiple of the block or the grid


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.mark.parametrize("which", ["quick_two_sum", "two_sum", "two_prod"])
def test_eft_bitwise(torch, which):
    from paper_2101_06584_gb300 import mpgemm
    rng = np.random.default_rng(100)
    a = np.ldexp(rng.uniform(-1, 1, N), rng.integers(-60, 60, N))
    b = np.ldexp(rng.uniform(-1, 1, N), rng.integers(-60, 60, N))
    b[::7] = -a[::7]
    b[1::7] = a[1::7]
    if which == "quick_two_sum":                  # its precondition |a| >= |b|
        sw = np.abs(a) < np.abs(b)
        a[sw], b[sw] = b[sw], a[sw].copy()
    s, e = mpgemm.eft(which, dev(torch, a), dev(torch, b))
    ws, we = oracle.vec_eft(which, a, b)
    assert_bitwise(host(s), ws, which + " s")
    assert_bitwise(host(e), we, which + " e")


OPS = [("dd", "add"), ("dd", "mul"), ("td", "add"), ("td", "addm"), ("td", "mul"),
       ("qd", "add"), ("qd", "mul")]


@pytest.mark.parametrize("prec,op", OPS)
def test_vec_bitwise_random(torch, prec, op):
    from paper_2101_06584_gb300 import mpgemm
    P = I.P_OF[prec]
    rng = np.random.default_rng(200 + P)
    x = I.random_mp(P, N, rng, spread=30)
    y = I.random_mp(P, N, rng, spread=30)
    if op != "mul":                                # a third nearly cancel
        cut = N // 3
        y[:, :cut] = I.expand(-x[0, :cut] * (1 + np.ldexp(1.0, -45)), P, rng)
    r = mpgemm.vec(prec, op, dev(torch, x), dev(torch, y))
    assert_bitwise(host(r), oracle.vec_op(prec, "add" if op == "addm" else op, x, y)
                   if op != "addm" else _addm(x, y), "%s %s" % (prec, op))


def _addm(x, y):
    out = np.empty_like(x)
    for t in range(x.shape[1]):
        out[:, t] = oracle.op("td", "addm", x[:, t], y[:, t])
    return out


@pytest.mark.parametrize("prec,op", OPS)
def test_vec_bitwise_edges(torch, prec, op):
    from paper_2101_06584_gb300 import mpgemm
    P = I.P_OF[prec]
    x, y = I.edge_mp(P)
    # both orders of every pair
    x2 = np.concatenate([x, y], axis=1)
    y2 = np.concatenate([y, x], axis=1)
    r = mpgemm.vec(prec, op, dev(torch, x2), dev(torch, y2))
    if op == "addm":
        want = _addm(x2, y2)
    else:
        want = oracle.vec_op(prec, op, x2, y2)
    assert_bitwise(host(r), want, "%s %s edges" % (prec, op))


def test_vec_in_place(torch):
    from paper_2101_06584_gb300 import mpgemm
    rng = np.random.default_rng(300)
    x = I.random_mp(4, 4097, rng)
    y = I.random_mp(4, 4097, rng)
    want = oracle.vec_op("qd", "mul", x, y)
    xt = dev(torch, x)
    mpgemm.vec("qd", "mul", xt, dev(torch, y), out=xt)
    assert_bitwise(host(xt), want, "in place")


def test_empty_vector(torch):
    from paper_2101_06584_gb300 import mpgemm
    z = torch.empty((2, 0), dtype=torch.float64, device="cuda")
    r = mpgemm.vec("dd", "add", z, z)
    assert r.shape == (2, 0)
