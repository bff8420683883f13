"""Elementwise EFTs, DD/TD/QD add/mul and the TD/QD variants (TDadd of
Alg. 3, TDmulq, the accurate TD product and QD addition) on the GPU are
bit-identical to the oracle (Sec. 2.1-2.5) on a million seeded elements,
gapped and cancelling operands, and edge cases."""
import numpy as np
import pytest

import oracle
from edge_operands import edge_operands, same_bits
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


@pytest.mark.parametrize("which", ["quick_two_sum", "two_sum", "two_prod"])
def test_eft_integer_pipes_bitwise(torch, which):
    """The integer-pipe form of each transformation (mp_eft_int, the form of
    the tiles that mpgemm_tile_int_ops reports) returns the bits of the
    operation sequence on the FP64 pipe for every input class, including
    NaN, infinity, overflow, subnormals, signed zeros and QuickTwoSum with
    |b| > |a|; where every value is finite it also equals the oracle."""
    from paper_2101_06584_gb300 import mpgemm
    rng = np.random.default_rng(300 + len(which))
    a, b = edge_operands(100_003, rng)
    with np.errstate(all="ignore"):
        si, ei = (host(t) for t in mpgemm.eft(which, dev(torch, a), dev(torch, b), int_pipes=True))
        ss, es = (host(t) for t in mpgemm.eft(which, dev(torch, a), dev(torch, b)))
        for got, want, nm in ((si, ss, "s"), (ei, es, "e")):
            ok = same_bits(got, want)
            bad = np.flatnonzero(~ok)
            assert ok.all(), "%s %s: %d mismatches, first a=%r b=%r got %r want %r" % (
                which, nm, bad.size, a[bad[0]], b[bad[0]], got[bad[0]], want[bad[0]])
        fin = np.isfinite(a) & np.isfinite(b) & np.isfinite(ss) & np.isfinite(es)
        ws, we = oracle.vec_eft(which, a[fin], b[fin])
    assert fin.sum() > 0.7 * a.size
    assert_bitwise(si[fin], ws, which + " s vs oracle")
    assert_bitwise(ei[fin], we, which + " e vs oracle")


OPS = [("dd", "add"), ("dd", "mul"), ("td", "add"), ("td", "addm"), ("td", "mul"),
       ("td", "mulq"), ("td", "mula"), ("qd", "add"), ("qd", "mul"), ("qd", "adda")]


@pytest.mark.parametrize("prec,op", OPS)
def test_vec_bitwise_random(torch, prec, op):
    from paper_2101_06584_gb300 import mpgemm
    P = I.P_OF[prec]
    rng = np.random.default_rng(200 + P)
    x = I.random_mp(P, N, rng, spread=30)
    y = I.random_mp(P, N, rng, spread=30)
    if op.startswith("add"):                       # a third nearly cancel
        cut = N // 3
        y[:, :cut] = I.expand(-x[0, :cut] * (1 + np.ldexp(1.0, -45)), P, rng)
    r = mpgemm.vec(prec, op, dev(torch, x), dev(torch, y))
    assert_bitwise(host(r), oracle.vec_op(prec, op, x, y), "%s %s" % (prec, op))


def _gapped(P, n, rng):
    """Normalised values whose components sit 0-30 bits further apart than
    adjacent binades (more bits than P components hold)."""
    out = np.empty((P, n))
    out[0] = np.ldexp(rng.uniform(-1, 1, n), rng.integers(-6, 7, n))
    for c in range(1, P):
        half_ulp = np.ldexp(np.spacing(np.abs(out[c - 1])), -1)
        out[c] = rng.uniform(-1, 1, n) * half_ulp * np.ldexp(1.0, -rng.integers(0, 30, n))
    return out


@pytest.mark.parametrize("prec,op", [("td", "add"), ("td", "addm"), ("qd", "add"), ("qd", "adda"),
                                     ("td", "mul"), ("td", "mulq"), ("td", "mula")])
def test_vec_bitwise_gapped_and_cancelling(torch, prec, op):
    """Operands with gapped components, and for the additions y = -x with
    one component scaled by 1 + d, |d| in 2^-52 .. 2^-1, and a quarter of the
    last components replaced, so that the sum cancels across components that
    do not line up: the sort, the accumulator's emissions and the tail all
    take data-dependent paths here."""
    from paper_2101_06584_gb300 import mpgemm
    P = I.P_OF[prec]
    n = 200_003
    rng = np.random.default_rng(400 + P)
    x = _gapped(P, n, rng)
    y = _gapped(P, n, rng)
    if op.startswith("add"):
        y = -x.copy()
        j = rng.integers(0, P, n)
        for c in range(P):
            sel = j == c
            y[c, sel] *= 1 + np.ldexp(rng.uniform(-1, 1, sel.sum()), -rng.integers(1, 53, sel.sum()))
        # and a quarter with one component replaced by fresh gapped values
        q = rng.integers(0, n, n // 4)
        y[P - 1, q] = _gapped(P, q.size, rng)[P - 1]
    r = mpgemm.vec(prec, op, dev(torch, x), dev(torch, y))
    assert_bitwise(host(r), oracle.vec_op(prec, op, x, y), "%s %s gapped" % (prec, op))


@pytest.mark.parametrize("prec,op", OPS)
def test_vec_bitwise_edges(torch, prec, op):
    from paper_2101_06584_gb300 import mpgemm
    P = I.P_OF[prec]
    x, y = I.edge_mp(P)
    # both orders of every pair
    x2 = np.concatenate([x, y], axis=1)
    y2 = np.concatenate([y, x], axis=1)
    r = mpgemm.vec(prec, op, dev(torch, x2), dev(torch, y2))
    assert_bitwise(host(r), oracle.vec_op(prec, op, x2, y2), "%s %s edges" % (prec, op))


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


@pytest.mark.parametrize("op", ["add", "mul"])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 6, 7, 64, 1_000_003, 1_000_004, 1_000_006])
def test_dd_paired_path(torch, op, n):
    """DD add and mul on 16-byte aligned planes take the four-elements-per-
    thread kernel (double2 loads; the last n mod 4 elements on their own),
    also in place and with unaligned planes (the one-element kernel):
    bit-identical to the oracle in every case."""
    from paper_2101_06584_gb300 import mpgemm
    rng = np.random.default_rng(250 + n % 97)
    x = I.random_mp(2, n, rng, spread=30)
    y = I.random_mp(2, n, rng, spread=30)
    y[:, : n // 3] = I.expand(-x[0, : n // 3] * (1 + np.ldexp(1.0, -45)), 2, rng)
    want = oracle.vec_op("dd", op, x, y)
    pad = n + (n % 2)                                 # an even plane stride keeps both planes aligned
    X = torch.zeros((2, pad), dtype=torch.float64, device="cuda")
    Y = torch.zeros((2, pad), dtype=torch.float64, device="cuda")
    X[:, :n] = dev(torch, x)
    Y[:, :n] = dev(torch, y)
    out = torch.full((2, pad), 7.0, dtype=torch.float64, device="cuda")
    mpgemm.vec("dd", op, X[:, :n], Y[:, :n], out=out[:, :n])
    assert_bitwise(host(out[:, :n]), want, "dd %s aligned n=%d" % (op, n))
    assert (host(out[:, n:]) == 7.0).all()
    mpgemm.vec("dd", op, X[:, :n], Y[:, :n], out=X[:, :n])          # in place
    assert_bitwise(host(X[:, :n]), want, "dd %s in place n=%d" % (op, n))
    Xu = torch.zeros((2, pad + 1), dtype=torch.float64, device="cuda")
    Xu[:, 1:n + 1] = dev(torch, x)                    # planes on an 8-byte boundary
    mpgemm.vec("dd", op, Xu[:, 1:n + 1], Y[:, :n], out=out[:, :n])
    assert_bitwise(host(out[:, :n]), want, "dd %s unaligned n=%d" % (op, n))
