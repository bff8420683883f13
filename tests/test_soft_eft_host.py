"""The integer-pipe error-free transformations (the device header
soft_fp64.cuh, Sec. 2.1's TwoSum, FastTwoSum and TwoProd formed from one
exact integer sum or product) compiled for the host and checked bit for bit
against the oracle's operation sequences, on every class of edge_operands:
NaN and infinity, subnormals, overflow, near-cancellation, exponent gaps
0-70 in either order, products at the subnormal and overflow boundaries,
signed zeros and ties.  Then the GEMM's whole multiply-add (mp_arith.cuh,
DDmul + DDadd, TDmul + TDaddq, QDmul + QDadd) under every arithmetic policy
equals the oracle's, step after step of a k-loop.  The same properties hold
on the GPU (test_gpu_elementwise.py, and every tile of test_gpu_gemm.py);
these checks run without one."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from edge_operands import edge_operands, same_bits
from paper_2101_06584_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2101_06584_gb300", "csrc")


@pytest.fixture(scope="module")
def soft(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("soft") / "libsofteft.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I", CSRC,
                    os.path.join(HERE, "soft_eft_host.cpp"), "-o", out], check=True)
    L = ctypes.CDLL(out)
    L.soft_eft_host.argtypes = [ctypes.c_int, ctypes.c_long] + [ctypes.c_void_p] * 4
    L.soft_eft_host.restype = None
    L.mad_host.argtypes = [ctypes.c_int, ctypes.c_uint, ctypes.c_long] + [ctypes.c_void_p] * 3
    L.mad_host.restype = None
    return L


def _run(L, which, a, b):
    a, b = np.ascontiguousarray(a), np.ascontiguousarray(b)
    s, e = np.empty_like(a), np.empty_like(a)
    idx = {"quick_two_sum": 0, "two_sum": 1, "two_prod": 2}[which]
    L.soft_eft_host(idx, a.size, a.ctypes.data, b.ctypes.data, s.ctypes.data, e.ctypes.data)
    return s, e


@pytest.mark.parametrize("which", ["quick_two_sum", "two_sum", "two_prod"])
def test_integer_form_equals_sequence(soft, which):
    rng = np.random.default_rng(700 + len(which))
    a, b = edge_operands(50_000, rng)
    s, e = _run(soft, which, a, b)
    with np.errstate(all="ignore"):
        ws, we = oracle.vec_eft(which, a, b)
    for got, want, nm in ((s, ws, "s"), (e, we, "e")):
        ok = same_bits(got, want)
        bad = np.flatnonzero(~ok)
        assert ok.all(), "%s %s: %d mismatches, first a=%r b=%r got %r want %r" % (
            which, nm, bad.size, a[bad[0]], b[bad[0]], got[bad[0]], want[bad[0]])


def test_signed_zero_errors(soft):
    """The zero conventions the sequences fix: TwoSum's exact zero error is
    +0; FastTwoSum returns b itself when b is a zero; TwoProd of a zero
    operand gives the signed zero product and a +0 error."""
    a = np.array([1.0, 1.0, -0.0, -0.0, 3.0, -2.5])
    b = np.array([-0.0, 0.0, -0.0, 0.0, -3.0, 0.0])
    s, e = _run(soft, "two_sum", a, b)
    assert same_bits(e, np.zeros(6)).all()
    assert same_bits(s, np.array([1.0, 1.0, -0.0, 0.0, 0.0, -2.5])).all()
    s, e = _run(soft, "quick_two_sum", a, b)
    assert same_bits(e, np.array([-0.0, 0.0, -0.0, 0.0, 0.0, 0.0])).all()
    s, e = _run(soft, "two_prod", np.array([-0.0, 5.0, -7.0]), np.array([3.0, -0.0, 0.0]))
    assert same_bits(s, np.array([-0.0, -0.0, -0.0])).all()
    assert same_bits(e, np.zeros(3)).all()



def _mad(L, P, mask, acc, a, b):
    """acc := add(acc, mul(a, b)) on SoA (P, n) arrays through the host build."""
    acc_aos = np.ascontiguousarray(acc.T)
    a_aos, b_aos = np.ascontiguousarray(a.T), np.ascontiguousarray(b.T)
    L.mad_host(P, mask, acc_aos.shape[0], acc_aos.ctypes.data, a_aos.ctypes.data, b_aos.ctypes.data)
    return np.ascontiguousarray(acc_aos.T)


@pytest.mark.parametrize("prec", ["dd", "td", "qd"])
def test_multiply_add_every_policy(soft, prec):
    """Sixteen steps of acc := add(acc, mul(a_j, b_j)) on 4000 random and the
    edge operand pairs (zeros, cancellation, ties, subnormal values and
    products): every mask of integer-pipe transformations gives the oracle's
    bits after every step."""
    P = I.P_OF[prec]
    rng = np.random.default_rng(720 + P)
    ex, ey = I.edge_mp(P)
    n_edge = ex.shape[1]
    n = 4000 + n_edge
    acc = {m: np.zeros((P, n)) for m in (0, 1, 2, 3, 4, 7)}
    want = np.zeros((P, n))
    for step in range(16):
        a = I.random_mp(P, n, rng)
        b = I.random_mp(P, n, rng)
        a[:, :n_edge], b[:, :n_edge] = (ex, ey) if step % 2 == 0 else (ey, ex)
        want = oracle.vec_op(prec, "add", want, oracle.vec_op(prec, "mul", a, b))
        for m in acc:
            acc[m] = _mad(soft, P, m, acc[m], a, b)
            ok = same_bits(acc[m], want)
            bad = np.argwhere(~ok)
            assert ok.all(), "%s mask %d step %d: %d mismatches, first %s" % (prec, m, step, len(bad), bad[0])


def test_boundaries_of_the_shortcuts(soft):
    """Where the integer form takes a shortcut or hands over to the sequence:
    TwoSum and FastTwoSum at exponent gaps 52-57 around powers of two (the
    spacing below a power of two is half the spacing above it, so a gap of 55
    is the first whose smaller operand never moves the sum), and TwoProd with
    e_a + e_b from 1070 to 1082 (its error term reaches the subnormal range
    below 1076, where the sequence runs), each against the oracle."""
    rng = np.random.default_rng(731)
    n = 20000
    big = np.ldexp(1.0, rng.integers(-40, 40, n)) * rng.choice([1.0, -1.0], n)
    big = np.where(rng.integers(0, 2, n).astype(bool), big, big * (1 + rng.random(n) * 2.0 ** -40))
    gap = rng.integers(52, 58, n)
    frac = 1.0 + rng.integers(0, 2 ** 52, n).astype(np.float64) * 2.0 ** -52
    small = np.ldexp(frac, (np.frexp(big)[1] - 1) - gap) * rng.choice([1.0, -1.0], n)
    for which in ("two_sum", "quick_two_sum"):
        s, e = _run(soft, which, big, small)
        ws, we = oracle.vec_eft(which, big, small)
        assert same_bits(s, ws).all() and same_bits(e, we).all(), which
    # products near 2^(e_a + e_b - 2046) with e_a + e_b from 1070 to 1082: their
    # 53-bit-lower error terms fall from the normal range into the subnormal one
    t = rng.integers(-40, 40, n)                          # keeps y normal
    x = np.ldexp(1.0 + rng.random(n), t) * rng.choice([1.0, -1.0], n)
    y = np.ldexp(1.0 + rng.random(n), rng.integers(1070, 1083, n) - 2046 - t)
    s, e = _run(soft, "two_prod", x, y)
    ws, we = oracle.vec_eft("two_prod", x, y)
    assert same_bits(s, ws).all() and same_bits(e, we).all()
    # the products do straddle the hand-over: some errors are subnormal or zero
    assert (np.abs(we) < 2.0 ** -1022).any() and (np.abs(we) >= 2.0 ** -1022).any()
