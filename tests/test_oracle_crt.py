"""Pins of the CRT-form oracle (oracle/crt.py) on the CPU: the moduli are
pairwise coprime and their residues fit int8/bf16; the recovery inverts the
residue map on every integer of the range (brute force on small moduli sets,
random and boundary values on the large ones); the residue route equals the
direct definition (the integer product A'B' computed without residues); the
nearest expansion is the correctly rounded greedy split; and the results stay
within the rounding bound of the scaled integers against exact arithmetic,
exactly for small-integer matrices."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import crt as R
from oracle import exact as X
from paper_2101_06584_gb300 import inputs as I


def test_moduli_are_pairwise_coprime_and_fit():
    ms = R.MODULI
    assert ms[0] == 256 and all(a > b for a, b in zip(ms, ms[1:]))
    for i, a in enumerate(ms):
        for b in ms[i + 1:]:
            assert math.gcd(a, b) == 1, (a, b)
        lo, hi = R.sym_mod(-10 ** 9, a), R.sym_mod(10 ** 9, a)
        assert -128 <= lo <= 127 and -128 <= hi <= 127
        reps = {R.sym_mod(x, a) for x in range(-3 * a, 3 * a)}
        assert reps == set(range(-(a // 2), (a + 1) // 2)), a      # a full residue system
    assert R.k_limit() * 128 * 128 < 2 ** 31 <= (R.k_limit() + 1) * 128 * 128 + 128 * 128


def test_recovery_inverts_residues():
    rng = np.random.default_rng(40)
    for N in (1, 2, 3):                       # brute force over the whole range
        M = R.modulus_product(N)
        if M > 2 ** 25:
            continue
        step = max(1, M // 4096)
        for x in range(-(M // 2), (M + 1) // 2, step):
            assert R.crt_recover([x % m for m in R.MODULI[:N]], N) == x
    for N in (8, 26, 28, 40, len(R.MODULI)):
        M = R.modulus_product(N)
        cases = [-(M // 2), (M + 1) // 2 - 1, 0, 1, -1]
        cases += [int(rng.integers(0, 2 ** 62)) * int(rng.integers(0, 2 ** 62)) % M - M // 2 for _ in range(200)]
        for x in cases:
            assert R.crt_recover([x % m for m in R.MODULI[:N]], N) == x, (N, x)


def test_beta_is_the_largest_safe_bit_count():
    for N in (4, 16, 26, 30, 48):
        for k in (1, 37, 1024, 4096, 100000):
            b = R.beta_bits(N, k)
            M = R.modulus_product(N)
            assert k * 2 ** (2 * b - 1) < M <= k * 2 ** (2 * b + 1)


def test_nearest_expansion():
    rng = np.random.default_rng(41)
    for _ in range(300):
        v = Fraction(int(rng.integers(-2 ** 62, 2 ** 62)) * 3 ** 70 + 1, 2 ** int(rng.integers(0, 400)))
        for P in (2, 3, 4):
            c = R.nearest_expansion(v, P)
            rest = v
            for t in range(P):
                assert c[t] == float(rest)
                rest -= Fraction(c[t])
            for t in range(P - 1):
                assert c[t + 1] == 0.0 or abs(c[t + 1]) <= math.ulp(c[t]) / 2
    assert R.nearest_expansion(Fraction(1) + Fraction(1, 2 ** 53), 2) == [1.0, 2.0 ** -53]   # a tie to even


def _direct(A, B, N):
    """The definition without residues: A'B' from the integers themselves."""
    P, m, k = A.shape
    n = B.shape[2]
    beta = R.beta_bits(N, k)
    sig, Ai = R.integer_rows(A, beta)
    tau, Bi = R.integer_rows(np.ascontiguousarray(B.transpose(0, 2, 1)), beta)
    C = np.zeros((P, m, n))
    for i in range(m):
        for j in range(n):
            Cp = sum(x * y for x, y in zip(Ai[i], Bi[j]))
            C[:, i, j] = R.nearest_expansion(Fraction(Cp) * Fraction(2) ** (sig[i] + tau[j] - 2 * beta), P)
    return C


@pytest.mark.parametrize("prec,N", [("dd", 3), ("dd", 26), ("td", 40), ("qd", 49)])
def test_residue_route_equals_the_direct_product(prec, N):
    P = I.P_OF[prec]
    rng = np.random.default_rng(42 + N)
    for A, B in ((I.uniform(P, (5, 23), rng), I.ill_scaled(P, (23, 4), rng)),
                 I.cancelling_pair(P, 4, 5, 18, rng)):
        C, _, _, _ = R.gemm(A, B, N)
        want = _direct(A, B, N)
        assert (C.view(np.int64) == want.view(np.int64)).all()


@pytest.mark.parametrize("prec,N", [("dd", 20), ("dd", 28), ("td", 44)])
def test_error_within_the_scaling_bound(prec, N):
    """|c_hat - c| <= k 2^(sigma_i + tau_j - beta - 1) (1 + 2^-beta) + 2^-(53P - 2) |c|
    per entry, exactly; the normwise error falls with beta."""
    P = I.P_OF[prec]
    rng = np.random.default_rng(43 + N)
    m, n, k = 6, 7, 40
    A, B = I.uniform(P, (m, k), rng), I.ill_scaled(P, (k, n), rng)
    C, sig, tau, beta = R.gemm(A, B, N)
    ex = X.ExactRows(A, B)
    for i in range(m):
        for j in range(n):
            c = ex.dot(i, j)
            bound = k * Fraction(2) ** (sig[i] + tau[j] - beta - 1) * (1 + Fraction(1, 2 ** 50)) + \
                Fraction(1, 2 ** (53 * P - 2)) * abs(c)
            assert abs(X.value(C[:, i, j]) - c) <= bound, (i, j)
    coarse, _, _, _ = R.gemm(A, B, N - 6)
    ent = [(i, j) for i in range(m) for j in range(n)]
    assert X.gemm_error(C, A, B, ent)["err_abs"] < X.gemm_error(coarse, A, B, ent)["err_abs"] * 2.0 ** -10


def test_small_integers_are_exact():
    """Integer entries below 2^10 scale to integers without rounding, so the
    product is exact (and representable) with zero lower components."""
    rng = np.random.default_rng(44)
    A = np.zeros((2, 9, 30))
    B = np.zeros((2, 30, 8))
    A[0] = rng.integers(-1000, 1000, size=(9, 30))
    B[0] = rng.integers(-1000, 1000, size=(30, 8))
    C, _, _, beta = R.gemm(A, B, 12)
    assert beta >= 20
    assert (C[0] == A[0].astype(object).dot(B[0].astype(object)).astype(np.float64)).all()
    assert (C[1] == 0).all()


def test_integers_round_to_nearest_even():
    """Scaled entries are the nearest integers: within 1/2 of a 2^(beta - sigma)
    for random DD entries, and at exact halves the even neighbour (entries
    built as (2j + 1) / 2 units of 2^(sigma - beta))."""
    rng = np.random.default_rng(45)
    A = I.uniform(2, (3, 50), rng)
    beta = 30
    sig, rows = R.integer_rows(A, beta)
    for i in range(3):
        for p in range(50):
            exact = X.value(A[:, i, p]) * Fraction(2) ** (beta - sig[i])
            assert abs(rows[i][p] - exact) <= Fraction(1, 2) + Fraction(2, 2 ** 64)
    T = np.zeros((2, 1, 6))
    T[0, 0, :] = [0.75, 2.5 / 64, 3.5 / 64, -2.5 / 64, -3.5 / 64, 5.5 / 64]   # sigma = 1 (ilogb(0.75) + 2)
    sig, rows = R.integer_rows(T, 7)                                         # units of 2^(1 - 7) = 1/64
    assert sig == [1] and rows[0] == [48, 2, 4, -2, -4, 6]


MUTANTS = {
    "residues shifted": lambda m: setattr(m, "sym_mod", lambda x, mod: (x % mod) - mod // 2),
    "floored integers": lambda m: setattr(
        m, "scaled_integer",
        lambda comps, sh: math.floor(sum((Fraction(float(c)) for c in comps), Fraction(0)) * Fraction(2) ** sh)),
    "guard bits dropped": lambda m: setattr(
        m, "scaled_integer",
        lambda comps, sh: round(Fraction(sum(math.floor(Fraction(float(c)) * Fraction(2) ** sh) for c in comps)))),
    "recovery not centred": lambda m: setattr(
        m, "crt_recover",
        lambda res, N: sum(res[i] * (m.modulus_product(N) // m.MODULI[i]) *
                           pow(m.modulus_product(N) // m.MODULI[i], -1, m.MODULI[i])
                           for i in range(N)) % m.modulus_product(N)),
    "one bit too many": lambda m: setattr(m, "beta_bits",
                                          (lambda f: lambda N, k, halves=1: f(N, k, halves) + 1)(m.beta_bits)),
    "low half not balanced": lambda m: setattr(m, "split", lambda x, w: (x >> w, x % (1 << w))),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistakes_are_caught(monkeypatch, name):
    """Each planted mistake in a copy of the oracle's steps fails a pin."""
    import importlib
    import sys
    mod = importlib.import_module("oracle.crt")
    saved = {k: getattr(mod, k) for k in ("sym_mod", "scaled_integer", "crt_recover", "beta_bits", "split")}
    try:
        MUTANTS[name](mod)
        caught = False
        for pin, args in ((test_recovery_inverts_residues, ()), (test_beta_is_the_largest_safe_bit_count, ()),
                          (test_residue_route_equals_the_direct_product, ("dd", 26)),
                          (test_error_within_the_scaling_bound, ("dd", 28)), (test_small_integers_are_exact, ()),
                          (test_integers_round_to_nearest_even, ()), (test_split_integers, ()),
                          (test_split_route_equals_the_direct_product, ("qd", 28))):
            try:
                pin(*args)
            except (AssertionError, ValueError, OverflowError):
                caught = True
                break
        assert caught, "planted mistake '%s' passed every pin" % name
    finally:
        for k, v in saved.items():
            setattr(mod, k, v)
        assert sys.modules["oracle.crt"] is mod


def test_split_integers():
    """x = x1 2^w + x0 with x0 in [-2^(w-1), 2^(w-1)), for random and boundary
    values; and w is the largest with k 2^(2w) < M."""
    rng = np.random.default_rng(46)
    for w in (1, 7, 64, 101):
        for x in [0, 1, -1, (1 << (2 * w - 1)), -(1 << (2 * w - 1)), (1 << (w - 1)), -(1 << (w - 1))] + \
                 [int(rng.integers(-2 ** 62, 2 ** 62)) << int(rng.integers(0, 2 * w)) for _ in range(100)]:
            x1, x0 = R.split(x, w)
            assert x1 * (1 << w) + x0 == x and -(1 << (w - 1)) <= x0 < (1 << (w - 1)), (x, w)
            if abs(x) <= 1 << (2 * w - 1):
                assert abs(x1) <= 1 << (w - 1)
    for N in (8, 26, 28, 40):
        for k in (1, 1024, 4096, 65535):
            b = R.beta_bits(N, k, halves=2)
            assert b % 2 == 0 and k * 2 ** b < R.modulus_product(N) <= k * 2 ** (b + 2)


@pytest.mark.parametrize("prec,N", [("dd", 12), ("qd", 28), ("td", 20)])
def test_split_route_equals_the_direct_product(prec, N):
    """The split-integer route (three products recovered by CRT, combined)
    equals the nearest expansion of A'B' computed from the integers directly,
    with beta = 2w; and stays within the scaling bound of the exact product."""
    P = I.P_OF[prec]
    rng = np.random.default_rng(47 + N)
    A, B = I.ill_scaled(P, (4, 33), rng), I.uniform(P, (33, 5), rng)
    C, sig, tau, beta = R.gemm(A, B, N, halves=2)
    assert beta == R.beta_bits(N, 33, halves=2)
    sigd, Ai = R.integer_rows(A, beta)
    taud, Bi = R.integer_rows(np.ascontiguousarray(B.transpose(0, 2, 1)), beta)
    ex = X.ExactRows(A, B)
    for i in range(4):
        for j in range(5):
            Cp = sum(x * y for x, y in zip(Ai[i], Bi[j]))
            want = R.nearest_expansion(Fraction(Cp) * Fraction(2) ** (sigd[i] + taud[j] - 2 * beta), P)
            assert list(C[:, i, j]) == want, (i, j)
            c = ex.dot(i, j)
            bound = 33 * Fraction(2) ** (sig[i] + tau[j] - beta - 1) * (1 + Fraction(1, 2 ** 50)) + \
                Fraction(1, 2 ** (53 * P - 2)) * abs(c)
            assert abs(X.value(C[:, i, j]) - c) <= bound, (i, j)
