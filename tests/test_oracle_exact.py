"""Pins for the exact checker (oracle/exact.py) that every error bound of the
tests relies on: its dot products against brute-force Fraction sums over the
components (mixed exponents, zeros, subnormals, negative values), and its
error metrics against planted errors of known size."""
import math
from fractions import Fraction

import numpy as np

from oracle import exact as X
from paper_2101_06584_gb300 import inputs as I


def _brute_dot(A, B, i, j, absolute=False):
    s = Fraction(0)
    for p in range(A.shape[2]):
        a = sum((Fraction(float(A[c, i, p])) for c in range(A.shape[0])), Fraction(0))
        b = sum((Fraction(float(B[c, p, j])) for c in range(B.shape[0])), Fraction(0))
        s += abs(a) * abs(b) if absolute else a * b
    return s


def test_value_and_ulp():
    assert X.value([1.0, 2.0 ** -60, -2.0 ** -120]) == 1 + Fraction(1, 2 ** 60) - Fraction(1, 2 ** 120)
    assert X.value([]) == 0
    assert X.ulp(1.0) == Fraction(1, 2 ** 52) and X.ulp(-3.0) == Fraction(1, 2 ** 51)
    assert X.ulp(2.0 ** -1074) == Fraction(1, 2 ** 1074) and X.ulp(2.0 ** -1022) == Fraction(1, 2 ** 1074)


def test_dot_and_absdot_against_brute_force():
    rng = np.random.default_rng(800)
    for P in (2, 3, 4):
        m, n, k = 4, 3, 9
        A = I.ill_scaled(P, (m, k), rng, -300, 300)
        B = I.ill_scaled(P, (k, n), rng, -300, 300)
        A[:, 1, 2] = 0.0                                # a zero entry
        A[0, 2, 3] = 2.0 ** -1074                        # subnormal leading component
        A[1:, 2, 3] = 0.0
        B[:, 4, 1] = -B[:, 4, 1]
        ex = X.ExactRows(A, B)
        for i in range(m):
            for j in range(n):
                assert ex.dot(i, j) == _brute_dot(A, B, i, j), (P, i, j)
                assert ex.absdot(i, j) == _brute_dot(A, B, i, j, absolute=True), (P, i, j)


def test_gemm_error_measures_planted_errors():
    """C equal to the exact product rounded to DD (error at most 2^-106
    relative per entry), then one entry moved by a known amount: the metrics
    report exactly that amount against the brute-force norms."""
    rng = np.random.default_rng(801)
    m, n, k = 3, 4, 6
    A, B = I.uniform(2, (m, k), rng), I.uniform(2, (k, n), rng)
    exact = {(i, j): _brute_dot(A, B, i, j) for i in range(m) for j in range(n)}
    C = np.zeros((2, m, n))
    for (i, j), v in exact.items():
        hi = float(v)
        C[0, i, j], C[1, i, j] = hi, float(v - Fraction(hi))
    ent = sorted(exact)
    base = X.gemm_error(C, A, B, ent)
    assert base["max_abs"] <= 2.0 ** -104
    delta = 2.0 ** -40
    C[1, 1, 2] += delta
    got = X.gemm_error(C, A, B, ent)
    num = sum((X.value(C[:, i, j]) - exact[(i, j)]) ** 2 for (i, j) in ent)
    den_abs = sum(_brute_dot(A, B, i, j, absolute=True) ** 2 for (i, j) in ent)
    den_c = sum(exact[e] ** 2 for e in ent)
    assert math.isclose(got["err_abs"], math.sqrt(float(num / den_abs)), rel_tol=1e-12)
    assert math.isclose(got["err_rel"], math.sqrt(float(num / den_c)), rel_tol=1e-12)
    ab = _brute_dot(A, B, 1, 2, absolute=True)
    assert math.isclose(got["max_abs"], float(abs(X.value(C[:, 1, 2]) - exact[(1, 2)]) / ab), rel_tol=1e-12)
    assert got["max_abs"] > 2.0 ** -42
