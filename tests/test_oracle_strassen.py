"""Pins for the Strassen oracle (CPU only): no levels, or odd dimensions, give
the k-sequential GEMM bit for bit; small-integer matrices come out exact at
every depth (so a wrong formula, sign or block is caught); planted mistakes
are caught; random DD/TD/QD products stay within a Strassen error bound of
the exact product."""
import numpy as np
import pytest

import oracle
from oracle import exact as X
from oracle import strassen as ST
from paper_2101_06584_gb300 import inputs as I


def int_matrices(P, m, k, n, seed, amp=200):
    rng = np.random.default_rng(seed)
    A = np.zeros((P, m, k))
    B = np.zeros((P, k, n))
    A[0] = rng.integers(-amp, amp + 1, (m, k))
    B[0] = rng.integers(-amp, amp + 1, (k, n))
    return A, B


def test_no_levels_and_odd_dimensions_are_the_plain_gemm():
    rng = I.rng_for(0)
    for (m, k, n, L) in ((8, 8, 8, 0), (7, 8, 8, 2), (8, 9, 8, 1), (8, 8, 5, 3), (6, 10, 4, 1)):
        A, B = I.uniform(2, (m, k), rng), I.uniform(2, (k, n), rng)
        got = ST.strassen("dd", A, B, L)
        want = oracle.gemm("dd", A, B)
        if L == 0 or m % 2 or k % 2 or n % 2:
            assert np.array_equal(got.view(np.int64), want.view(np.int64))


@pytest.mark.parametrize("prec,L", [("dd", 1), ("dd", 2), ("dd", 3), ("td", 2), ("qd", 2)])
def test_integer_matrices_are_exact(prec, L):
    P = I.P_OF[prec]
    for (m, k, n) in ((8, 8, 8), (16, 24, 8), (24, 16, 32)):
        A, B = int_matrices(P, m, k, n, seed=m * 100 + k + n + L)
        exact = A[0].astype(np.int64) @ B[0].astype(np.int64)
        C = ST.strassen(prec, A, B, L)
        assert np.array_equal(C[0], exact.astype(np.float64)), (prec, L, m, k, n)
        assert not np.any(C[1:])


def test_two_by_two_blocks_against_brute_force():
    """The seven products and four combinations give the textbook 2 x 2
    product for every sign pattern of small integers."""
    rng = np.random.default_rng(5)
    for _ in range(200):
        A, B = int_matrices(2, 2, 2, 2, seed=int(rng.integers(1 << 30)), amp=9)
        C = ST.strassen("dd", A, B, 1)
        assert np.array_equal(C[0], A[0] @ B[0])


def test_planted_mistakes_are_caught():
    """Each formula of the oracle, changed in a plausible way (a product with
    a wrong sign, a combination with a term dropped, blocks swapped), breaks
    the exact integer product."""
    A, B = int_matrices(2, 8, 8, 8, seed=99)
    exact = (A[0].astype(np.int64) @ B[0].astype(np.int64)).astype(np.float64)
    orig = ST.strassen

    def mutant(kind):
        def f(prec, A_, B_, levels):
            A_ = np.asarray(A_, dtype=np.float64)
            B_ = np.asarray(B_, dtype=np.float64)
            _, m, k = A_.shape
            n = B_.shape[2]
            if levels <= 0 or m % 2 or n % 2 or k % 2:
                return oracle.gemm(prec, A_, B_)
            m2, n2, k2 = m // 2, n // 2, k // 2
            A11, A12, A21, A22 = A_[:, :m2, :k2], A_[:, :m2, k2:], A_[:, m2:, :k2], A_[:, m2:, k2:]
            B11, B12, B21, B22 = B_[:, :k2, :n2], B_[:, :k2, n2:], B_[:, k2:, :n2], B_[:, k2:, n2:]
            add = lambda x, y: ST._add(prec, x, y)
            sub = lambda x, y: ST._sub(prec, x, y)
            rec = lambda x, y: f(prec, x, y, levels - 1)
            M1 = rec(add(A11, A22), add(B11, B22))
            M2 = rec(add(A21, A22), B11)
            M3 = rec(A11, sub(B12, B22))
            M4 = rec(A22, sub(B21, B11) if kind != "M4 sign" else sub(B11, B21))
            M5 = rec(add(A11, A12), B22 if kind != "M5 block" else B21)
            M6 = rec(sub(A21, A11), add(B11, B12))
            M7 = rec(sub(A12, A22), add(B21, B22))
            C = np.empty((A_.shape[0], m, n))
            C[:, :m2, :n2] = add(sub(add(M1, M4), M5), M7) if kind != "C11 drop" else sub(add(M1, M4), M5)
            C[:, :m2, n2:] = add(M3, M5)
            C[:, m2:, :n2] = add(M2, M4)
            C[:, m2:, n2:] = add(add(sub(M1, M2), M3), M6) if kind != "C22 sign" else add(add(add(M1, M2), M3), M6)
            return C
        return f

    # the unmodified copy reproduces the oracle
    assert np.array_equal(mutant("none")("dd", A, B, 1)[0], exact)
    assert np.array_equal(orig("dd", A, B, 1)[0], exact)
    for kind in ("M4 sign", "M5 block", "C11 drop", "C22 sign"):
        assert not np.array_equal(mutant(kind)("dd", A, B, 2)[0], exact), kind


@pytest.mark.parametrize("prec,L", [("dd", 1), ("dd", 3), ("td", 2), ("qd", 2)])
def test_random_products_within_bound(prec, L):
    """Strassen's normwise error grows with the depth (each level adds a few
    block additions ahead of the products); on random inputs the error stays
    within 4^L k 2^-p of the exact product."""
    P = I.P_OF[prec]
    p = {"dd": 100, "td": 150, "qd": 200}[prec]
    rng = I.rng_for(4)
    n = 32
    A, B = I.uniform(P, (n, n), rng), I.uniform(P, (n, n), rng)
    C = ST.strassen(prec, A, B, L)
    err = X.gemm_error(C, A, B, [(i, j) for i in range(0, n, 3) for j in range(0, n, 5)])
    assert err["err_abs"] <= 4.0 ** L * n * 2.0 ** -p, err
