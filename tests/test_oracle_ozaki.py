"""Pins for the oracle of the INT8 error-free slicing form (CPU only): the
digits reconstruct each entry exactly, stay in [-64, 64] and round ties to
even; the scale keeps |a| 2^-sigma < 1/2; small-integer matrices come out
exact; the error against the exact product falls by ~2^-7 per slice and meets
k 2^-100 at 14 slices; and planted mistakes are caught."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import exact as X
from oracle import ozaki as OZ
from paper_2101_06584_gb300 import inputs as I


def check_digits(components, S, sigma=None):
    comps = [float(c) for c in components]
    sg = OZ.scale_exponent([comps[0]]) if sigma is None else sigma
    ds, rem = OZ.digits(comps, sg, S)
    a = sum(map(Fraction, comps), Fraction(0))
    recon = sum((Fraction(d) * Fraction(2) ** (-7 * (s + 1)) for s, d in enumerate(ds)), Fraction(0))
    recon = (recon + rem * Fraction(2) ** (-7 * S)) * Fraction(2) ** sg
    assert recon == a
    assert all(-64 <= d <= 64 for d in ds)
    assert abs(rem) <= Fraction(1, 2)
    return ds


def test_digits_reconstruct_exactly():
    rng = np.random.default_rng(500)
    x = I.random_mp(2, 400, rng, spread=40)
    for t in range(x.shape[1]):
        for S in (1, 5, 14, 16):
            check_digits(x[:, t], S)


def test_scale_exponent_bounds():
    rng = np.random.default_rng(501)
    for _ in range(300):
        row = I.random_mp(2, 17, rng, spread=30)
        sg = OZ.scale_exponent(row[0])
        for p in range(row.shape[1]):
            assert abs(X.value(row[:, p])) * Fraction(2) ** (-sg) < Fraction(1, 2)
        assert max(abs(v) for v in row[0]) * 2.0 ** (-sg) >= 0.25
    assert OZ.scale_exponent([0.0, -0.0]) == 0


def test_ties_round_to_even():
    # a 2^-sigma = 3/256: y = 1.5 -> digit 2, remainder -1/2; then -64
    sg = 0
    ds, rem = OZ.digits([3.0 / 256.0, 0.0], sg, 3)
    assert ds == [2, -64, 0] and rem == 0
    ds, _ = OZ.digits([5.0 / 256.0, 0.0], sg, 2)          # y = 2.5 -> 2
    assert ds == [2, 64]
    ds, _ = OZ.digits([5.0 / 256.0, 2.0 ** -80], sg, 2)   # just above the tie -> 3
    assert ds[0] == 3
    ds, _ = OZ.digits([-3.0 / 256.0, 0.0], sg, 2)         # y = -1.5 -> -2
    assert ds == [-2, 64]


def test_small_integer_matrices_are_exact():
    rng = np.random.default_rng(502)
    m, n, k = 6, 7, 33
    A = np.zeros((2, m, k))
    B = np.zeros((2, k, n))
    A[0] = rng.integers(-63, 64, (m, k))
    B[0] = rng.integers(-63, 64, (k, n))
    A[0][:, 0] = 63                         # every row / column reaches 2^5..2^6
    B[0][0, :] = -40
    C, _, _ = OZ.gemm(A, B, 3)
    want = A[0].astype(object).dot(B[0].astype(object))
    assert (C[0] == want.astype(np.float64)).all() and (C[1] == 0).all()


@pytest.mark.parametrize("gen", ["uniform", "cancelling"])
def test_error_shrinks_per_slice_and_meets_bound(gen):
    rng = np.random.default_rng(503)
    m, n, k = 10, 9, 40
    if gen == "uniform":
        A, B = I.uniform(2, (m, k), rng), I.uniform(2, (k, n), rng)
    else:
        A, B = I.cancelling_pair(2, m, n, k, rng)
    ent = [(i, j) for i in range(m) for j in range(n)]
    errs = {}
    for S in (8, 10, 14, 16):
        C, _, _ = OZ.gemm(A, B, S)
        errs[S] = X.gemm_error(C, A, B, ent)["err_abs"]
    # entries spread over 2^+-20 within a row need more slices than uniform ones
    assert errs[16 if gen == "cancelling" else 14] <= k * 2.0 ** -100
    assert errs[10] < errs[8] * 2.0 ** -10


def test_matches_plain_definition_of_weights():
    """The weight sums equal the full double sum over slice pairs with s+t=w."""
    rng = np.random.default_rng(504)
    A, B = I.uniform(2, (3, 12), rng), I.uniform(2, (12, 4), rng)
    S = 4
    _, DA = OZ.slice_rows(A, S)
    _, DB = OZ.slice_cols(B, S)
    Pw = OZ.weight_products(DA, DB, S)
    for w in range(2, S + 2):
        for i in range(3):
            for j in range(4):
                tot = 0
                for s in range(1, S + 1):
                    for t in range(1, S + 1):
                        if s + t == w:
                            tot += sum(int(DA[s - 1, i, p]) * int(DB[t - 1, j, p]) for p in range(12))
                assert Pw[w][i, j] == tot


MUTANTS = [
    ("ties away from zero", "digits",
     lambda comps, sigma, S, truncate=False: _digits_mut(comps, sigma, S, tie="away")),
    ("scale one too small", "scale_exponent",
     lambda hv: (lambda mx: 0 if mx == 0 else OZ.ilogb(mx) + 1)(max(abs(float(v)) for v in hv))),
    ("drops the least significant weight", "weight_products",
     lambda DA, DB, S: {w: (v if w < S + 1 else v * 0) for w, v in _orig_wp(DA, DB, S).items()}),
    ("groups shifted the wrong way", "weight_groups",
     lambda S, P: [list(reversed(g)) for g in _orig_groups(S, P)]),
]
_orig_digits = OZ.digits
_orig_wp = OZ.weight_products
_orig_groups = OZ.weight_groups


def _digits_mut(comps, sigma, S, tie):
    x = sum((Fraction(float(c)) for c in comps), Fraction(0)) * Fraction(2) ** (-sigma)
    out = []
    for _ in range(S):
        y = x * 128
        d = math.floor(y + Fraction(1, 2)) if y >= 0 else -math.floor(-y + Fraction(1, 2))
        out.append(int(d))
        x = y - d
    return out, x


@pytest.mark.parametrize("name,attr,fn", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_caught(monkeypatch, name, attr, fn):
    monkeypatch.setattr(OZ, attr, fn)
    failures = 0
    for t in (test_ties_round_to_even, test_scale_exponent_bounds,
              lambda: test_error_shrinks_per_slice_and_meets_bound("uniform")):
        try:
            t()
        except (AssertionError, ValueError):     # a crash inside the definition also exposes it
            failures += 1
    assert failures, name


@pytest.mark.parametrize("P", [3, 4])
def test_wide_truncation_and_digits(P):
    """TD/QD slicing input: each component floored at 2^(sigma - F - 64); the
    truncation is below the value by less than P units of that power, and the
    digits reconstruct the truncated value exactly."""
    rng = np.random.default_rng(510 + P)
    x = I.random_mp(P, 200, rng, spread=40)
    for t in range(x.shape[1]):
        comps = [float(c) for c in x[:, t]]
        for S in (3, 22, 40):
            sg = OZ.scale_exponent([comps[0]])
            tv = OZ.truncated_value(comps, sg, S)
            exact = X.value(comps)
            unit = Fraction(2) ** (sg - (7 * S + 12) - OZ.GUARD_BITS)
            assert 0 <= exact - tv < P * unit
            ds, rem = OZ.digits(comps, sg, S, truncate=True)
            recon = sum((Fraction(d) * Fraction(2) ** (-7 * (s + 1)) for s, d in enumerate(ds)), Fraction(0))
            assert (recon + rem * Fraction(2) ** (-7 * S)) * Fraction(2) ** sg == tv
            assert all(-64 <= d <= 64 for d in ds) and abs(rem) <= Fraction(1, 2)


def test_split_exact():
    """hi = RN(V) with ties to even, lo = V - hi exactly."""
    for V in (0, 1, -1, 2 ** 53 + 1, 2 ** 53 + 3, -(2 ** 60) - 2 ** 7 - 1, 2 ** 93 - 1, 3 * 2 ** 52 + 1):
        hi, lo = OZ.split_exact(V)
        assert Fraction(hi) + Fraction(lo) == V
        assert abs(Fraction(lo)) <= X.ulp(hi) / 2 if hi else lo == 0
    assert OZ.split_exact(2 ** 53 + 1) == (2.0 ** 53, 1.0)        # tie -> even
    assert OZ.split_exact(2 ** 53 + 3) == (2.0 ** 53 + 4, -1.0)   # tie -> even (up)


@pytest.mark.parametrize("prec", ["dd", "td", "qd"])
def test_first_group_add_is_the_identity(prec):
    """DDadd (Alg. 1), TDaddq (Sec. 2.3) and QDadd (Alg. 5) of zero and an exact
    split (hi 2^e, lo 2^e, 0, ...) return the split bit for bit: the tcgen05
    kernels store the first group of a tile without the addition, and this is
    why that changes no result."""
    P = {"dd": 2, "td": 3, "qd": 4}[prec]
    rng = np.random.default_rng(77)
    Vs = [0, 1, -1, 2 ** 53 + 1, 2 ** 53 + 3, -(2 ** 54) - 2, 2 ** 59 - 1, -(2 ** 59) + 1, 2 ** 52, 2 ** 53 - 1]
    Vs += [int(v) for v in rng.integers(-(2 ** 62), 2 ** 62, 4000)]
    Vs += [int(rng.integers(1, 2 ** 20)) << int(rng.integers(0, 40)) for _ in range(1000)]
    # ties and near-ties on both sides of a power of two
    Vs += [(1 << b) + (1 << (b - 54)) * t for b in range(55, 60) for t in (1, -1, 2, -2, 3, -3)]
    for V in Vs:
        hi, lo = OZ.split_exact(V)
        for e in (-300, -60, 0, 17):
            y = (math.ldexp(hi, e), math.ldexp(lo, e)) + (0.0,) * (P - 2)
            got = oracle.op(prec, "add", (0.0,) * P, y)
            assert [math.copysign(1, g) for g in got] == [math.copysign(1, v) for v in y] and got == y, (V, e, got, y)


def test_weight_groups():
    for S in (1, 2, 3, 4, 13, 22, 29, 40):
        for P in (2, 3, 4):
            groups = OZ.weight_groups(S, P)
            flat = [w for g in groups for w in g]
            assert flat == list(range(S + 1, 1, -1))
            G = OZ.group_size(P)
            assert all(len(g) == G for g in groups[:-1]) and 1 <= len(groups[-1]) <= G


@pytest.mark.parametrize("P,S", [(3, 22), (4, 29)])
def test_td_qd_error_meets_bound(P, S):
    rng = np.random.default_rng(520 + P)
    m, n, k = 6, 5, 40
    pbits = {3: 150, 4: 200}[P]
    for A, B in ((I.uniform(P, (m, k), rng), I.uniform(P, (k, n), rng)),
                 I.cancelling_pair(P, m, n, k, rng)):
        C, _, _ = OZ.gemm(A, B, S)
        err = X.gemm_error(C, A, B, [(i, j) for i in range(m) for j in range(n)])
        assert err["err_abs"] <= k * 2.0 ** -pbits, err
        # three fewer slices lose about 2^21
        C2, _, _ = OZ.gemm(A, B, S - 3)
        err2 = X.gemm_error(C2, A, B, [(i, j) for i in range(m) for j in range(n)])
        assert err2["err_abs"] > err["err_abs"] * 2.0 ** 10


def _rne_binary64(v):
    """The rational v rounded to binary64 by exact arithmetic: the nearest
    multiple of the spacing at |v| (2^-1074 below the normal range), ties to
    even, +-inf beyond the largest finite value; v = 0 gives +0."""
    if v == 0:
        return 0.0
    a = abs(v)
    ex = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** ex > a:
        ex -= 1                                         # 2^ex <= a < 2^(ex+1)
    sp = Fraction(2) ** max(ex - 52, -1074)
    q = a // sp
    r = a - q * sp
    if r > sp / 2 or (r == sp / 2 and q % 2 == 1):
        q += 1
    x = q * sp
    sign = -1.0 if v < 0 else 1.0
    if x > Fraction(float.fromhex("0x1.fffffffffffffp+1023")):
        return sign * math.inf
    return sign * float(x)


def test_scale2_rounds_like_ieee():
    """The group parts are scaled as ldexp: exact in the normal range, rounded
    to the nearest multiple of 2^-1074 (ties to even, signed zeros) below it,
    +-inf above it -- checked against exact rational rounding."""
    rng = np.random.default_rng(506)
    cases = [(1.0, -1074), (1.0, -1075), (3.0, -1076), (-3.0, -1076), (1.5, -1075), (2.5, -1075),
             (-1.0, -1076), (float(2 ** 53), -1127), (float(2 ** 53 - 1), -1126), (1.0, 1023),
             (1.0, 1024), (-float(2 ** 52 + 1), 972), (float(2 ** 52 + 1), 971)]
    for _ in range(3000):
        q = float(int(rng.integers(1, 2 ** 53)) * (1 if rng.uniform() < .5 else -1))
        e = int(rng.integers(-1180, -1000)) if rng.uniform() < .8 else int(rng.integers(900, 1000))
        cases.append((q, e))
    for x, e in cases:
        got = OZ.scale2(x, e)
        want = _rne_binary64(Fraction(x) * Fraction(2) ** e)
        if want == 0:
            want = math.copysign(0.0, x)                # a part that rounds to zero keeps its sign
        assert got == want and math.copysign(1, got) == math.copysign(1, want), (x, e, got, want)


def test_tiny_products_round_in_the_subnormal_range():
    """Rows of A and columns of B scaled by 2^-530 (and two rows of A by
    2^-1060, subnormal): products of two tiny factors fall below the normal
    range, so the group parts are rounded there; every entry stays within the
    slicing form's relative bound plus a few units of 2^-1074 per group of
    the exact product."""
    rng = np.random.default_rng(507)
    m, n, k, S = 6, 5, 24, 14
    A, B = I.uniform(2, (m, k), rng), I.uniform(2, (k, n), rng)
    A[:, :3] *= 2.0 ** -530
    A[:, 3:5] *= 2.0 ** -1060                           # subnormal leading components
    B[:, :, :2] *= 2.0 ** -530
    C, sig, tau = OZ.gemm(A, B, S)
    ex = X.ExactRows(A, B)
    groups = len(OZ.weight_groups(S, 2))
    tiny = 0
    for i in range(m):
        for j in range(n):
            err = abs(X.value(C[:, i, j]) - ex.dot(i, j))
            assert err <= k * Fraction(2) ** -100 * ex.absdot(i, j) + 4 * groups * Fraction(2) ** -1074, (i, j)
            tiny += abs(C[0, i, j]) < 2.0 ** -1022
    assert tiny >= 6                                    # the two-tiny-factor entries are subnormal
