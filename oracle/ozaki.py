"""Oracle for the INT8 error-free slicing forms of the DD/TD/QD GEMM --
TEST INFRASTRUCTURE ONLY (tests, smoke check and the benchmark's CPU leg).

The paper's GEMM (Sec. 3, Eq. 1) computed through an Ozaki-style error-free
splitting; every step is the plain definition, in Python integers, so a
reader can check it line by line.  DD (P = 2):

  scale    sigma_i = ilogb(max_p |hi(a_ip)|) + 2 for row i of A (0 for an
           all-zero row); tau_j likewise for column j of B.  Then
           |a_ip| 2^-sigma_i < 1/2.
  slices   x_0 = a 2^-sigma exactly; for s = 1..S: y = 2^7 x_{s-1},
           d_s = nearest integer to y (ties to even), x_s = y - d_s.
           Every |d_s| <= 64.  a = 2^sigma (sum_s d_s 2^-7s + 2^-7S x_S).
  products P_w = sum over s + t = w (1 <= s, t <= S) of A^(s) B^(t), for
           w = 2..S+1, computed exactly in integers.
  accumulate  weights are taken in groups of G = 5 from the least
           significant end (w = S+1, ..., S-3; then S-4, ...):
           V = sum_j P_(w-j) 2^(7j), an exact integer below 2^60; V is split
           exactly into hi = RN(V) (ties to even) and lo = V - hi;
           acc = (0, 0); for each group in that order:
           acc = DDadd(acc, (hi 2^e, lo 2^e)), e = sigma_i + tau_j - 7w, w
           the group's largest weight, with the oracle's DDadd (Alg. 1).  The
           scaled parts are C's ldexp of hi and lo: exact while they stay in
           the normal binary64 range (as for all but the tiniest or largest
           products), rounded to nearest (ties to even) below it, +-inf above.

TD and QD (P = 3, 4) differ in two places:
  slices   each component is first floored to a multiple of
           2^(sigma - F - 64), F = 7S + 12 (64 guard bits below the last
           digit's unit); the digits are those of the sum of the floored
           components, exactly as above.
  accumulate  as for DD with groups of G = 11 (TD; V below 2^102) or
           G = 10 (QD; V below 2^95) and TDaddq (Sec. 2.3) or QDadd (Alg. 5)
           of (hi 2^e, lo 2^e, 0, ...).
"""
import math
from fractions import Fraction

import numpy as np

from . import op as _op

BASE_BITS = 7


def _exact_int(x):
    """(M, E) with x == M * 2**E exactly, M an int."""
    if x == 0.0:
        return 0, 0
    f, e = math.frexp(x)
    return int(f * (1 << 53)), e - 53


def ilogb(x):
    return math.frexp(abs(x))[1] - 1


def scale_exponent(hi_values):
    """sigma for a row (or column) given its leading components."""
    mx = max((abs(float(v)) for v in hi_values), default=0.0)
    return 0 if mx == 0.0 else ilogb(mx) + 2


GUARD_BITS = 64


def truncated_value(components, sigma, S):
    """Sum of the components, each floored to a multiple of 2^(sigma - F - 64)
    with F = 7S + 12 (the TD/QD slicing input), as a Fraction."""
    q = sigma - (7 * S + 12) - GUARD_BITS
    tot = 0
    for c in components:
        M, E = _exact_int(float(c))
        sh = E - q
        tot += (M << sh) if sh >= 0 else (M >> -sh)    # Python >> floors
    return Fraction(tot) * Fraction(2) ** q


def digits(components, sigma, S, truncate=False):
    """The S balanced base-2^7 digits of (sum of components) * 2^-sigma and
    the exact remainder x_S (a Fraction).  With truncate, of the sum of the
    components floored as in truncated_value (TD/QD)."""
    if truncate:
        x = truncated_value(components, sigma, S) * Fraction(2) ** (-sigma)
    else:
        x = sum((Fraction(float(c)) for c in components), Fraction(0)) * Fraction(2) ** (-sigma)
    out = []
    for _ in range(S):
        y = x * (1 << BASE_BITS)
        d = round(y)              # Fraction.__round__: nearest, ties to even
        out.append(int(d))
        x = y - d
    return out, x


def slice_rows(planes, S, rows=None):
    """planes (P, m, k).  Returns sigma (list per row) and D with
    D[s-1][r][p] the s-th digit of element (rows[r], p)."""
    planes = np.asarray(planes)
    rows = range(planes.shape[1]) if rows is None else rows
    truncate = planes.shape[0] > 2
    sig, D = [], np.zeros((S, len(rows), planes.shape[2]), dtype=np.int64)
    for r, i in enumerate(rows):
        sg = scale_exponent(planes[0, i, :])
        sig.append(sg)
        for p in range(planes.shape[2]):
            ds, _ = digits(planes[:, i, p], sg, S, truncate)
            D[:, r, p] = ds
    return sig, D


def slice_cols(planes, S, cols=None):
    """planes (P, k, n): slices of the columns of B (as rows of B^T)."""
    planes = np.asarray(planes)
    return slice_rows(np.ascontiguousarray(planes.transpose(0, 2, 1)), S, cols)


def weight_products(DA, DB, S):
    """P_w for w = 2..S+1: dict w -> integer matrix (rows of DA x rows of DB).
    Exact in int64: every |digit| <= 64, so |P_w| <= S k 2^12, far below 2^63
    for any k the slicing form accepts."""
    k = DA.shape[2]
    assert S * k * 64 * 64 < 2 ** 62
    DA = DA.astype(np.int64)
    DB = DB.astype(np.int64)
    out = {}
    for w in range(2, S + 2):
        acc = np.zeros((DA.shape[1], DB.shape[1]), dtype=np.int64)
        for s in range(max(1, w - S), min(S, w - 1) + 1):
            t = w - s
            acc = acc + DA[s - 1].dot(DB[t - 1].T)
        out[w] = acc
    return out


PREC_OF = {2: "dd", 3: "td", 4: "qd"}


def group_size(P):
    """Weights combined exactly per add: 5 for DD (64-bit sums), 11 for TD and
    10 for QD (128-bit sums; 11 TD weights make the default 22 two groups)."""
    return {2: 5, 3: 11, 4: 10}[P]


def weight_groups(S, P):
    """The weights in accumulation order, group_size(P) to a group, from the
    least significant (w = S+1) end (the last group may be shorter)."""
    ws = list(range(S + 1, 1, -1))
    G = group_size(P)
    return [ws[i:i + G] for i in range(0, len(ws), G)]


def split_exact(V):
    """(hi, lo) with hi = RN(V) (ties to even) and lo = V - hi, both exact
    binary64 values, for an integer |V| < 2^106."""
    hi = float(V)                      # Python rounds int -> float to nearest, ties to even
    lo = V - int(hi)
    assert abs(lo) < 2 ** 53 and float(lo) == lo
    return hi, float(lo)


def scale2(x, e):
    """x 2^e as binary64, as C's ldexp: exact in the normal range; below it
    the nearest multiple of 2^-1074 (ties to even; a zero keeps the sign of
    x); above it +-inf."""
    try:
        return math.ldexp(x, e)
    except OverflowError:
        return math.copysign(math.inf, x)


def _in_normal_range(x, v):
    return x == 0 or 2.0 ** -1022 <= abs(v) < math.inf


def gemm(A, B, S, rows=None, cols=None, L=None):
    """C = A B through S-slice error-free splitting, for the selected rows of
    A and columns of B (all by default).  A (P, m, k), B (P, k, n), P = 2, 3
    or 4.  Returns C (P, len(rows), len(cols)), sigma, tau."""
    A = np.asarray(A)
    B = np.asarray(B)
    P = A.shape[0]
    prec = PREC_OF[P]
    rows = list(range(A.shape[1])) if rows is None else list(rows)
    cols = list(range(B.shape[2])) if cols is None else list(cols)
    sig, DA = slice_rows(A, S, rows)
    tau, DB = slice_cols(B, S, cols)
    Pw = weight_products(DA, DB, S)
    C = np.zeros((P, len(rows), len(cols)))
    for r in range(len(rows)):
        for c in range(len(cols)):
            acc = (0.0,) * P
            for grp in weight_groups(S, P):
                wmax = grp[0]
                V = sum(int(Pw[w][r, c]) << (BASE_BITS * (wmax - w)) for w in grp)
                assert abs(V) < {2: 2 ** 60, 3: 2 ** 102, 4: 2 ** 95}[P]
                hi, lo = split_exact(V)
                e = sig[r] + tau[c] - BASE_BITS * wmax
                vh, vl = scale2(hi, e), scale2(lo, e)
                if _in_normal_range(hi, vh) and _in_normal_range(lo, vl):
                    assert Fraction(vh) + Fraction(vl) == Fraction(V) * Fraction(2) ** e, "scaled group sum not exact"
                acc = _op(prec, "add", acc, (vh, vl) + (0.0,) * (P - 2), L)
            C[:, r, c] = acc
    return C, sig, tau


def max_pairs(S):
    return S


def k_limit(S):
    """Largest k for which every weight's INT32 sum is exact:
    pairs * k * 64 * 64 < 2^31."""
    return (2 ** 31 - 1) // (max_pairs(S) * 64 * 64)
