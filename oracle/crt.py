"""Oracle for the CRT form of the DD/TD/QD GEMM (Ozaki scheme II) -- TEST
INFRASTRUCTURE ONLY (tests, smoke check and the benchmark's CPU leg).

Not in the paper: the product of Sec. 3 (Eq. 1) computed with the scaled
operands turned into integers, the integer product recovered exactly from its
residues modulo N small pairwise coprime moduli (Chinese remainder theorem),
each residue product running on the tensor cores.  Every step is the plain
definition in Python integers:

  scale    sigma_i = ilogb(max_p |a_ip[0]|) + 2 for row i of A (0 for an
           all-zero row), tau_j likewise for column j of B, so that
           |a_ip| 2^-sigma_i < 1/2.
  integers A'_ip = the nearest integer (ties to even) of the sum of the
           components of a_ip, each first floored to a multiple of
           2^(sigma_i - beta - 64), in units of 2^(sigma_i - beta)
           (the floor, 64 bits below the unit, is part of the definition and
           moves A' only when the exact value lies within about 2^-62 units
           of a half); |A'| <= 2^(beta - 1).  B' likewise with tau_j.
  moduli   m_1, ..., m_N: the first N of MODULI, pairwise coprime integers
           <= 256 taken greedily from 256 downward; M = m_1 ... m_N.
  bits     beta = the largest integer with k 2^(2 beta - 1) < M, so that
           |A' B'| <= k 2^(2 beta - 2) < M / 2 (beta >= 1 is required).
  residues r(x, m) = the representative of x mod m in [-floor(m/2),
           ceil(m/2) - 1]; |r| <= 128, exact in int8 and in bf16.
  products Q_i = r(A', m_i) r(B', m_i)^T, exact integers
           (|Q_i| <= k 2^14 < 2^31 for k < 2^17).
  recover  C' = the integer in [-M/2, M/2) with C' = Q_i mod m_i for every
           i (C' = A'B' exactly).
  output   v = C' 2^(sigma_i + tau_j - 2 beta); the P components are
           c_0 = RN(v), c_1 = RN(v - c_0), ..., each the nearest binary64
           (ties to even) of the exact remainder.

The result is deterministic; its error against the exact product comes from
rounding the scaled entries to integers (about 2^-beta relative to the row
and column scales) and from the final rounding to P components.

Split integers (halves = 2), for more bits than the moduli's product allows
one integer product to carry:
  bits     w = the largest integer with k 2^(2w) < M; beta = 2w.
  split    A' = A1 2^w + A0 with A0 = the representative of A' mod 2^w in
           [-2^(w-1), 2^(w-1)) and A1 = (A' - A0) / 2^w (|A1| <= 2^(w-1));
           B' likewise.
  products Q_hh,i = r(A1) r(B1)^T, Q_mid,i = r(A1) r(B0)^T + r(A0) r(B1)^T,
           Q_ll,i = r(A0) r(B0)^T (|Q| <= 2k 2^14 < 2^31 for k < 2^16).
  recover  P_hh, P_mid, P_ll in [-M/2, M/2) from their residues (each is
           below k 2^(2w-1) < M/2 in magnitude).
  output   C' = P_hh 2^(2w) + P_mid 2^w + P_ll (= A'B' exactly), rounded as
           above.
"""
import math
from fractions import Fraction

import numpy as np


def _coprime_moduli(limit=256, count=64):
    out = []
    m = limit
    while m > 1 and len(out) < count:
        if all(math.gcd(m, x) == 1 for x in out):
            out.append(m)
        m -= 1
    return out


MODULI = _coprime_moduli()
RES_BITS = 14            # |r(a) r(b)| <= 128 * 128 = 2^14


def k_limit(halves=1):
    """Largest k whose residue products (two of them summed for the middle
    product of split integers) sum exactly in int32."""
    return (2 ** 31 - 1) // (halves * (1 << RES_BITS))


def modulus_product(N):
    return math.prod(MODULI[:N])


def beta_bits(N, k, halves=1):
    """The largest beta with k 2^(2 beta - 1) < M (0 if none); with split
    integers beta = 2w for the largest w with k 2^(2w) < M."""
    M = modulus_product(N)
    if halves == 2:
        w = 0
        while max(k, 1) * 2 ** (2 * (w + 1)) < M:
            w += 1
        return 2 * w
    b = 0
    while max(k, 1) * 2 ** (2 * (b + 1) - 1) < M:
        b += 1
    return b


def split(x, w):
    """(x1, x0) with x = x1 2^w + x0, x0 in [-2^(w-1), 2^(w-1))."""
    x0 = x % (1 << w)
    if x0 >= 1 << (w - 1):
        x0 -= 1 << w
    return (x - x0) >> w, x0


def sym_mod(x, m):
    """Representative of x mod m in [-floor(m/2), ceil(m/2) - 1]."""
    r = x % m
    return r - m if r >= (m + 1) // 2 else r


def ilogb(x):
    return math.frexp(abs(x))[1] - 1


def scale_exponent(hi_values):
    mx = max((abs(float(v)) for v in hi_values), default=0.0)
    return 0 if mx == 0.0 else ilogb(mx) + 2


GUARD = 64


def scaled_integer(components, shift):
    """Nearest integer (ties to even) of the sum of the components times
    2^shift, each component first floored to a multiple of 2^-64 in those
    units."""
    W = sum(math.floor(Fraction(float(c)) * Fraction(2) ** (shift + GUARD)) for c in components)
    return round(Fraction(W, 2 ** GUARD))          # Fraction.__round__: nearest, ties to even


def integer_rows(planes, beta):
    """planes (P, r, k): exponents (list) and the integers A' (list of lists)."""
    planes = np.asarray(planes)
    sig, rows = [], []
    for i in range(planes.shape[1]):
        s = scale_exponent(planes[0, i, :])
        sig.append(s)
        rows.append([scaled_integer(planes[:, i, p], beta - s) for p in range(planes.shape[2])])
    return sig, rows


def nearest_expansion(v, P):
    """The P components c_t = RN(v - c_0 - ... - c_(t-1)) of an exact rational v."""
    out = []
    rest = Fraction(v)
    for _ in range(P):
        try:
            c = float(rest)                    # correctly rounded, ties to even
        except OverflowError:
            c = math.copysign(math.inf, rest)
        out.append(c)
        if not math.isfinite(c):
            rest = Fraction(0)
        else:
            rest -= Fraction(c)
    return out


def crt_recover(residues, N):
    """The integer in [-M/2, M/2) congruent to residues[i] mod MODULI[i]."""
    M = modulus_product(N)
    x = 0
    for i in range(N):
        m = MODULI[i]
        Mi = M // m
        x += residues[i] * Mi * pow(Mi, -1, m)
    x %= M
    return x - M if x >= (M + 1) // 2 else x


def residues(planes, N, beta):
    """planes (P, r, k): exponents and the residues [N][r][k] of the integers."""
    sig, rows = integer_rows(planes, beta)
    return sig, np.array([[[sym_mod(a, MODULI[i]) for a in row] for row in rows] for i in range(N)],
                         dtype=np.int64).reshape(N, len(rows), np.asarray(planes).shape[2])


def _res(vals, N):
    """int64 array [N][len(vals)][k] of the residues of a list of integer rows."""
    return np.array([[[sym_mod(a, MODULI[i]) for a in row] for row in vals] for i in range(N)],
                    dtype=np.int64).reshape(N, len(vals), len(vals[0]) if vals else 0)


def gemm2(A, B, N, rows=None, cols=None):
    """C = A B through the CRT form with split integers (halves = 2).  As gemm;
    returns C, sigma, tau and beta = 2w."""
    A = np.asarray(A)
    B = np.asarray(B)
    P = A.shape[0]
    k = A.shape[2]
    rows = list(range(A.shape[1])) if rows is None else list(rows)
    cols = list(range(B.shape[2])) if cols is None else list(cols)
    beta = beta_bits(N, k, halves=2)
    w = beta // 2
    assert w >= 1, "too few moduli for this k"
    sig, Ai = integer_rows(A[:, rows, :], beta)
    tau, Bi = integer_rows(np.ascontiguousarray(B[:, :, cols].transpose(0, 2, 1)), beta)
    A1 = [[split(a, w)[0] for a in row] for row in Ai]
    A0 = [[split(a, w)[1] for a in row] for row in Ai]
    B1 = [[split(b, w)[0] for b in row] for row in Bi]
    B0 = [[split(b, w)[1] for b in row] for row in Bi]
    RA1, RA0, RB1, RB0 = _res(A1, N), _res(A0, N), _res(B1, N), _res(B0, N)
    Qhh = np.einsum("irk,ick->irc", RA1, RB1)
    Qmid = np.einsum("irk,ick->irc", RA1, RB0) + np.einsum("irk,ick->irc", RA0, RB1)
    Qll = np.einsum("irk,ick->irc", RA0, RB0)
    C = np.zeros((P, len(rows), len(cols)))
    for r in range(len(rows)):
        for c in range(len(cols)):
            hh, mid, ll = (crt_recover([int(Q[i, r, c]) % MODULI[i] for i in range(N)], N)
                           for Q in (Qhh, Qmid, Qll))
            Cp = (hh << (2 * w)) + (mid << w) + ll
            v = Fraction(Cp) * Fraction(2) ** (sig[r] + tau[c] - 2 * beta)
            C[:, r, c] = nearest_expansion(v, P)
    return C, sig, tau, beta


def gemm(A, B, N, rows=None, cols=None, halves=1):
    """C = A B through the CRT form with N moduli, for the selected rows of A
    and columns of B (all by default).  A (P, m, k), B (P, k, n).  Returns
    C (P, len(rows), len(cols)), sigma, tau and beta.  halves = 2: split
    integers (gemm2)."""
    if halves == 2:
        return gemm2(A, B, N, rows, cols)
    A = np.asarray(A)
    B = np.asarray(B)
    P = A.shape[0]
    k = A.shape[2]
    rows = list(range(A.shape[1])) if rows is None else list(rows)
    cols = list(range(B.shape[2])) if cols is None else list(cols)
    beta = beta_bits(N, k)
    assert beta >= 1, "too few moduli for this k"
    sig, Ai = integer_rows(A[:, rows, :], beta)
    tau, Bi = integer_rows(np.ascontiguousarray(B[:, :, cols].transpose(0, 2, 1)), beta)
    # residues as int64 arrays [N][rows][k] and [N][cols][k]; the products are
    # exact in int64 (|Q_i| <= k 2^14)
    RA = np.array([[[sym_mod(a, MODULI[i]) for a in Ai[r]] for r in range(len(rows))] for i in range(N)],
                  dtype=np.int64).reshape(N, len(rows), k)
    RB = np.array([[[sym_mod(b, MODULI[i]) for b in Bi[c]] for c in range(len(cols))] for i in range(N)],
                  dtype=np.int64).reshape(N, len(cols), k)
    Q = np.einsum("irk,ick->irc", RA, RB)
    C = np.zeros((P, len(rows), len(cols)))
    for r in range(len(rows)):
        for c in range(len(cols)):
            Cp = crt_recover([int(Q[i, r, c]) % MODULI[i] for i in range(N)], N)
            v = Fraction(Cp) * Fraction(2) ** (sig[r] + tau[c] - 2 * beta)
            C[:, r, c] = nearest_expansion(v, P)
    return C, sig, tau, beta
