"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module draws random numbers and lays them out; it contains none of the
multi-component arithmetic.  A P-component number is built already normalised
by construction: each lower component is u * ulp(previous)/2 with u uniform in
(-1, 1), an exact power-of-two scaling, so |c_{i+1}| < ulp(c_i)/2 and
fl(c_i + c_{i+1}) = c_i without any renormalisation step.

Layout: structure-of-arrays planes, shape (P, rows, cols), row-major, float64,
component 0 the most significant (Sec. 2.5, Fig. 1).
"""
import math
from fractions import Fraction

import numpy as np

P_OF = {"dd": 2, "td": 3, "qd": 4}
SEED_BASE = 20210117


def rng_for(cfg):
    """The generator for workload ``cfg`` (0..4): PCG64(20210117 + cfg)."""
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(cfg)))


def _open_unit(rng, shape):
    """Uniform in the open interval (-1, 1)."""
    u = rng.uniform(-1.0, 1.0, size=shape)
    return np.where(u == -1.0, 0.0, u)


def _half_ulp(x):
    return np.spacing(np.abs(x)) * 0.5


def expand(lead, P, rng):
    """Planes (P, ...) whose component 0 is ``lead`` and each lower component is
    u * ulp(previous)/2, u uniform in (-1, 1)."""
    lead = np.asarray(lead, dtype=np.float64)
    out = np.empty((P,) + lead.shape)
    out[0] = lead
    for c in range(1, P):
        out[c] = _open_unit(rng, lead.shape) * _half_ulp(out[c - 1])
        out[c][out[c - 1] == 0.0] = 0.0
    return out


def uniform(P, shape, rng):
    """Leading component uniform in [-1, 1); lower components as in ``expand``."""
    return expand(rng.uniform(-1.0, 1.0, size=shape), P, rng)


def ill_scaled(P, shape, rng, emin=-20, emax=20):
    """Leading component (2r - 1) * 2**e, r uniform [0, 1), e a uniform integer in
    [emin, emax]; lower components as in ``expand``."""
    r = rng.uniform(0.0, 1.0, size=shape)
    e = rng.integers(emin, emax + 1, size=shape)
    return expand(np.ldexp(2.0 * r - 1.0, e), P, rng)


def cancelling_pair(P, m, n, k, rng):
    """A (P,m,k), B (P,k,n) with forced cancellation inside every c_ij.

    Ill-scaled entries; for the second half of the inner dimension, row p of B
    repeats the leading component of row p - k/2 and column p of A repeats the
    negated leading component of column p - k/2, each with fresh lower
    components, so the two halves of each dot product nearly cancel.
    """
    A = ill_scaled(P, (m, k), rng)
    B = ill_scaled(P, (k, n), rng)
    h = k // 2
    if h:
        A[:, :, k - h:] = expand(-A[0][:, :h], P, rng)
        B[:, k - h:, :] = expand(B[0][:h, :], P, rng)
    return A, B


def _sqrt_expansion(c, t, P, bits=64 * 8):
    """P-component expansion of t*sqrt(c) (t >= 0 integer): each component is the
    correctly rounded value of what the previous ones leave, from an exact
    integer square root carried to ``bits`` fractional bits."""
    if t == 0:
        return [0.0] * P
    V = math.isqrt(c * t * t << (2 * bits))      # floor(t*sqrt(c) * 2**bits)
    rest = Fraction(V, 1 << bits)
    comps = []
    for _ in range(P):
        x = float(rest)                            # correctly rounded
        comps.append(x)
        rest -= Fraction(x)
    return comps


def paper_matrices(P, n):
    """The test matrices of Sec. 3: A = [sqrt(5)(i+j-1)], B = [sqrt(3)(n-i)]
    (1-based), as correctly rounded P-component expansions."""
    a_vals = {t: _sqrt_expansion(5, t, P) for t in range(1, 2 * n)}
    b_vals = {t: _sqrt_expansion(3, t, P) for t in range(0, n)}
    A = np.empty((P, n, n))
    B = np.empty((P, n, n))
    for i in range(n):
        for j in range(n):
            A[:, i, j] = a_vals[i + j + 1]
        B[:, i, :] = np.asarray(b_vals[n - 1 - i])[:, None]
    return A, B


def paper_closed_form(n, i):
    """Integer N with c_ij = sqrt(15) * N for the Sec. 3 matrices (1-based i):
    sum_k (i-1+k)(n-k) = (i-1) n(n-1)/2 + (n-1) n (n+1)/6, independent of j."""
    return (i - 1) * n * (n - 1) // 2 + (n - 1) * n * (n + 1) // 6


def batch_shapes(count, rng, lo=16, hi=512):
    """``count`` (m, n, k) triples, each dimension a log-uniform integer in [lo, hi]."""
    def draw():
        x = np.exp(rng.uniform(np.log(lo), np.log(hi + 1), size=count))
        return np.clip(np.floor(x).astype(np.int64), lo, hi)
    m, n, k = draw(), draw(), draw()
    return [(int(a), int(b), int(c)) for a, b, c in zip(m, n, k)]


def random_mp(P, n, rng, spread=30):
    """Elementwise-test operands: leading components with random signs and
    exponents over +-spread, lower components as in ``expand``."""
    return ill_scaled(P, (n,), rng, -spread, spread)


def edge_mp(P):
    """Hand-picked operand pairs (x, y), each (P, count): zeros of both signs,
    exact cancellation, equal magnitudes, far exponents, ties, powers of two,
    values near the bottom of the normal range, subnormal values and products
    that fall into or below the subnormal range."""
    rows_x, rows_y = [], []
    tiny = 2.0 ** -900
    lead_pairs = [
        (0.0, 0.0), (-0.0, 0.0), (-0.0, -0.0), (1.0, -1.0), (1.0, 1.0),
        (1.0, 2.0 ** -53), (1.0, 2.0 ** -54), (1.0, -2.0 ** -53), (1.0 + 2.0 ** -52, -1.0),
        (2.0 ** 500, 2.0 ** -500), (3.0, 1.0 / 3.0), (0.1, 0.2), (-0.7, 0.7 + 2.0 ** -53),
        (tiny, tiny), (tiny, -tiny * 0.75), (2.0 ** 30, -2.0 ** 30 + 1.0),
        (1.5, 1.5), (math.pi, math.e), (-math.pi, 1e-30), (2.0 ** -60, 2.0 ** 60),
        (2.0 ** -1060, 2.0 ** -1062), (2.0 ** -1074, -2.0 ** -1074), (3 * 2.0 ** -1074, 2.0 ** -1073),
        (2.0 ** -540 * 1.25, -2.0 ** -540 * 1.75), (2.0 ** -1000, -2.0 ** -1001 * 1.5),
        (2.0 ** -600, 2.0 ** -600), (-2.0 ** -1022, 2.0 ** -1023),
    ]
    for (a, b) in lead_pairs:
        xa = [a] + [0.0] * (P - 1)
        yb = [b] + [0.0] * (P - 1)
        rows_x.append(xa)
        rows_y.append(yb)
        # the same leads with full lower components
        xa2, yb2 = [a], [b]
        for c in range(1, P):
            xa2.append(xa2[-1] * 2.0 ** -53 * 0.375 if xa2[-1] else 0.0)
            yb2.append(-yb2[-1] * 2.0 ** -53 * 0.3125 if yb2[-1] else 0.0)
        rows_x.append(xa2)
        rows_y.append(yb2)
    x = np.asarray(rows_x, dtype=np.float64).T.copy()
    y = np.asarray(rows_y, dtype=np.float64).T.copy()
    return x, y
