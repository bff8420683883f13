"""Exact rational arithmetic on binary64 expansions -- TEST INFRASTRUCTURE ONLY.

The definition of C := A B (Eq. 1) written out exactly: every binary64 is
m * 2**e with integer m, so sums and products of multi-component numbers are
computed without rounding as Python integers.  Used to pin the oracle and to
check the GPU results against the exact product within an error bound.
"""
import math
from fractions import Fraction

import numpy as np


def frac(x):
    """Exact value of a finite binary64 as a Fraction."""
    return Fraction(float(x))


def value(components):
    """Exact value of a multi-component number (sequence of binary64)."""
    return sum((Fraction(float(c)) for c in components), Fraction(0))


def ulp(x):
    """Unit in the last place of a finite nonzero binary64 (spacing at |x|)."""
    return Fraction(float(np.spacing(abs(float(x)))))


def _mant_exp(planes):
    """Integer mantissas and exponents: planes == mant * 2**exp, elementwise."""
    f, e = np.frexp(np.asarray(planes, dtype=np.float64))
    mant = np.ldexp(f, 53).astype(np.int64)    # exact: f * 2**53 is an integer
    return mant, (e - 53).astype(np.int64)


class ExactRows:
    """Exact integer images of selected rows of A and columns of B.

    A_planes: (P, m, k), B_planes: (P, k, n).  ``dot(i, j)`` returns the exact
    value of sum_k a_ik b_kj as a Fraction, ``absdot(i, j)`` the exact value of
    sum_k |a_ik| |b_kj|.
    """

    def __init__(self, A_planes, B_planes):
        self.A = np.asarray(A_planes, dtype=np.float64)
        self.B = np.asarray(B_planes, dtype=np.float64)
        self._rows = {}
        self._cols = {}

    @staticmethod
    def _scaled(vecs):
        # vecs: (P, k).  Returns (list of ints, E) with vec_total[t] = ints[t] * 2**E.
        mant, ex = _mant_exp(vecs)
        nz = mant != 0
        E = int(ex[nz].min()) if nz.any() else 0
        P, k = vecs.shape
        out = [0] * k
        for c in range(P):
            mc, ec = mant[c], ex[c]
            for t in range(k):
                m = int(mc[t])
                if m:
                    out[t] += m << (int(ec[t]) - E)
        return out, E

    def row(self, i):
        if i not in self._rows:
            self._rows[i] = self._scaled(self.A[:, i, :])
        return self._rows[i]

    def col(self, j):
        if j not in self._cols:
            self._cols[j] = self._scaled(self.B[:, :, j])
        return self._cols[j]

    def dot(self, i, j):
        a, ea = self.row(i)
        b, eb = self.col(j)
        s = sum(x * y for x, y in zip(a, b))
        return Fraction(s) * Fraction(2) ** (ea + eb)

    def absdot(self, i, j):
        a, ea = self.row(i)
        b, eb = self.col(j)
        s = sum(abs(x) * abs(y) for x, y in zip(a, b))
        return Fraction(s) * Fraction(2) ** (ea + eb)


def gemm_error(C_planes, A_planes, B_planes, entries):
    """Errors of a computed product on the given (i, j) entries.

    Returns a dict with
      err_abs  = ||C_hat - C||_F / || |A||B| ||_F   (normwise, the pass/fail metric)
      err_rel  = ||C_hat - C||_F / ||C||_F
      max_abs  = max |c_hat - c| / (|A||B|)_ij
    all as floats, the norms taken over ``entries``.
    """
    ex = ExactRows(A_planes, B_planes)
    C = np.asarray(C_planes)
    num = Fraction(0)
    den_abs = Fraction(0)
    den_c = Fraction(0)
    worst = 0.0
    for (i, j) in entries:
        c = ex.dot(i, j)
        ab = ex.absdot(i, j)
        d = value(C[:, i, j]) - c
        num += d * d
        den_abs += ab * ab
        den_c += c * c
        if ab:
            worst = max(worst, float(abs(d) / ab))
    def ratio(a, b):
        if b == 0:
            return 0.0 if a == 0 else math.inf
        return math.sqrt(float(a / b))
    return {"err_abs": ratio(num, den_abs), "err_rel": ratio(num, den_c), "max_abs": worst}


def sample_entries(m, n, count, rng, full_rows=2):
    """Seeded sample of (i, j) entries: ``count`` random ones plus whole rows."""
    ent = set()
    if m and n:
        for _ in range(count):
            ent.add((int(rng.integers(m)), int(rng.integers(n))))
        for r in rng.choice(m, size=min(full_rows, m), replace=False):
            for j in range(n):
                ent.add((int(r), j))
    return sorted(ent)
