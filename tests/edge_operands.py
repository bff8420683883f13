"""Seeded operand pairs for the error-free transformations, in classes that
reach every branch of their integer-pipe form (no arithmetic of the method
here: bit patterns, exponent ranges and signs only)."""
import numpy as np


def _bits_to_f64(u):
    return np.asarray(u, dtype=np.uint64).view(np.float64)


def edge_operands(n, rng):
    """a, b of 10 * n elements in ten classes: any bit pattern (NaN and
    infinity included), moderate, tiny (subnormal), huge, near-cancelling,
    exponent gaps 0-70 in either order, products near the subnormal and the
    overflow boundaries, zeros of both signs among small values, and short
    significands (ties)."""
    def bits(k):
        return rng.integers(0, 2 ** 64 - 1, k, dtype=np.uint64, endpoint=True)

    def with_exp(k, lo, hi):
        m = bits(k) & np.uint64(0x800FFFFFFFFFFFFF)
        e = rng.integers(lo, hi + 1, k).astype(np.uint64) << np.uint64(52)
        return _bits_to_f64(m | e)

    A, B = [], []
    a, b = _bits_to_f64(bits(n)), _bits_to_f64(bits(n))
    special = np.array([np.inf, -np.inf, np.nan, 0.0, -0.0])
    a[::97] = special[rng.integers(0, 5, a[::97].size)]
    b[::89] = special[rng.integers(0, 5, b[::89].size)]
    A.append(a); B.append(b)
    A.append(with_exp(n, 1003, 1043)); B.append(with_exp(n, 1003, 1043))
    A.append(with_exp(n, 0, 60)); B.append(with_exp(n, 0, 60))
    A.append(with_exp(n, 2000, 2046)); B.append(with_exp(n, 1003, 2046))
    a = with_exp(n, 1003, 1043)
    b = _bits_to_f64((a.view(np.uint64) ^ np.uint64(1 << 63))
                     + rng.integers(-32, 33, n).astype(np.int64).view(np.uint64))
    A.append(a); B.append(b)
    a = with_exp(n, 1003, 1043)
    b = np.ldexp(with_exp(n, 1023, 1023), -rng.integers(0, 71, n)) * np.abs(a)
    sw = rng.integers(0, 2, n).astype(bool)
    A.append(np.where(sw, b, a)); B.append(np.where(sw, a, b))
    A.append(np.ldexp(1.0 + rng.random(n), -rng.integers(480, 600, n)) * rng.choice([-1.0, 1.0], n))
    B.append(np.ldexp(1.0 + rng.random(n), -rng.integers(480, 600, n)))
    A.append(np.ldexp(1.0 + rng.random(n), rng.integers(500, 530, n)))
    B.append(np.ldexp(1.0 + rng.random(n), rng.integers(490, 530, n)) * rng.choice([-1.0, 1.0], n))
    small = np.array([0.0, -0.0, 1.0, -1.0, 5e-324, -5e-324])
    a = small[rng.integers(0, 6, n)]
    a = np.where(rng.integers(0, 2, n).astype(bool), with_exp(n, 1003, 1043), a)
    b = small[rng.integers(0, 6, n)]
    sw = rng.integers(0, 2, n).astype(bool)
    A.append(np.where(sw, b, a)); B.append(np.where(sw, a, b))
    a = rng.integers(0, 2 ** 53, n).astype(np.float64) * np.ldexp(1.0, -rng.integers(0, 60, n))
    b = np.ldexp(1.0, rng.integers(-30, 30, n)) * rng.choice([1.5, -1.0], n)
    A.append(a); B.append(b)
    return np.concatenate(A), np.concatenate(B)


def same_bits(x, y):
    """Bit-identical, any two NaNs counting as equal."""
    x, y = np.asarray(x), np.asarray(y)
    return (x.view(np.uint64) == y.view(np.uint64)) | (np.isnan(x) & np.isnan(y))
