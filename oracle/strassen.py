"""Oracle of the Strassen form of the DD/TD/QD GEMM -- TEST INFRASTRUCTURE ONLY.

Sec. 3 of the paper runs C := AB either by the block algorithm (Eq. 1 per
entry, k ascending) or by Strassen's divide-and-conquer: for even dimensions
A and B are cut into four blocks each and C is assembled from seven block
products.  The figure with the formulas is not in the text; this oracle takes
Strassen's original seven products (Strassen 1969), written out below, with
the same multi-component arithmetic as the rest of the method:

  M1 = (A11 + A22)(B11 + B22)     M5 = (A11 + A12) B22
  M2 = (A21 + A22) B11            M6 = (A21 - A11)(B11 + B12)
  M3 = A11 (B12 - B22)            M7 = (A12 - A22)(B21 + B22)
  M4 = A22 (B21 - B11)
  C11 = ((M1 + M4) - M5) + M7     C12 = M3 + M5
  C21 = M2 + M4                   C22 = ((M1 - M2) + M3) + M6

Readings fixed here:
  - "+" is the precision's GEMM addition, elementwise: DDadd (Alg. 1),
    TDaddq (Sec. 2.3), QDadd (Alg. 5); x - y is x + (-y), -y negating every
    component;
  - each sum above is evaluated left to right;
  - the recursion runs `levels` times and stops early when m, n or k is odd
    or zero; the leaf products are the k-sequential GEMM (Eq. 1), which is
    also what the paper's block algorithm gives per entry.
"""
import numpy as np

from . import gemm as _gemm
from . import vec_op as _vec_op


def _add(prec, x, y):
    shape = x.shape
    P = shape[0]
    r = _vec_op(prec, "add", np.ascontiguousarray(x).reshape(P, -1), np.ascontiguousarray(y).reshape(P, -1))
    return r.reshape(shape)


def _sub(prec, x, y):
    return _add(prec, x, -np.asarray(y))


def strassen(prec, A, B, levels):
    """C = A B for planes A (P, m, k), B (P, k, n) by `levels` levels of
    Strassen's algorithm over the k-sequential GEMM."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    _, m, k = A.shape
    n = B.shape[2]
    if levels <= 0 or m % 2 or n % 2 or k % 2 or min(m, n, k) == 0:
        return _gemm(prec, A, B)
    m2, n2, k2 = m // 2, n // 2, k // 2
    A11, A12, A21, A22 = A[:, :m2, :k2], A[:, :m2, k2:], A[:, m2:, :k2], A[:, m2:, k2:]
    B11, B12, B21, B22 = B[:, :k2, :n2], B[:, :k2, n2:], B[:, k2:, :n2], B[:, k2:, n2:]
    add = lambda x, y: _add(prec, x, y)
    sub = lambda x, y: _sub(prec, x, y)
    rec = lambda x, y: strassen(prec, x, y, levels - 1)
    M1 = rec(add(A11, A22), add(B11, B22))
    M2 = rec(add(A21, A22), B11)
    M3 = rec(A11, sub(B12, B22))
    M4 = rec(A22, sub(B21, B11))
    M5 = rec(add(A11, A12), B22)
    M6 = rec(sub(A21, A11), add(B11, B12))
    M7 = rec(sub(A12, A22), add(B21, B22))
    C = np.empty((A.shape[0], m, n))
    C[:, :m2, :n2] = add(sub(add(M1, M4), M5), M7)
    C[:, :m2, n2:] = add(M3, M5)
    C[:, m2:, :n2] = add(M2, M4)
    C[:, m2:, n2:] = add(add(sub(M1, M2), M3), M6)
    return C
