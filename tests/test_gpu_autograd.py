"""DDMatmul gradients on the GPU (m = n = k = 2048, loss = sum(W * C)):
bit-identical to the oracle's DD products dC B^T and A^T dC on sampled rows,
and within n 2^-100 of QD central finite differences (h = 2^-40, computed by
the CPU oracle) on 64 sampled entries of each gradient."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from gpu_util import assert_bitwise, dev, host, torch_cuda
from oracle import exact as X
from paper_2101_06584_gb300 import inputs as I

pytestmark = pytest.mark.gpu
H = 2.0 ** -40


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def _qd(dd):
    z = np.zeros((4,) + dd.shape[1:])
    z[:2] = dd
    return z


def test_small_gradients_bitwise(torch):
    from paper_2101_06584_gb300.autograd import dd_matmul
    rng = np.random.default_rng(800)
    A, B, W = I.uniform(2, (37, 45), rng), I.uniform(2, (45, 29), rng), I.uniform(2, (37, 29), rng)
    Ad = dev(torch, A).requires_grad_(True)
    Bd = dev(torch, B).requires_grad_(True)
    C = dd_matmul(Ad, Bd)
    C.backward(dev(torch, W))
    assert_bitwise(host(C.detach()), oracle.gemm("dd", A, B), "forward")
    assert_bitwise(host(Ad.grad), oracle.gemm("dd", W, np.ascontiguousarray(B.transpose(0, 2, 1))), "dA")
    assert_bitwise(host(Bd.grad), oracle.gemm("dd", np.ascontiguousarray(A.transpose(0, 2, 1)), W), "dB")


def test_small_gradients_slicing_form_bitwise(torch):
    """With the tcgen05 slicing form, the forward product and both gradients
    equal the slicing oracle on the same operands bit for bit."""
    from oracle import ozaki as OZ
    from paper_2101_06584_gb300.autograd import dd_matmul
    rng = np.random.default_rng(820)
    S = 12
    A, B, W = I.uniform(2, (70, 90), rng), I.uniform(2, (90, 50), rng), I.uniform(2, (70, 50), rng)
    Ad = dev(torch, A).requires_grad_(True)
    Bd = dev(torch, B).requires_grad_(True)
    C = dd_matmul(Ad, Bd, algo="bf16", slices=S)
    C.backward(dev(torch, W))
    Bt = np.ascontiguousarray(B.transpose(0, 2, 1))
    At = np.ascontiguousarray(A.transpose(0, 2, 1))
    assert_bitwise(host(C.detach()), OZ.gemm(A, B, S)[0], "forward")
    assert_bitwise(host(Ad.grad), OZ.gemm(W, Bt, S)[0], "dA")
    assert_bitwise(host(Bd.grad), OZ.gemm(At, W, S)[0], "dB")


def test_small_gradients_crt_form_bitwise(torch):
    """With the tcgen05 CRT form, the forward product and both gradients
    equal the CRT oracle on the same operands bit for bit."""
    from oracle import crt as R
    from paper_2101_06584_gb300.autograd import dd_matmul
    rng = np.random.default_rng(821)
    N = 24
    A, B, W = I.uniform(2, (70, 90), rng), I.uniform(2, (90, 50), rng), I.uniform(2, (70, 50), rng)
    Ad = dev(torch, A).requires_grad_(True)
    Bd = dev(torch, B).requires_grad_(True)
    C = dd_matmul(Ad, Bd, algo="crt_bf16", slices=N)
    C.backward(dev(torch, W))
    Bt = np.ascontiguousarray(B.transpose(0, 2, 1))
    At = np.ascontiguousarray(A.transpose(0, 2, 1))
    assert_bitwise(host(C.detach()), R.gemm(A, B, N)[0], "forward")
    assert_bitwise(host(Ad.grad), R.gemm(W, Bt, N)[0], "dA")
    assert_bitwise(host(Bd.grad), R.gemm(At, W, N)[0], "dB")


def _fd_rows(A, B, W, samples):
    """QD central differences of loss(A) = sum(W * (A B)) wrt A[p, q]: only
    row p of C changes, so each needs a 1 x k by k x n QD product and a QD dot
    with row p of W (oracle, CPU)."""
    n = B.shape[2]
    rows = []
    for (p, q) in samples:
        for sgn in (1.0, -1.0):
            r = _qd(A[:, p:p + 1, :]).copy()
            # a +- h: exact in QD as (a0, a1, +-h) renormalised by the oracle add
            add = oracle.op("qd", "add", tuple(r[:, 0, q]), (sgn * H, 0.0, 0.0, 0.0))
            r[:, 0, q] = add
            rows.append(r[:, 0, :])
    R = np.stack(rows, axis=1)                          # (4, 2s, k)
    Cr = oracle.gemm("qd", R, _qd(B), nthreads=oracle.num_cpus())
    out = []
    for t, (p, q) in enumerate(samples):
        wq = _qd(W[:, p:p + 1, :])                     # (4, 1, n)
        lp = oracle.gemm("qd", wq, Cr[:, 2 * t:2 * t + 1, :].transpose(0, 2, 1).copy())
        lm = oracle.gemm("qd", wq, Cr[:, 2 * t + 1:2 * t + 2, :].transpose(0, 2, 1).copy())
        out.append((X.value(lp[:, 0, 0]) - X.value(lm[:, 0, 0])) / (2 * Fraction(H)))
    return out


@pytest.fixture(scope="module")
def full_size():
    n = 2048
    rng = I.rng_for(4)
    return n, I.uniform(2, (n, n), rng), I.uniform(2, (n, n), rng), I.uniform(2, (n, n), rng)


_FD_CACHE = {}


def _check_fd(A, B, W, dA, dB, n, srng):
    """dA and dB within n 2^-100 of QD central differences on 64 entries each
    (the differences of one set of samples are computed once per module)."""
    Bt = np.ascontiguousarray(B.transpose(0, 2, 1))
    At = np.ascontiguousarray(A.transpose(0, 2, 1))
    samples = [(int(srng.integers(n)), int(srng.integers(n))) for _ in range(64)]
    Wt = np.ascontiguousarray(W.transpose(0, 2, 1))
    key = (id(A), id(B), id(W), tuple(samples))
    if key not in _FD_CACHE:
        _FD_CACHE[key] = (_fd_rows(A, B, W, samples), _fd_rows(Bt, At, Wt, samples))
    fd, fdb = _FD_CACHE[key]
    absWB = X.ExactRows(np.abs(W), np.abs(Bt))
    for (p, q), g in zip(samples, fd):
        bound = n * Fraction(2) ** -100 * absWB.dot(p, q)
        assert abs(X.value(dA[:, p, q]) - g) <= bound, ("dA", p, q)
    absWA = X.ExactRows(np.abs(Wt), np.abs(A))
    for (p, q), g in zip(samples, fdb):
        bound = n * Fraction(2) ** -100 * absWA.dot(p, q)
        assert abs(X.value(dB[:, q, p]) - g) <= bound, ("dB", q, p)


def test_full_size_slicing_form_against_fd(torch, full_size):
    """The tcgen05 slicing form (default 14 slices) at 2048^3: both gradients
    within n 2^-100 of QD central differences, like the k-sequential ones."""
    from paper_2101_06584_gb300.autograd import dd_matmul
    n, A, B, W = full_size
    Ad = dev(torch, A).requires_grad_(True)
    Bd = dev(torch, B).requires_grad_(True)
    C = dd_matmul(Ad, Bd, algo="bf16")
    C.backward(dev(torch, W))
    _check_fd(A, B, W, host(Ad.grad), host(Bd.grad), n, np.random.default_rng(830))


def test_full_size_crt_form_against_fd(torch, full_size):
    """The tcgen05 CRT form with 26 moduli (94 bits per scaled entry at
    k = 2048, the benchmark's count) at 2048^3: both gradients within
    n 2^-100 of QD central differences on the same 64 entries."""
    from paper_2101_06584_gb300.autograd import dd_matmul
    n, A, B, W = full_size
    Ad = dev(torch, A).requires_grad_(True)
    Bd = dev(torch, B).requires_grad_(True)
    C = dd_matmul(Ad, Bd, algo="crt_bf16", slices=26)
    C.backward(dev(torch, W))
    _check_fd(A, B, W, host(Ad.grad), host(Bd.grad), n, np.random.default_rng(830))


def test_full_size_against_fd_and_oracle(torch, full_size):
    from paper_2101_06584_gb300.autograd import dd_matmul
    n, A, B, W = full_size
    Ad = dev(torch, A).requires_grad_(True)
    Bd = dev(torch, B).requires_grad_(True)
    C = dd_matmul(Ad, Bd)
    C.backward(dev(torch, W))
    dA, dB = host(Ad.grad), host(Bd.grad)

    srng = np.random.default_rng(810)
    # the oracle gradient: full DD products on sampled rows, bit for bit
    rows = np.sort(srng.choice(n, 4, replace=False))
    Bt = np.ascontiguousarray(B.transpose(0, 2, 1))
    want = oracle.gemm("dd", np.ascontiguousarray(W[:, rows, :]), Bt, nthreads=oracle.num_cpus())
    assert_bitwise(dA[:, rows, :], want, "dA rows")
    At = np.ascontiguousarray(A.transpose(0, 2, 1))
    want = oracle.gemm("dd", np.ascontiguousarray(At[:, rows, :]), W, nthreads=oracle.num_cpus())
    assert_bitwise(dB[:, rows, :], want, "dB rows")

    # QD central differences on 64 entries of dA (dB by the same formula on
    # the transposed problem: loss = sum(W^T * (B^T A^T)))
    samples = [(int(srng.integers(n)), int(srng.integers(n))) for _ in range(64)]
    fd = _fd_rows(A, B, W, samples)
    absWB = X.ExactRows(np.abs(W), np.abs(Bt))
    for (p, q), g in zip(samples, fd):
        bound = n * Fraction(2) ** -100 * absWB.dot(p, q)
        assert abs(X.value(dA[:, p, q]) - g) <= bound, ("dA", p, q)
    # on the transposed problem the difference at (p, q) is dB[q, p] =
    # sum_i A[i, q] W[i, p], bounded by (|W^T| |A|)[p, q]
    Wt = np.ascontiguousarray(W.transpose(0, 2, 1))
    fdb = _fd_rows(Bt, At, Wt, samples)
    absWA = X.ExactRows(np.abs(Wt), np.abs(A))
    for (p, q), g in zip(samples, fdb):
        bound = n * Fraction(2) ** -100 * absWA.dot(p, q)
        assert abs(X.value(dB[:, q, p]) - g) <= bound, ("dB", q, p)
