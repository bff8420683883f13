"""Differentiation through the DD GEMM (not in the paper).

DDMatmul is a torch.autograd.Function over C = A B in double-double, with A
(2, m, k), B (2, k, n) and C (2, m, n) as component planes (Sec. 2.5).  Its
hand-written backward runs the library's DD kernels on the transposed
operands (no transpose copies):

    dA = dC B^T   (mpgemm_ex with trans_b; mul(x = dC entry, y = B entry))
    dB = A^T dC   (mpgemm_ex with trans_a; mul(x = A entry, y = dC entry))

Each is the k-sequential DD product of Sec. 3, Eq. 1, so the gradients are
bit-identical to that product evaluated anywhere.  The incoming gradient is
itself a DD plane pair: for loss = sum(W * C), call C.backward(W).
"""
import torch

from . import mpgemm


class DDMatmul(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B):
        ctx.save_for_backward(A, B)
        return mpgemm.gemm("dd", A, B)

    @staticmethod
    def backward(ctx, dC):
        A, B = ctx.saved_tensors
        dC = dC.contiguous()
        dA = dB = None
        if ctx.needs_input_grad[0]:
            dA = mpgemm.gemm("dd", dC, B, trans_b=True)
        if ctx.needs_input_grad[1]:
            dB = mpgemm.gemm("dd", A, dC, trans_a=True)
        return dA, dB


def dd_matmul(A, B):
    """C = A B in DD with gradients through the DD kernels."""
    return DDMatmul.apply(A, B)


def dd_weighted_sum(W, C, split_k=32):
    """The DD value of sum_ij W_ij C_ij (no gradient), as a (2,) tensor:
    a 1 x (mn) by (mn) x 1 DD product with the warp split-K kernel."""
    mn = W.shape[1] * W.shape[2]
    w = W.reshape(2, 1, mn)
    c = C.reshape(2, mn, 1)
    return mpgemm.gemm("dd", w, c, split_k=split_k).reshape(2)
