"""Differentiation through the DD GEMM (not in the paper).

DDMatmul is a torch.autograd.Function over C = A B in double-double, with A
(2, m, k), B (2, k, n) and C (2, m, n) as component planes (Sec. 2.5).  Its
hand-written backward runs the library's DD kernels on the transposed
operands (no transpose copies):

    dA = dC B^T   (mpgemm_ex with trans_b; mul(x = dC entry, y = B entry))
    dB = A^T dC   (mpgemm_ex with trans_a; mul(x = A entry, y = dC entry))

By default each is the k-sequential DD product of Sec. 3, Eq. 1, so the
gradients are bit-identical to that product evaluated anywhere.  With
algo="bf16" (or "int8") the forward product and both gradients run the
error-free slicing form on the tensor cores instead, and with
algo="crt_bf16" (or "crt") the CRT form, `slices` then counting moduli (the
forms defined in include/mpgemm.h): each product is bit-identical to that
form's steps on the same operands and within its DD error bound of the exact
product.  The incoming
gradient is itself a DD plane pair: for loss = sum(W * C), call C.backward(W).
"""
import torch

from . import mpgemm


def _product(A, B, algo, slices, trans_a=False, trans_b=False):
    if algo in ("auto", "fp64"):
        return mpgemm.gemm("dd", A, B, trans_a=trans_a, trans_b=trans_b, algo=algo)
    m = A.shape[2] if trans_a else A.shape[1]
    k = A.shape[1] if trans_a else A.shape[2]
    n = B.shape[1] if trans_b else B.shape[2]
    ws = torch.empty(mpgemm.workspace_size("dd", m, n, k, algo=algo, slices=slices), dtype=torch.uint8,
                     device=A.device)
    return mpgemm.gemm("dd", A, B, trans_a=trans_a, trans_b=trans_b, algo=algo, slices=slices, workspace=ws)


class DDMatmul(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, algo="auto", slices=0):
        ctx.save_for_backward(A, B)
        ctx.algo, ctx.slices = algo, slices
        return _product(A, B, algo, slices)

    @staticmethod
    def backward(ctx, dC):
        A, B = ctx.saved_tensors
        dC = dC.contiguous()
        dA = dB = None
        if ctx.needs_input_grad[0]:
            dA = _product(dC, B, ctx.algo, ctx.slices, trans_b=True)
        if ctx.needs_input_grad[1]:
            dB = _product(A, dC, ctx.algo, ctx.slices, trans_a=True)
        return dA, dB, None, None


def dd_matmul(A, B, algo="auto", slices=0):
    """C = A B in DD with gradients through the DD kernels (algo "auto" /
    "fp64"), the slicing form on the tensor cores ("bf16", "int8"; slices
    0 = the library's default) or the CRT form ("crt_bf16", "crt"; slices =
    moduli, 0 = the library's default)."""
    return DDMatmul.apply(A, B, algo, slices)


def dd_weighted_sum(W, C, split_k=32):
    """The DD value of sum_ij W_ij C_ij (no gradient), as a (2,) tensor:
    a 1 x (mn) by (mn) x 1 DD product with the warp split-K kernel."""
    mn = W.shape[1] * W.shape[2]
    w = W.reshape(2, 1, mn)
    c = C.reshape(2, mn, 1)
    return mpgemm.gemm("dd", w, c, split_k=split_k).reshape(2)
