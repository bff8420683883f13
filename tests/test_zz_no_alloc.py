"""mpgemm_dd_int8_static: the INT8 slicing DD product for callers that cannot
allocate device memory -- code running inside a host framework that owns all
device memory through its own pool, or a latency-critical loop that cannot
afford cudaMalloc's implicit synchronisation.  It keeps its scratch in a
fixed 32 MiB array inside the library instead of taking a workspace.

Checked through the C ABI: two calls in a row give exactly the bits of
mpgemm_ex with a caller-provided workspace (the INT8 tests' tolerance is
bit-identity), and a product whose scratch exceeds the array is refused with
MPG_EWORKSPACE before anything runs.  This file is collected last so that a
run stopping at the first failure has already run every other test; it also
passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest

from gpu_util import assert_bitwise, dev, host, torch_cuda
from paper_2101_06584_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def _static(torch, Ad, Bd, S):
    from paper_2101_06584_gb300 import mpgemm as mm
    L = mm.lib()
    m, k = Ad.shape[1], Ad.shape[2]
    n = Bd.shape[2]
    C = torch.full((2, m, n), float("nan"), dtype=torch.float64, device="cuda")
    mm._bind_stream()
    rc = L.mpgemm_dd_int8_static(m, n, k, mm.planes(Ad), k, mm.planes(Bd), n, mm.planes(C), n, S)
    mm.check(rc)
    return C


def _with_workspace(torch, Ad, Bd, S):
    from paper_2101_06584_gb300 import mpgemm as mm
    m, k = Ad.shape[1], Ad.shape[2]
    n = Bd.shape[2]
    ws = torch.empty(mm.workspace_size("dd", m, n, k, algo="int8", slices=S),
                     dtype=torch.uint8, device="cuda")
    return mm.gemm("dd", Ad, Bd, algo="int8", slices=S, workspace=ws)


def test_two_calls_in_a_row_match_the_workspace_entry(torch):
    rng = np.random.default_rng(900)
    for (m, n, k, S) in ((200, 150, 130, 13), (96, 80, 112, 10)):
        A = I.uniform(2, (m, k), rng)
        B = I.ill_scaled(2, (k, n), rng)
        Ad, Bd = dev(torch, A), dev(torch, B)
        got = host(_static(torch, Ad, Bd, S))
        want = host(_with_workspace(torch, Ad, Bd, S))
        assert_bitwise(got, want, "static scratch %s" % ((m, n, k, S),))


def test_oversized_product_is_refused(torch):
    from paper_2101_06584_gb300 import mpgemm as mm
    L = mm.lib()
    n = 2048
    A = torch.zeros((2, n, n), dtype=torch.float64, device="cuda")
    C = torch.zeros((2, n, n), dtype=torch.float64, device="cuda")
    mm._bind_stream()
    rc = L.mpgemm_dd_int8_static(n, n, n, mm.planes(A), n, mm.planes(A), n, mm.planes(C), n, 14)
    assert rc == -3
    assert b"fixed array" in L.mpgemm_last_error()


def test_back_to_back_calls_on_one_stream(torch):
    """Two different products issued back to back on one stream, with a single
    synchronisation at the end: the second call reuses the array while the
    first may still be queued, so they are ordered only by the stream (op(B)
    of each is sliced on a side stream forked from and joined back to it).
    Both results equal the workspace entry's bit for bit."""
    from paper_2101_06584_gb300 import mpgemm as mm
    rng = np.random.default_rng(910)
    shapes = ((300, 260, 250, 14), (130, 190, 170, 9))
    ops = []
    for (m, n, k, S) in shapes:
        A = I.ill_scaled(2, (m, k), rng)
        B = I.uniform(2, (k, n), rng)
        ops.append((dev(torch, A), dev(torch, B), S))
    wants = [host(_with_workspace(torch, Ad, Bd, S)) for Ad, Bd, S in ops]
    torch.cuda.synchronize()
    L = mm.lib()
    mm._bind_stream()
    outs = []
    for Ad, Bd, S in ops:
        m, k = Ad.shape[1], Ad.shape[2]
        n = Bd.shape[2]
        C = torch.full((2, m, n), float("nan"), dtype=torch.float64, device="cuda")
        mm.check(L.mpgemm_dd_int8_static(m, n, k, mm.planes(Ad), k, mm.planes(Bd), n, mm.planes(C), n, S))
        outs.append(C)
    torch.cuda.synchronize()
    for (m, n, k, S), C, want in zip(shapes, outs, wants):
        assert_bitwise(host(C), want, "back to back %s" % ((m, n, k, S),))
