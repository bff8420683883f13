"""Helpers for the GPU parity tests: host<->device transfer and bitwise
comparison.  No arithmetic of the method lives here."""
import numpy as np
import pytest


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_06584_gb300 import build
    build.build()
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def assert_bitwise(got, want, what=""):
    got = np.ascontiguousarray(got)
    want = np.ascontiguousarray(want)
    assert got.shape == want.shape, (what, got.shape, want.shape)
    g = got.view(np.int64)
    w = want.view(np.int64)
    bad = np.argwhere(g != w)
    assert bad.size == 0, "%s: %d of %d values differ; first at %s: got %r want %r" % (
        what, len(bad), g.size, tuple(bad[0]), got[tuple(bad[0])], want[tuple(bad[0])])
