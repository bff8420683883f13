"""The autotuner (mpgemm_autotune, mpgemm_batch_autotune) and its cache on the
GPU: the chosen tile is remembered for the shape's bucket, written to the
file MPGEMM_TUNE_CACHE names as JSON, read back after a reset, and taken by
mpgemm_ex with tile 0, whose result stays bit-identical to the oracle; a
batch's policy is returned from the cache for the same list of shapes."""
import json

import numpy as np
import pytest

import oracle
from gpu_util import assert_bitwise, dev, host, torch_cuda
from paper_2101_06584_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.fixture
def cache_file(tmp_path, monkeypatch):
    from paper_2101_06584_gb300 import mpgemm as mm
    path = tmp_path / "tune.json"
    monkeypatch.setenv("MPGEMM_TUNE_CACHE", str(path))
    mm.tune_cache_reset()
    yield path
    monkeypatch.delenv("MPGEMM_TUNE_CACHE")
    mm.tune_cache_reset()


def _entries(path):
    return json.loads(path.read_text())["entries"]


def test_gemm_tile_remembered(torch, cache_file):
    from paper_2101_06584_gb300 import mpgemm as mm
    rng = np.random.default_rng(910)
    A, B = I.uniform(2, (100, 128), rng), I.uniform(2, (128, 90), rng)
    Ad, Bd = dev(torch, A), dev(torch, B)
    tile, ms = mm.autotune("dd", Ad, Bd, reps=2)
    assert 1 <= tile <= mm.num_tiles("dd") and ms > 0
    ent = _entries(cache_file)
    key = [k for k in ent if k.endswith("|gemm:2:7:7:7")]
    assert len(key) == 1 and ent[key[0]]["choice"] == tile
    assert mm.tuned_tile("dd", 100, 128, 90) == tile
    assert mm.tuned_tile("dd", 65, 120, 70) == tile          # the same bucket
    mm.tune_cache_reset()                                     # read back from the file
    assert mm.tuned_tile("dd", 100, 128, 90) == tile
    want = oracle.gemm("dd", A, B)
    assert_bitwise(host(mm.gemm_plain("dd", Ad, Bd)), want, "tile 0 after tuning")
    assert_bitwise(host(mm.gemm("dd", Ad, Bd, tile=tile)), want, "the tuned tile")


def test_batch_policy_remembered(torch, cache_file):
    from paper_2101_06584_gb300 import mpgemm as mm
    rng = np.random.default_rng(911)
    shapes = [(40, 70, 30), (200, 16, 100), (17, 300, 64)]
    triples = []
    for (m, n, k) in shapes:
        A, B = dev(torch, I.uniform(4, (m, k), rng)), dev(torch, I.uniform(4, (k, n), rng))
        triples.append((A, B, torch.empty((4, m, n), dtype=torch.float64, device="cuda")))
    plan = mm.BatchPlan("qd", triples, policy=None, reps=1)
    first = plan.policy
    plan.close()
    assert any("|batch:4:3:" in k and v["choice"] == first for k, v in _entries(cache_file).items())
    plan = mm.BatchPlan("qd", triples, policy=None, reps=1)
    assert plan.policy == first
    plan.run()
    torch.cuda.synchronize()
    for (A, B, C) in triples:
        assert_bitwise(host(C), oracle.gemm("qd", host(A), host(B)), "batched after a remembered policy")
    plan.close()
