"""Batched persistent GEMM on the GPU: every C_i of a batch is bit-identical
to the oracle's k-sequential product of that problem, for every tile policy,
on graph replays, with transposes, empty and k = 0 problems, and on sampled
problems of the 512-problem log-uniform batch."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_bitwise, dev, host, torch_cuda
from paper_2101_06584_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def _make(torch, prec, shapes, rng, trans=False):
    P = I.P_OF[prec]
    triples, host_in = [], []
    for t, (m, n, k) in enumerate(shapes):
        A = I.uniform(P, (m, k), rng)
        B = I.uniform(P, (k, n), rng)
        ta = trans and t % 3 == 1
        tb = trans and t % 3 == 2
        Ad = dev(torch, A.transpose(0, 2, 1) if ta else A)
        Bd = dev(torch, B.transpose(0, 2, 1) if tb else B)
        C = torch.full((P, m, n), float("nan"), dtype=torch.float64, device="cuda")
        triples.append((Ad, Bd, C, ta, tb))
        host_in.append((A, B))
    return triples, host_in


@pytest.mark.parametrize("prec", ["dd", "td", "qd"])
def test_batch_bitwise_every_policy(torch, prec):
    from paper_2101_06584_gb300 import mpgemm as mm
    rng = np.random.default_rng(700 + I.P_OF[prec])
    shapes = [(1, 1, 1), (17, 33, 9), (64, 64, 64), (5, 90, 40), (70, 3, 120), (0, 5, 5),
              (7, 0, 3), (9, 12, 0), (33, 31, 65), (48, 16, 1)]
    triples, host_in = _make(torch, prec, shapes, rng, trans=True)
    wants = [oracle.gemm(prec, A, B, nthreads=4) for A, B in host_in]
    for policy in range(mm.BATCH_POLICIES):  # mm.BATCH_INT_POLICY: integer-pipe transformations
        for (_, _, C, _, _) in triples:
            C.fill_(float("nan"))
        plan = mm.BatchPlan(prec, triples, policy=policy)
        plan.run()
        plan.run()                        # a replay gives the same bits
        torch.cuda.synchronize()
        for i, ((_, _, C, _, _), want) in enumerate(zip(triples, wants)):
            assert_bitwise(host(C), want, "%s policy %d problem %d %s" % (prec, policy, i, shapes[i]))
        info = plan.info()
        assert info["policy"] == policy and info["count"] == len(shapes)
        plan.close()


def test_autotune_and_large_batch(torch):
    """The 512-problem batch (m, n, k log-uniform in [16, 512]), DD: the
    autotuner picks a policy; sampled problems are bit-identical to the
    oracle (full products for the smaller ones, sampled rows otherwise)."""
    from paper_2101_06584_gb300 import mpgemm as mm
    rng = I.rng_for(3)
    shapes = I.batch_shapes(512, rng)
    triples, host_in = _make(torch, "dd", shapes, rng)
    plan = mm.BatchPlan("dd", triples, policy=None, reps=1)
    assert 0 <= plan.policy < mm.BATCH_POLICIES and plan.tune_ms > 0
    plan.run()
    torch.cuda.synchronize()
    srng = np.random.default_rng(710)
    for i in srng.choice(len(shapes), 8, replace=False):
        A, B = host_in[i]
        C = host(triples[i][2])
        rows = np.arange(A.shape[1]) if A.shape[1] <= 64 else np.sort(srng.choice(A.shape[1], 16, replace=False))
        want = oracle.gemm("dd", np.ascontiguousarray(A[:, rows, :]), B, nthreads=8)
        assert_bitwise(C[:, rows, :], want, "batch problem %d %s" % (i, shapes[i]))
    plan.close()


def test_qd_512_problem_batch_of_the_benchmark(torch):
    """The QD half of the benchmark's batch: the same generator in the same
    order (the 512 shapes, the DD inputs, then the QD inputs), tuned plan as
    the benchmark builds it.  Ten sampled problems and the one with the most
    work are bit-identical to the oracle (every row of the smaller ones,
    sampled rows of the others)."""
    from paper_2101_06584_gb300 import mpgemm as mm
    rng = I.rng_for(3)
    shapes = I.batch_shapes(512, rng)
    dd_triples, _ = _make(torch, "dd", shapes, rng)            # drawn first, as in the benchmark
    del dd_triples
    triples, host_in = _make(torch, "qd", shapes, rng)
    plan = mm.BatchPlan("qd", triples, policy=None, reps=1)
    plan.run()
    torch.cuda.synchronize()
    srng = np.random.default_rng(720)
    work = [m * n * k for (m, n, k) in shapes]
    picks = set(int(i) for i in srng.choice(len(shapes), 10, replace=False)) | {int(np.argmax(work))}
    for i in sorted(picks):
        A, B = host_in[i]
        C = host(triples[i][2])
        rows = np.arange(A.shape[1]) if A.shape[1] <= 48 else np.sort(srng.choice(A.shape[1], 12, replace=False))
        want = oracle.gemm("qd", np.ascontiguousarray(A[:, rows, :]), B, nthreads=8)
        assert_bitwise(C[:, rows, :], want, "qd batch problem %d %s" % (i, shapes[i]))
    plan.close()
