"""The N > 1 benchmark path on CPU with torch.distributed (gloo, world size 2):
each rank runs its own independent problem (distinct seeds, rank 0 on the
workload's own seed), the timing is the max over ranks, and the reported
value is the units all ranks processed over that time.  No data-path
collective exists: only the host-side timing is reduced."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # timings differ per rank; every rank sees the max
    mx = bench.reduce_max(10.0 + 5.0 * rank, world)
    first = bench.replica_rng(1, rank).uniform()
    own = np.random.Generator(np.random.PCG64(20210117 + 1)).uniform()
    bench.barrier(world)
    out.put((rank, mx, first, own))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, mx0, f0, own0), (r1, mx1, f1, _) = res
    assert mx0 == mx1 == 15.0                      # max over ranks
    assert f0 == own0                              # rank 0 runs the workload's seed
    assert f0 != f1                                # independent problems


def test_aggregate_value():
    import bench
    # 2 ranks x 2e9 mads x 3 steps over the slowest rank's 1.5 s
    assert bench.aggregate_value(2, 2e9, 3, 1500.0) == pytest.approx(8e9)
    assert bench.aggregate_value(1, 2e9, 3, 1500.0) == pytest.approx(4e9)
