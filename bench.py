#!/usr/bin/env python3
"""Benchmark: multi-component (DD/TD/QD) GEMM on one GB300 (or N independent
replicas), reported as multiply-adds per second and as a fraction of the FP64
roofline, with the CPU oracle timed beside it.

Default workload (one "step"): the TD GEMM and the QD GEMM, m = n = k = 1024,
on seeded ill-scaled inputs whose inner dimension is built to cancel (the
k-sequential FP64-EFT kernels, bit-identical to the oracle).  Other
workloads are measured once each and reported under "configs".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own independent problem (weak scaling);
only host-side timing is reduced across ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "DD/TD/QD GEMM multiply-adds/s and % FP64 roofline; INT8-sliced vs plain speedup"
UNIT = "mad/s"
# binary64 instructions per multiply-add of the implemented sequences (FMA
# counted once): DD = DDmul 9 + DDadd 11; TD = TDmul 47 + TDaddq 81 (the
# operations on the constant zero fourth components are folded away);
# QD = QDmul 123 + QDadd 87.
FP64_OPS_PER_MAD = {"dd": 20, "td": 128, "qd": 210}
L2_FLUSH_BYTES = 256 << 20          # larger than the 129 MB L2


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=1024, help="m = n = k of the TD/QD workload")
    ap.add_argument("--no-extras", action="store_true", help="skip the other configurations")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value, world):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank):
        self.proc = None
        self.path = None
        self.index = str(local_rank)
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        if vis:
            ids = vis.split(",")
            if local_rank < len(ids) and ids[local_rank].strip().isdigit():
                self.index = ids[local_rank].strip()

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.index, "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 8 and parts[0].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows]
        smax = max(float(r[1]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[2]) for r in rows
                                                          if r[2].replace(".", "").isdigit())}


# ------------------------------------------------------------ CPU baseline

def cpu_sample_rate(prec_list, size, rows, cfg=1):
    """Oracle (as it stands) on all host cores: mad/s over the first ``rows``
    rows of C for each precision, same inputs as the GPU workload."""
    import oracle
    from paper_2101_06584_gb300 import inputs as I
    cores = oracle.num_cpus()
    mads = 0
    secs = 0.0
    for prec in prec_list:
        P = I.P_OF[prec]
        A, B = I.cancelling_pair(P, size, size, size, I.rng_for(cfg))
        A = np.ascontiguousarray(A[:, :rows, :])
        t0 = time.perf_counter()
        oracle.gemm(prec, A, B, nthreads=cores)
        secs += time.perf_counter() - t0
        mads += rows * size * size
    return mads / secs, cores, secs


# ------------------------------------------------------------------ GPU arm

def fp64_peaks(torch, mm):
    """Measured FP64 lane-operation rate of the probe kernel (add and fma),
    at this run's clocks."""
    from paper_2101_06584_gb300 import mpgemm
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = sms * 8
    out = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    res = {}
    for kind, name in ((0, "dadd"), (1, "dmul"), (2, "dfma")):
        iters = 2048
        mpgemm.fp64_probe(kind, blocks, 64, out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mpgemm.fp64_probe(kind, blocks, iters, out)
        e1.record()
        torch.cuda.synchronize()
        ops = blocks * 256 * iters * 8
        res[name] = ops / (e0.elapsed_time(e1) * 1e-3)
    return res


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2101_06584_gb300 import build as libbuild
    libbuild.build()
    from paper_2101_06584_gb300 import inputs as I
    from paper_2101_06584_gb300 import mpgemm as mm

    n = args.size
    precs = ("td", "qd")
    rng = np.random.Generator(np.random.PCG64(I.SEED_BASE + 1 + 1000 * rank))
    host_in = {}
    dev_in = {}
    for prec in precs:
        P = I.P_OF[prec]
        A, B = I.cancelling_pair(P, n, n, n, rng)
        host_in[prec] = (A, B)
        dev_in[prec] = (torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                        torch.empty((P, n, n), dtype=torch.float64, device="cuda"))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    peaks = fp64_peaks(torch, mm)

    def step(events=None):
        for prec in precs:
            A, B, C = dev_in[prec]
            if events is not None:
                events[prec][0].record(stream)
            mm.gemm_plain(prec, A, B, out=C)
            if events is not None:
                events[prec][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    launch_ms = {p: [] for p in precs}
    step_ms = []
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()                                   # evict L2 between steps (untimed)
        ev = {p: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for p in precs}
        step(ev)
        torch.cuda.synchronize()
        for p in precs:
            launch_ms[p].append(ev[p][0].elapsed_time(ev[p][1]))
        step_ms.append(ev[precs[0]][0].elapsed_time(ev[precs[-1]][1]))
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - t_wall
    clocks = sampler.stop()

    total_ms = max_over_ranks(sum(step_ms), world)
    mads_per_step = len(precs) * n * n * n
    value = world * mads_per_step * args.steps / (total_ms * 1e-3)

    # dominant kernel: the one with the larger share of the step
    avg = {p: statistics.mean(launch_ms[p]) for p in precs}
    dom = max(precs, key=lambda p: avg[p])
    ops_per_launch = n * n * n * FP64_OPS_PER_MAD[dom]
    achieved = ops_per_launch / (avg[dom] * 1e-3)
    peak = peaks["dfma"]

    # end to end through the public API: pinned host -> device, GEMM, device -> host
    pinned = {p: tuple(torch.from_numpy(x).pin_memory() for x in host_in[p]) for p in precs}
    out_host = {p: torch.empty((I.P_OF[p], n, n), dtype=torch.float64).pin_memory() for p in precs}
    h2d = sum(x.numel() * 8 for p in precs for x in pinned[p])
    d2h = sum(out_host[p].numel() * 8 for p in precs)

    def e2e_step():
        for p in precs:
            A, B, C = dev_in[p]
            A.copy_(pinned[p][0], non_blocking=True)
            B.copy_(pinned[p][1], non_blocking=True)
            mm.gemm_plain(p, A, B, out=C)
            out_host[p].copy_(C, non_blocking=True)
        torch.cuda.synchronize()

    e2e_step()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    barrier(world)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e_value = world * mads_per_step * args.steps / e2e_s

    # consistency: the timed results equal a fresh call (deterministic kernels)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded PCG64; ill-scaled TD/QD entries with cancelling inner halves)",
        "config": {"workload": "TD GEMM + QD GEMM, m=n=k=%d, k-sequential FP64-EFT" % n,
                   "precisions": list(precs), "m": n, "n": n, "k": n,
                   "mads_per_step": mads_per_step, "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "per_precision_mad_s": {p: n ** 3 / (statistics.mean(launch_ms[p]) * 1e-3) for p in precs},
        "roofline": {"bound": "alu", "kernel": "gemm_kseq_kernel<%s>" % dom.upper(),
                     "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFP64op/s",
                     "frac": achieved / peak, "traffic": None,
                     "ops_per_mad": FP64_OPS_PER_MAD[dom],
                     "peak_source": "measured FP64 FMA probe at this run's clocks "
                                    "(dadd %.1f, dmul %.1f, dfma %.1f G lane-op/s)" % (
                                        peaks["dadd"] / 1e9, peaks["dmul"] / 1e9, peaks["dfma"] / 1e9)},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": len(precs) * args.steps,
        "clocks": clocks,
        "wall_s": wall,
    }
    if not args.no_extras and rank == 0:
        line["configs"] = extras(torch, mm, I)
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        rows = max(oracle.num_cpus(), n // 16)
        rate, cores, secs = cpu_sample_rate(precs, n, rows=rows)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "first %d rows of C for TD and QD at m=n=k=%d "
                                          "(%.1f s on %d threads)" % (rows, n, secs, cores)}
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def _time_call(torch, fn, reps=1):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def extras(torch, mm, I):
    """The other workloads, each measured once after the main timing."""
    out = {}
    # DD m=n=k=128, uniform inputs
    P = 2
    A, B = I.uniform(P, (128, 128), I.rng_for(0)), I.uniform(P, (128, 128), I.rng_for(0))
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C = torch.empty((P, 128, 128), dtype=torch.float64, device="cuda")
    ms = _time_call(torch, lambda: mm.gemm_plain("dd", Ad, Bd, out=C), reps=20)
    ms_sk = _time_call(torch, lambda: mm.gemm("dd", Ad, Bd, out=C, split_k=8), reps=20)
    out["dd_128"] = {"mad_s_kseq": 128 ** 3 / (ms * 1e-3), "mad_s_splitk8": 128 ** 3 / (ms_sk * 1e-3)}
    # DD m=n=k=4096, plain FP64-EFT
    n = 4096
    rng = I.rng_for(2)
    A, B = I.uniform(P, (n, n), rng), I.uniform(P, (n, n), rng)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C = torch.empty((P, n, n), dtype=torch.float64, device="cuda")
    ms = _time_call(torch, lambda: mm.gemm_plain("dd", Ad, Bd, out=C), reps=1)
    out["dd_4096_fp64_eft"] = {"mad_s": n ** 3 / (ms * 1e-3), "ms": ms}
    # the same product through the INT8 error-free slicing form
    for S in (13, 14):
        ws = torch.empty(mm.workspace_size("dd", n, n, n, algo="int8", slices=S),
                         dtype=torch.uint8, device="cuda")
        C8 = torch.empty_like(C)
        ms8 = _time_call(torch, lambda: mm.gemm("dd", Ad, Bd, out=C8, algo="int8", slices=S,
                                                workspace=ws), reps=3)
        pairs = S * (S + 1) // 2
        out["dd_4096_int8_s%d" % S] = {
            "mad_s": n ** 3 / (ms8 * 1e-3), "ms": ms8, "speedup_vs_fp64_eft": ms / ms8,
            "int8_tops": 2.0 * pairs * n ** 3 / (ms8 * 1e-3) / 1e12}
        del ws
    return out


# --------------------------------------------------------- reference arm

def run_reference(args):
    """The oracle (CPU, as it stands) on a bounded sample of the same workload."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    precs = ("td", "qd")
    n = args.size
    import oracle
    rows = max(oracle.num_cpus(), n // 64)
    for _ in range(args.warmup):
        cpu_sample_rate(precs, n, rows=1)
    rates, secs_all = [], 0.0
    cores = 1
    for _ in range(args.steps):
        r, cores, secs = cpu_sample_rate(precs, n, rows=rows)
        rates.append(r)
        secs_all += secs
    value = statistics.mean(rates)
    sample = "first %d rows of C for TD and QD at m=n=k=%d per step" % (rows, n)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded PCG64; ill-scaled TD/QD entries with cancelling inner halves)",
            "config": {"workload": "TD GEMM + QD GEMM, m=n=k=%d, k-sequential (CPU oracle)" % n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
