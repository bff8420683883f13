#!/usr/bin/env python3
"""Benchmark: multi-component (DD/TD/QD) GEMM on one GB300 (or N independent
replicas), reported as multiply-adds per second and as a fraction of the
roofline of the dominant kernel, with the CPU oracle timed beside it.

Workloads (one "step" = one pass of the workload's kernels over its inputs):
  td_qd     (default) TD GEMM + QD GEMM, m = n = k = 1024, seeded ill-scaled
            inputs whose inner dimension cancels; k-sequential FP64-EFT kernels
            (bit-identical to the oracle)
  dd_small  DD GEMM 128^3, uniform inputs
  dd_int8   DD GEMM 4096^3 through the INT8 error-free slicing form (slicing +
            tensor-core slice products + EFT accumulation), S the smallest
            slice count whose product meets n 2^-100 on sampled entries
  dd_tc     the dd_int8 product with the digits as bf16 on tcgen05 (TMEM
            accumulators, TMA staging)
  td_qd_int8, td_qd_tc  the TD and QD GEMMs of td_qd through the slicing form
            (S = 22 / 29) on either engine
  batched   512 DD and 512 QD problems, m, n, k log-uniform in [16, 512], each
            precision one persistent launch replayed from a CUDA graph
  autograd  DDMatmul forward + backward (3 DD GEMMs), m = n = k = 2048

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME]

The default line also carries, under "configs", one measurement of every
other workload.  Under torchrun each rank runs its own independent problem
(weak scaling); only timings are reduced across ranks.
"""
import argparse
import json
import math
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
# The same multiply-adds by kind: (TwoSum, FastTwoSum, TwoProd, other
# rounded operations); a transformation is 6, 3 or 2 binary64 operations as
# a sequence, so 6 a + 3 b + 2 c + d = FP64_OPS_PER_MAD.
EFT_MIX = {"dd": (1, 2, 1, 6), "td": (14, 10, 3, 8), "qd": (22, 16, 6, 18)}


def kseq_bound(prec, int_ops, pk):
    """Lower bound in seconds per multiply-add of a k-sequential tile that
    computes the transformations in `int_ops` (1 TwoSum, 2 FastTwoSum, 4
    TwoProd) on the integer pipes, at the measured rates `pk`: the larger of
    the FP64-pipe time of the operations left there and the integer-pipe time
    of the transformations moved (the two pipes run side by side).  Returns
    (seconds, FP64-pipe operations per multiply-add)."""
    ts, qts, tp, other = EFT_MIX[prec]
    f64 = other + (0 if int_ops & 1 else 6 * ts) + (0 if int_ops & 2 else 3 * qts) + (0 if int_ops & 4 else 2 * tp)
    t_int = ((ts / pk["int_two_sum"] if int_ops & 1 else 0.0)
             + (qts / pk["int_fast_two_sum"] if int_ops & 2 else 0.0)
             + (tp / pk["int_two_prod"] if int_ops & 4 else 0.0))
    return max(f64 / pk["dfma"], t_int), f64


def kseq_roofline(prec, mads, ms, pk, ti):
    """The roofline fields of a k-sequential GEMM launch on tile `ti`
    (mpgemm.tile_info): achieved = binary64 operations of the algorithm per
    second (FP64_OPS_PER_MAD per multiply-add, wherever they run); peak =
    the same operations at the kseq_bound rate."""
    bound_s, f64 = kseq_bound(prec, ti["int_ops"], pk)
    ops = FP64_OPS_PER_MAD[prec]
    ach = mads * ops / (ms * 1e-3)
    peak = ops / bound_s
    return {"bound": "alu", "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "TFP64op/s",
            "frac": ach / peak, "ops_per_unit": ops, "int_ops": ti["int_ops"],
            "fp64_pipe_ops_per_unit": f64, "frac_of_fp64_pipe_alone": ach / pk["dfma"],
            "peak_source": "max(FP64-pipe operations / measured DFMA rate, integer-pipe transformations / "
                           "measured TwoSum, FastTwoSum, TwoProd rates) per multiply-add, this run's clocks"}
L2_FLUSH_BYTES = 256 << 20          # larger than the 129 MB L2
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


def bf16_peak():
    """Dense bf16 tensor peak (FLOP/s) for a kernel timed alone: the measured
    burst figure of MEASURED_PEAKS.json, else the profiling recipe's fallback."""
    try:
        with open(PEAKS_FILE) as f:
            v = json.load(f).get("bf16_tflops")
        if v:
            return float(v) * 1e12, "measured (MEASURED_PEAKS.json bf16_tflops, cuBLAS burst)"
    except (OSError, ValueError):
        pass
    return 1.9e15, "fallback 1.9 PFLOP/s"


# the sources each recorded kernel is compiled from
TRAFFIC_SOURCES = {
    "td_qd": ["mp_arith.cuh", "soft_fp64.cuh", "gemm_kernel.cuh", "gemm_qd.cu", "internal.h"],
    "dd_int8": ["mp_arith.cuh", "ozaki.cu", "ozaki_common.cuh", "ozaki.h", "internal.h"],
    "dd_tc": ["mp_arith.cuh", "ozaki.cu", "ozaki_common.cuh", "ozaki.h", "internal.h"],
    "dd_crtint8": ["crt.cu", "ozaki_common.cuh", "ozaki.h", "internal.h"],
    "dd_crttc": ["crt.cu", "ozaki_common.cuh", "ozaki.h", "internal.h"],
}


def kernel_source_hash(key):
    """SHA-256 over the sources of the kernel recorded under `key`."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2101_06584_gb300", "csrc")
    for f in TRAFFIC_SOURCES[key.split("_")[0] + "_" + key.split("_")[1]]:
        h.update(f.encode())
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(key):
    """DRAM bytes per launch (read + write) recorded from an ncu capture of the
    current kernel sources, or None when those sources changed since."""
    try:
        with open(TRAFFIC_FILE) as f:
            ent = json.load(f).get(key)
    except (OSError, ValueError):
        return None
    if ent is None or ent.get("source_sha256") != kernel_source_hash(key):
        return None
    return ent.get("bytes_per_launch")


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="td_qd",
                    choices=["td_qd", "dd_small", "dd_int8", "dd_tc", "dd_crt", "dd_crt_int8", "td_crt", "qd_crt",
                             "td_qd_int8", "td_qd_tc",
                             "batched", "autograd", "elementwise", "strassen", "autograd_tc",
                             "autograd_crt"])
    ap.add_argument("--size", type=int, default=None, help="override the workload's m = n = k")
    ap.add_argument("--slices", type=int, default=None,
                    help="slice (or moduli) count of the DD slicing/CRT workloads instead of the search")
    ap.add_argument("--no-extras", action="store_true", help="skip the other workloads")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the error figures (the slicing forms then take fixed slice counts)")
    ap.add_argument("--record-traffic", metavar="NCU_CSV",
                    help="record DRAM bytes per launch from an ncu --csv log (dram__bytes_read.sum, "
                         "dram__bytes_write.sum) into profiles/traffic.json and exit")
    ap.add_argument("--traffic-key", help="key to record under (e.g. td_qd_1024:qd)")
    ap.add_argument("--kernel-regex", help="kernels of the log that make up one launch/call")
    ap.add_argument("--per-call", type=int, default=1,
                    help="matching launches per call (their bytes are summed)")
    ap.add_argument("--command", default="", help="the ncu command, stored with the record")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers

def dist_env():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def reduce_max(value, world):
    """Max of a host-side value over ranks (timings only; no data path)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rng(cfg, rank):
    """The generator of rank `rank`'s independent problem for workload `cfg`
    (rank 0 uses the workload's own seed)."""
    from paper_2101_06584_gb300 import inputs as I
    return np.random.Generator(np.random.PCG64(I.SEED_BASE + cfg + 1000 * rank))


def aggregate_value(world, mads_per_step, steps, max_total_ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * mads_per_step * steps / (max_total_ms * 1e-3)


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
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        power = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(float(r[0]) for r in rows),
                "sm_max_mhz": max(float(r[1]) for r in rows), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(power) if power else None}


def peaks(torch, mm):
    """Measured pipe rates at this run's clocks (the roofline denominators):
    FP64 lane-operations/s for add, mul, fma, int8 ops/s of mma.sync s8 and
    TwoSum, FastTwoSum and TwoProd per second on the integer pipes."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = sms * 8
    out = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    res = {}
    for kind, name, iters, ops in ((0, "dadd", 2048, 8), (1, "dmul", 2048, 8), (2, "dfma", 2048, 8),
                                   (3, "mma_s8", 4096, 4 * 8192 / 32), (4, "int_two_sum", 1024, 4),
                                   (5, "int_fast_two_sum", 1024, 4), (6, "int_two_prod", 1024, 4)):
        mm.peak_probe(kind, blocks, 16, out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mm.peak_probe(kind, blocks, iters, out)
        e1.record()
        torch.cuda.synchronize()
        res[name] = blocks * 256 * iters * ops / (e0.elapsed_time(e1) * 1e-3)
    return res


# ---------------------------------------------------------------- accuracy
#
# The error of a computed product against the exact one, on sampled entries
# (a seeded set of random entries plus whole rows).  Each exact entry
# c_ij = sum_p sum_{c,d} a_ip[c] b_pj[d] is a sum of binary64 products; every
# product is split exactly into two binary64 (Veltkamp's splitting and
# Dekker's product, exact while nothing overflows or underflows -- checked),
# and math.fsum, which returns the correctly rounded value of the exact sum of
# its arguments, peels the exact sum into a non-overlapping expansion
# s0 + s1 + ... (s_t the rounded remainder of the terms after s0..s_{t-1}).
# The residual of any candidate c_hat is then fsum(s + (-c_hat)), rounded
# once.  This is independent of the library (plain Python floats).

SPLIT = 134217729.0                 # 2**27 + 1


def _exact_products(a, b):
    """(p, e) with a*b = p + e exactly, elementwise (Dekker's product on
    Veltkamp's halves)."""
    p = a * b
    t = SPLIT * a
    ah = t - (t - a)
    al = a - ah
    t = SPLIT * b
    bh = t - (t - b)
    bl = b - bh
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def _expansion(terms, cap):
    """Non-overlapping expansion (list of binary64) of the exact sum of terms,
    stopped after ``cap`` components (the part left is then below about
    2^(-53 cap) of the sum's magnitude)."""
    out = []
    rest = list(terms)
    for _ in range(cap):
        s = math.fsum(rest)
        if s == 0.0:
            break
        out.append(s)
        rest.append(-s)
    return out


def exact_entries_task(args):
    """Exact expansions and sum_p |a_ip| |b_pj| for the pairs (A row r, B column
    c): A_rows (P, R, k), B_cols (P, k, Cn), pairs [(r, c)].  Returns a list of
    (expansion, absdot)."""
    A_rows, B_cols, pairs = args
    P = A_rows.shape[0]
    ri = np.array([r for r, _ in pairs])
    ci = np.array([c for _, c in pairs])
    a = A_rows[:, ri, :]                              # (P, npairs, k)
    b = np.transpose(B_cols[:, :, ci], (0, 2, 1))      # (P, npairs, k)
    nz_a, nz_b = np.abs(a[a != 0]), np.abs(b[b != 0])
    if nz_a.size and nz_b.size:
        lo = nz_a.min() * nz_b.min()
        hi = nz_a.max() * nz_b.max()
        if lo < 2.0 ** -900 or hi > 2.0 ** 900:
            raise ValueError("entries outside the range in which the exact products are exact")
    parts = []
    for c in range(P):
        for d in range(P):
            p, e = _exact_products(a[c], b[d])
            parts.append(p)
            parts.append(e)
    terms = np.concatenate(parts, axis=1)             # (npairs, 2 P^2 k)
    absdot = np.einsum("ik,ik->i", np.abs(a.sum(axis=0)), np.abs(b.sum(axis=0)))
    return [(_expansion(terms[t].tolist(), P + 3), float(absdot[t])) for t in range(len(pairs))]


def sample_entries(m, n, count, rng, full_rows=2):
    """Seeded sample: ``count`` random (i, j) plus ``full_rows`` whole rows."""
    ent = set()
    for _ in range(count):
        ent.add((int(rng.integers(m)), int(rng.integers(n))))
    for r in rng.choice(m, size=min(full_rows, m), replace=False):
        ent.update((int(r), j) for j in range(n))
    return sorted(ent)


class ExactReference:
    """Exact values of sampled entries of A B (planes (P, m, k), (P, k, n)),
    computed once on the host cores by a spawned process pool."""

    def __init__(self, A, B, entries, pool=None):
        self.entries = list(entries)
        A = np.asarray(A, dtype=np.float64)
        B = np.asarray(B, dtype=np.float64)
        tasks = []
        by_row = {}
        for (i, j) in self.entries:
            by_row.setdefault(i, []).append(j)
        singles = []
        for i, js in sorted(by_row.items()):
            if len(js) >= 64:                          # a whole (or long) row: chunks of 128 columns
                for s in range(0, len(js), 128):
                    cols = js[s:s + 128]
                    tasks.append((A[:, [i], :], B[:, :, cols], [(0, t) for t in range(len(cols))]))
            else:
                singles.extend((i, j) for j in js)
        for s in range(0, len(singles), 16):
            chunk = singles[s:s + 16]
            tasks.append((A[:, [i for i, _ in chunk], :], B[:, :, [j for _, j in chunk]],
                          [(t, t) for t in range(len(chunk))]))
        res = pool.map(exact_entries_task, tasks) if pool is not None else map(exact_entries_task, tasks)
        flat = [x for part in res for x in part]
        order = [(i, j) for i, js in sorted(by_row.items()) if len(js) >= 64 for j in js] + singles
        got = dict(zip(order, flat))
        self.exp = [got[e][0] for e in self.entries]
        self.absdot = np.array([got[e][1] for e in self.entries])
        self.value = np.array([x[0] if x else 0.0 for x in self.exp])

    def errors(self, C):
        """err_abs = ||C_hat - C||_F / || |A||B| ||_F, err_rel = ||C_hat - C||_F /
        ||C||_F and the worst entry's |c_hat - c| / (|A||B|)_ij over the
        sample, for C_hat given as planes (Pc, m, n) (or one plane (m, n))
        whose sampled entries are read here."""
        ii = np.array([i for i, _ in self.entries])
        jj = np.array([j for _, j in self.entries])
        if isinstance(C, np.ndarray):
            chat = (C if C.ndim == 3 else C[None])[:, ii, jj]      # (Pc, entries)
        else:                                           # a torch tensor: gather on its device
            import torch
            Ct = C if C.dim() == 3 else C[None]
            chat = Ct[:, torch.as_tensor(ii, device=Ct.device),
                      torch.as_tensor(jj, device=Ct.device)].cpu().numpy()
        res = np.array([math.fsum(s + [-float(x) for x in chat[:, t]])
                        for t, s in enumerate(self.exp)])
        num = math.sqrt(math.fsum(res * res))
        den_abs = math.sqrt(math.fsum(self.absdot * self.absdot))
        den_c = math.sqrt(math.fsum(self.value * self.value))
        with np.errstate(divide="ignore", invalid="ignore"):
            worst = np.where(self.absdot > 0, np.abs(res) / self.absdot, 0.0)
        return {"err_abs": num / den_abs if den_abs else 0.0,
                "err_rel": num / den_c if den_c else (0.0 if num == 0 else math.inf),
                "max_abs": float(worst.max()) if worst.size else 0.0}


# precision p of the normwise bound n 2^-p each product is checked against
# (the binary64-only product: its bound is k 2^-53)
GEMM_PBITS = {"d": 53, "dd": 100, "td": 150, "qd": 200}
# "enabled": accuracy figures and slice-count selection run (rank 0 of a
# single-rank run); otherwise the slicing workloads take FIXED_SLICES
_ACC = {"pool": None, "refs": {}, "enabled": False}
FIXED_SLICES = {"dd": 13, "td": 22, "qd": 29}


def exact_reference(key, A, B, entries):
    """The ExactReference of sampled entries of A B, computed once per key."""
    if key not in _ACC["refs"]:
        _ACC["refs"][key] = ExactReference(A, B, entries, pool=_ACC["pool"])
    return _ACC["refs"][key]


def accuracy_of(ref, C, prec, k, bound_factor=1.0):
    """Errors of C against the exact product with the pass/fail bound
    bound_factor * k 2^-p of its precision."""
    e = ref.errors(C)
    bound = bound_factor * k * 2.0 ** -GEMM_PBITS[prec]
    return dict(e, bound=bound, meets_bound=bool(e["err_abs"] <= bound))


def fp64_only_accuracy(mm, ref, A, B, k):
    """Errors of the binary64-only product of the leading planes."""
    return accuracy_of(ref, mm.gemm_fp64(A[0], B[0]), "d", k)


def choose_slices(run, ref, bound, start, smax):
    """The smallest slice count whose product meets ``bound`` (normwise, on
    the sampled entries): from ``start`` downward while the bound holds, or
    upward to ``smax`` when it does not hold at ``start``.  ``run(S)`` returns
    the product.  Returns (S or None, {S: err_abs} of every count tried)."""
    tried = {}

    def err(S):
        if S not in tried:
            tried[S] = ref.errors(run(S))["err_abs"]
        return tried[S]
    S = start
    if err(S) <= bound:
        while S > 1 and err(S - 1) <= bound:
            S -= 1
        return S, tried
    while S < smax:
        S += 1
        if err(S) <= bound:
            return S, tried
    return None, tried


def error_pool():
    """A spawn-started process pool over the host cores (safe after CUDA
    initialisation, unlike fork)."""
    import multiprocessing as mp
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    return mp.get_context("spawn").Pool(max(1, min(cores, 32)))


# --------------------------------------------------------------- workloads

class Workload:
    """One benchmark workload: device inputs, a step, and its dominant kernel."""
    name = ""
    launches_per_step = 1

    def timed_step(self, stream):
        """Run one step; returns [(start, end)] events around each dominant launch."""
        raise NotImplementedError


class TdQd(Workload):
    name = "td_qd"

    def __init__(self, torch, mm, I, rank, n=1024):
        self.torch, self.mm, self.n = torch, mm, n
        self.precs = ("td", "qd")
        rng = replica_rng(1, rank)
        self.host = {}
        self.dev = {}
        for prec in self.precs:
            P = I.P_OF[prec]
            A, B = I.cancelling_pair(P, n, n, n, rng)
            self.host[prec] = (A, B)
            self.dev[prec] = (torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                              torch.empty((P, n, n), dtype=torch.float64, device="cuda"))
        self.mads = len(self.precs) * n ** 3
        self.launches_per_step = 2
        self.dominant = "qd"
        self.config = {"workload": "TD GEMM + QD GEMM, m=n=k=%d, k-sequential FP64-EFT" % n,
                       "m": n, "n": n, "k": n, "precisions": list(self.precs)}

    def timed_step(self, stream):
        torch = self.torch
        evs = {}
        for prec in self.precs:
            A, B, C = self.dev[prec]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            self.mm.gemm_plain(prec, A, B, out=C)
            e1.record(stream)
            evs[prec] = (e0, e1)
        return evs

    def roofline(self, launch_ms, pk):
        n = self.n
        ti = self.mm.tile_info("qd", self.mm.default_tile("qd", n, n, n))
        r = kseq_roofline("qd", n ** 3, statistics.mean(launch_ms["qd"]), pk, ti)
        r.update({"kernel": "gemm_kseq_kernel<4,%d,%d,%d,%d,%d,ints=%d> (QD)" % (
                      ti["bm"], ti["bn"], ti["bk"], ti["tm"], ti["tn"], ti["int_ops"]),
                  "traffic": recorded_traffic("td_qd_%d:qd" % n),
                  "unit_of_work": "QD multiply-add", "units_per_launch": n ** 3,
                  "per_precision_mad_s": {p: n ** 3 / (statistics.mean(launch_ms[p]) * 1e-3)
                                          for p in self.precs}})
        return r

    def accuracy(self):
        """Errors of the TD and QD products and of the binary64-only product of
        their leading planes, on 256 sampled entries plus 2 whole rows."""
        out = {}
        n = self.n
        for prec in self.precs:
            A, B = self.host[prec]
            ref = exact_reference(("cfg1", prec, n), A, B,
                                  sample_entries(n, n, 256, np.random.default_rng(11 + len(prec))))
            Ad, Bd, C = self.dev[prec]
            self.mm.gemm_plain(prec, Ad, Bd, out=C)
            out[prec] = dict(accuracy_of(ref, C, prec, n), fp64_only=fp64_only_accuracy(self.mm, ref, Ad, Bd, n),
                             entries=len(ref.entries))
        return out

    def e2e(self, steps, world):
        torch = self.torch
        pinned = {p: tuple(torch.from_numpy(x).pin_memory() for x in self.host[p]) for p in self.precs}
        outs = {p: torch.empty(self.dev[p][2].shape, dtype=torch.float64).pin_memory()
                for p in self.precs}
        h2d = sum(x.numel() * 8 for p in self.precs for x in pinned[p])
        d2h = sum(outs[p].numel() * 8 for p in self.precs)

        def one():
            for p in self.precs:
                A, B, C = self.dev[p]
                A.copy_(pinned[p][0], non_blocking=True)
                B.copy_(pinned[p][1], non_blocking=True)
                self.mm.gemm_plain(p, A, B, out=C)
                outs[p].copy_(C, non_blocking=True)
            torch.cuda.synchronize()
        one()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(steps):
            one()
        barrier(world)
        secs = reduce_max(time.perf_counter() - t0, world)
        return {"value": world * self.mads * steps / secs, "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}


class DdSmall(Workload):
    name = "dd_small"

    def __init__(self, torch, mm, I, rank, n=128):
        self.torch, self.mm, self.n = torch, mm, n
        rng = replica_rng(0, rank)
        self.A = torch.from_numpy(I.uniform(2, (n, n), rng)).cuda()
        self.B = torch.from_numpy(I.uniform(2, (n, n), rng)).cuda()
        self.C = torch.empty((2, n, n), dtype=torch.float64, device="cuda")
        self.mads = n ** 3
        self.host = (host_of(self.A), host_of(self.B))
        self.config = {"workload": "DD GEMM m=n=k=%d, k-sequential FP64-EFT" % n, "m": n, "n": n, "k": n,
                       "launch": "the mpgemm_dd call captured in a CUDA graph, one replay per step"}

    def accuracy(self):
        """Errors of the DD product and of the binary64-only product over every entry."""
        n = self.n
        ref = exact_reference(("cfg0", n), *self.host, [(i, j) for i in range(n) for j in range(n)])
        self.mm.gemm_plain("dd", self.A, self.B, out=self.C)
        return {"dd": dict(accuracy_of(ref, self.C, "dd", n),
                           fp64_only=fp64_only_accuracy(self.mm, ref, self.A, self.B, n), entries=n * n)}

    def _graph(self):
        """The library call captured once in a CUDA graph: a 128^3 product runs
        for about 0.1 ms, and a call enqueued from Python after the timing event
        would leave the GPU idle for tens of microseconds inside the timed
        region; a graph replay is enqueued in a few."""
        torch = self.torch
        if getattr(self, "graph", None) is None:
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                self.mm.gemm_plain("dd", self.A, self.B, out=self.C)
            torch.cuda.current_stream().wait_stream(side)
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self.mm.gemm_plain("dd", self.A, self.B, out=self.C)
        return self.graph

    def timed_step(self, stream):
        graph = self._graph()
        e0, e1 = self.torch.cuda.Event(enable_timing=True), self.torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        return {"dd": (e0, e1)}

    def roofline(self, launch_ms, pk):
        ach = self.mads * 20 / (statistics.mean(launch_ms["dd"]) * 1e-3)
        # the split-K variant for reference (not bit-identical, within bound)
        ms = _time_call(self.torch, lambda: self.mm.gemm("dd", self.A, self.B, out=self.C, split_k=8), 20)
        ti = self.mm.tile_info("dd", self.mm.default_tile("dd", self.n, self.n, self.n))
        kern = "gemm_kseq_kernel<2,%d,%d,%d,%d,%d,ints=%d>" % (ti["bm"], ti["bn"], ti["bk"], ti["tm"], ti["tn"],
                                                               ti["int_ops"])
        r = kseq_roofline("dd", self.mads, statistics.mean(launch_ms["dd"]), pk, ti)
        return {**r, "kernel": kern, "traffic": None,
                "unit_of_work": "DD multiply-add", "units_per_launch": self.mads,
                "note": "16K entries = 512 warps, one per SM sub-partition at most (FP64 floor 0.84 of peak); "
                        "warp split-K 8 (not k-sequential) runs at %.3g mad/s" % (self.mads / (ms * 1e-3))}


class DdInt8(Workload):
    """DD GEMM through the slicing form; engine "int8" (mma.sync s8) or "tc"
    (the same digits as bf16 on tcgen05).  With S = None the slice count is
    the smallest that meets the DD bound n 2^-100 on the sampled entries."""
    name = "dd_int8"

    # (algo, first slice count tried, largest allowed, fixed count without the search)
    FORMS = {"int8": ("int8", 14, 16, FIXED_SLICES["dd"]), "tc": ("bf16", 14, 16, FIXED_SLICES["dd"]),
             "crt_int8": ("crt", 28, 49, 28), "crt_tc": ("crt_bf16", 28, 49, 28)}

    def __init__(self, torch, mm, I, rank, n=4096, S=None, engine="int8"):
        self.torch, self.mm, self.n, self.engine = torch, mm, n, engine
        self.algo, self.s_start, self.s_max, s_fixed = self.FORMS[engine]
        self.crt = self.algo.startswith("crt")
        rng = replica_rng(2, rank)
        A, B = I.uniform(2, (n, n), rng), I.uniform(2, (n, n), rng)
        self.host = (A, B)
        self.A = torch.from_numpy(A).cuda()
        self.B = torch.from_numpy(B).cuda()
        self.C = torch.empty((2, n, n), dtype=torch.float64, device="cuda")
        self.search = None
        if S is None:
            S, self.search = self._choose(n) if _ACC["enabled"] else (s_fixed, None)
        self.S = S
        self.ws = torch.empty(mm.workspace_size("dd", n, n, n, algo=self.algo, slices=S),
                              dtype=torch.uint8, device="cuda")
        self.mads = n ** 3
        # scale + slice for each operand (+ exponent padding when n is not a tile multiple) and the product
        self.launches_per_step = 5 if n % 128 == 0 else 7
        if engine != "int8":
            self.launches_per_step += 1          # the workspace-header clear
        eng = ("mma.sync s8 engine" if engine in ("int8", "crt_int8")
               else "tcgen05 engine (bf16 operands, TMEM accumulators)")
        if self.crt:
            form = "CRT form (Ozaki scheme II), N=%d moduli, beta=%d bits" % (S, mm.crt_beta(S, n))
            self.launches_per_step = 6 + (1 if engine == "crt_tc" else 0)
        else:
            form = "INT8 error-free slicing form, S=%d" % S
        self.config = {"workload": "DD GEMM m=n=k=%d, %s, %s" % (n, form, eng),
                       "m": n, "n": n, "k": n, "slices": S, "engine": engine,
                       "slices_rule": ("smallest %s meeting n 2^-100 on the sampled entries" %
                                       ("N" if self.crt else "S")) if self.search is not None else "given"}

    def reference(self):
        n = self.n
        return exact_reference(("cfg2", n), *self.host, sample_entries(n, n, 256, np.random.default_rng(12)))

    def _choose(self, n):
        ref = self.reference()

        def run(S):
            ws = self.torch.empty(self.mm.workspace_size("dd", n, n, n, algo=self.algo, slices=S),
                                  dtype=self.torch.uint8, device="cuda")
            return self.mm.gemm("dd", self.A, self.B, out=self.C, algo=self.algo, slices=S, workspace=ws)
        S, tried = choose_slices(run, ref, n * 2.0 ** -100, self.s_start, self.s_max)
        if S is None:
            raise RuntimeError("no count up to %d meets n 2^-100: %r" % (self.s_max, tried))
        return S, {str(k): v for k, v in sorted(tried.items())}

    def timed_step(self, stream):
        e0, e1 = self.torch.cuda.Event(enable_timing=True), self.torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        self.mm.gemm("dd", self.A, self.B, out=self.C, algo=self.algo, slices=self.S, workspace=self.ws)
        e1.record(stream)
        return {"call": (e0, e1)}

    def accuracy(self):
        """Errors of the sliced product (at the chosen S), of the FP64-EFT
        product of the same inputs and of the binary64-only product."""
        n = self.n
        ref = self.reference()
        self.mm.gemm("dd", self.A, self.B, out=self.C, algo=self.algo, slices=self.S, workspace=self.ws)
        out = {"dd": dict(accuracy_of(ref, self.C, "dd", n), slices=self.S, entries=len(ref.entries))}
        if self.search is not None:
            out["dd"]["err_abs_by_slices"] = self.search
        if getattr(self, "plain_C", None) is None:
            self.plain_C = self.mm.gemm_plain("dd", self.A, self.B)
        out["dd"]["fp64_eft"] = accuracy_of(ref, self.plain_C, "dd", n)
        out["dd"]["fp64_only"] = fp64_only_accuracy(self.mm, ref, self.A, self.B, n)
        return out

    def roofline(self, launch_ms, pk):
        S, n = self.S, self.n
        pairs = S if self.crt else S * (S + 1) // 2
        ops = 2.0 * pairs * n ** 3
        ms = statistics.mean(launch_ms["call"])
        ach = ops / (ms * 1e-3)
        self.plain_C = self.torch.empty_like(self.C)
        plain_ms = _time_call(self.torch, lambda: self.mm.gemm_plain("dd", self.A, self.B, out=self.plain_C), 1)
        if self.engine == "crt_int8":
            peak, src, unit, kern = (pk["mma_s8"], "measured mma.sync s8 probe at this run's clocks",
                                     "Tint8op/s", "crt_gemm_kernel (mma.sync m16n8k32 s8) incl. residues and recovery")
            key = "dd_crtint8_%d_s%d:call" % (n, S)
        elif self.engine == "crt_tc":
            peak, src = bf16_peak()
            unit, kern = "TFLOP/s", "crt_tc_kernel (tcgen05.mma kind::f16, 128 x 128) incl. residues and recovery"
            key = "dd_crttc_%d_s%d:call" % (n, S)
        elif self.engine == "int8":
            peak, src, unit, kern = (pk["mma_s8"], "measured mma.sync s8 probe at this run's clocks "
                                     "(tcgen05 has no int8 kind on sm_103a)", "Tint8op/s",
                                     "ozaki_gemm_kernel (mma.sync m16n8k32 s8) incl. slicing")
            key = "dd_int8_%d_s%d:call" % (n, S)
        else:
            peak, src = bf16_peak()
            unit, kern = "TFLOP/s", ("ozaki_tc_pair_kernel (tcgen05.mma.cta_group::2 kind::f16, CTA pairs) "
                                     "incl. slicing")
            key = "dd_tc_%d_s%d:call" % (n, S)
        return {"bound": "tensor", "kernel": kern, "achieved": ach / 1e12, "peak": peak / 1e12,
                "unit": unit, "frac": ach / peak, "traffic": recorded_traffic(key),
                "ops_per_unit": 2 * pairs,
                "unit_of_work": "DD multiply-add (%d %s MACs)" % (pairs, "residue" if self.crt else "slice-pair"),
                "units_per_launch": n ** 3, "peak_source": src,
                "fp64_eft_ms": plain_ms, "speedup_vs_fp64_eft": plain_ms / ms}


class DdCrt(DdInt8):
    name = "dd_crt"

    def __init__(self, torch, mm, I, rank, n=4096, S=None):
        super().__init__(torch, mm, I, rank, n=n, S=S, engine="crt_tc")


class DdCrtInt8(DdInt8):
    name = "dd_crt_int8"

    def __init__(self, torch, mm, I, rank, n=4096, S=None):
        super().__init__(torch, mm, I, rank, n=n, S=S, engine="crt_int8")


class TdQdInt8(Workload):
    """The TD and QD GEMMs of td_qd through the slicing form (engine "int8" or "tc")."""
    name = "td_qd_int8"

    ALGO = {"int8": "int8", "tc": "bf16", "crt_tc": "crt_bf16", "crt2_tc": "crt2_bf16"}
    # first count tried (the library's defaults) and the largest, per precision
    START = {"td": (22, 40), "qd": (29, 40)}
    START_CRT = {"td": (44, 49)}
    START_CRT2 = {"qd": (30, 44)}

    def __init__(self, torch, mm, I, rank, n=1024, engine="int8", S=None):
        self.torch, self.mm, self.n, self.engine = torch, mm, n, engine
        self.algo = self.ALGO[engine]
        self.crt = self.algo.startswith("crt")
        self.split = self.algo.startswith("crt2")
        self.precs = ("qd",) if self.split else ("td",) if self.crt else ("td", "qd")
        rng = replica_rng(1, rank)
        self.dev, self.host, self.search = {}, {}, {}
        for prec in ("td", "qd"):                 # drawn in this order whichever precisions run
            P = I.P_OF[prec]
            A, B = I.cancelling_pair(P, n, n, n, rng)
            if prec not in self.precs:
                continue
            self.host[prec] = (A, B)
            self.dev[prec] = [torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                              torch.empty((P, n, n), dtype=torch.float64, device="cuda"), None]
        starts = self.START_CRT2 if self.split else self.START_CRT if self.crt else self.START
        if S is None and not _ACC["enabled"]:
            S = {p: starts[p][0] if self.crt else FIXED_SLICES[p] for p in self.precs}
        if S is None:
            # the smallest count meeting n 2^-150 (TD) / n 2^-200 (QD) on the
            # sampled entries, searched from the library's defaults
            S = {}
            for prec in self.precs:
                S[prec], self.search[prec] = self._choose(prec, *starts[prec])
        self.S = S
        for prec in self.precs:
            self.dev[prec][3] = torch.empty(mm.workspace_size(prec, n, n, n, algo=self.algo, slices=S[prec]),
                                            dtype=torch.uint8, device="cuda")
        self.mads = len(self.precs) * n ** 3
        eng = "mma.sync s8 engine" if engine == "int8" else "tcgen05 engine"
        if self.split:
            self.launches_per_step = 7
            self.config = {"workload": "QD GEMM, m=n=k=%d, CRT form with split integers (N = %d moduli, beta = %d "
                                       "bits, 3N products), %s, inputs of the main workload"
                                       % (n, self.S["qd"], mm.crt_beta(self.S["qd"], n, split=True), eng),
                           "m": n, "n": n, "k": n, "slices": self.S, "engine": engine,
                           "slices_rule": "smallest N meeting n 2^-200 on the sampled entries"
                           if self.search else "given"}
        elif self.crt:
            self.launches_per_step = 7
            self.config = {"workload": "TD GEMM, m=n=k=%d, CRT form (N = %d moduli, beta = %d bits), %s, "
                                       "inputs of the main workload" % (n, self.S["td"], mm.crt_beta(self.S["td"], n),
                                                                         eng),
                           "m": n, "n": n, "k": n, "slices": self.S, "engine": engine,
                           "slices_rule": "smallest N meeting n 2^-150 on the sampled entries"
                           if self.search else "given"}
        else:
            self.launches_per_step = 2 * (5 if n % 128 == 0 else 7) + (0 if engine == "int8" else 2)
            self.config = {"workload": "TD GEMM + QD GEMM, m=n=k=%d, INT8 error-free slicing form "
                                       "(S = %d / %d), %s, inputs of the main workload"
                                       % (n, self.S["td"], self.S["qd"], eng),
                           "m": n, "n": n, "k": n, "slices": self.S, "engine": engine,
                           "slices_rule": "smallest S meeting n 2^-150 (TD) / n 2^-200 (QD) on the sampled "
                                          "entries" if self.search else "given"}

    def reference(self, prec):
        n = self.n
        return exact_reference(("cfg1", prec, n), *self.host[prec],
                               sample_entries(n, n, 256, np.random.default_rng(11 + len(prec))))

    def _choose(self, prec, start, smax):
        n = self.n
        A, B, C, _ = self.dev[prec]

        def run(S):
            ws = self.torch.empty(self.mm.workspace_size(prec, n, n, n, algo=self.algo, slices=S),
                                  dtype=self.torch.uint8, device="cuda")
            return self.mm.gemm(prec, A, B, out=C, algo=self.algo, slices=S, workspace=ws)
        S, tried = choose_slices(run, self.reference(prec), n * 2.0 ** -GEMM_PBITS[prec], start, smax)
        if S is None:
            raise RuntimeError("no count up to %d meets the %s bound: %r" % (smax, prec, tried))
        return S, {str(k): v for k, v in sorted(tried.items())}

    def accuracy(self):
        """Errors of the sliced TD and QD products at the chosen slice counts."""
        out = {}
        for prec in self.precs:
            A, B, C, ws = self.dev[prec]
            ref = self.reference(prec)
            self.mm.gemm(prec, A, B, out=C, algo=self.algo, slices=self.S[prec], workspace=ws)
            out[prec] = dict(accuracy_of(ref, C, prec, self.n), slices=self.S[prec], entries=len(ref.entries))
            if self.search:
                out[prec]["err_abs_by_slices"] = self.search[prec]
        return out

    def timed_step(self, stream):
        evs = {}
        for prec in self.precs:
            A, B, C, ws = self.dev[prec]
            e0, e1 = self.torch.cuda.Event(enable_timing=True), self.torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            self.mm.gemm(prec, A, B, out=C, algo=self.algo, slices=self.S[prec], workspace=ws)
            e1.record(stream)
            evs[prec] = (e0, e1)
        return evs

    def roofline(self, launch_ms, pk):
        n = self.n
        dom = self.precs[-1]
        S = self.S[dom]
        # residue products per multiply-add: N, or 4N with split integers
        # (hh, the two halves of mid, ll)
        pairs = 4 * S if self.split else S if self.crt else S * (S + 1) // 2
        ms = statistics.mean(launch_ms[dom])
        ach = 2.0 * pairs * n ** 3 / (ms * 1e-3)
        plain = {}
        for prec in self.precs:
            A, B, C, _ = self.dev[prec]
            plain[prec] = _time_call(self.torch, lambda: self.mm.gemm_plain(prec, A, B, out=C), 1)
        if self.engine == "int8":
            peak, src, unit = pk["mma_s8"], "measured mma.sync s8 probe", "Tint8op/s"
        else:
            (peak, src), unit = bf16_peak(), "TFLOP/s"
        # FP64 work of the QD call: one QDadd (87 of the 210 operations of a QD
        # multiply-add) per output per group of ten weights (S weights; the
        # first group of a tile needs none on the tcgen05 engine)
        fp64_ops = 0 if self.crt else (n * n) * (-(-S // 10)) * FP64_OPS_PER_MAD["qd"] * 87 // 210
        kern = ("QD CRT form with split integers (crt_tc_kernel) incl. residues and recovery" if self.split
                else "TD CRT form (crt_tc_kernel) incl. residues and recovery" if self.crt
                else "QD slicing form (%s) incl. slicing" % self.engine)
        return {"bound": "tensor", "kernel": kern,
                "achieved": ach / 1e12, "peak": peak / 1e12, "unit": unit, "peak_source": src,
                "frac": ach / peak, "traffic": None, "ops_per_unit": 2 * pairs,
                "unit_of_work": "%s multiply-add (%d %s MACs)" % (dom.upper(), pairs,
                                                                  "residue" if self.crt else "slice-pair"),
                "units_per_launch": n ** 3,
                "fp64_epilogue_ops_per_call": fp64_ops,
                "per_precision_mad_s": {p: n ** 3 / (statistics.mean(launch_ms[p]) * 1e-3)
                                        for p in self.precs},
                "speedup_vs_fp64_eft": {p: plain[p] / statistics.mean(launch_ms[p]) for p in self.precs}}


class DdTc(DdInt8):
    name = "dd_tc"

    def __init__(self, torch, mm, I, rank, n=4096, S=None):
        super().__init__(torch, mm, I, rank, n=n, S=S, engine="tc")


class TdQdTc(TdQdInt8):
    name = "td_qd_tc"

    def __init__(self, torch, mm, I, rank, n=1024):
        super().__init__(torch, mm, I, rank, n=n, engine="tc")


class TdCrt(TdQdInt8):
    """The TD GEMM of the main workload through the CRT form on tcgen05 (QD
    needs more bits than 49 moduli of at most 256 give one integer product)."""
    name = "td_crt"

    def __init__(self, torch, mm, I, rank, n=1024):
        super().__init__(torch, mm, I, rank, n=n, engine="crt_tc")


class QdCrt(TdQdInt8):
    """The QD GEMM of the main workload through the CRT form with split
    integers on tcgen05."""
    name = "qd_crt"

    def __init__(self, torch, mm, I, rank, n=1024):
        super().__init__(torch, mm, I, rank, n=n, engine="crt2_tc")


class Elementwise(Workload):
    """The paper's elementwise benchmarks (Sec. 4, Figs. 2-4): DDadd/DDmul,
    TDaddq, merge TDadd (Alg. 3), TDmul, QDadd/QDmul, and the variants TDmulq,
    accurate TD product and accurate QD addition, over SoA vectors of n
    elements, every op on its own buffers (inputs far larger than L2)."""
    name = "elementwise"
    # (precision, op, FP64 operations per element of the implemented sequence;
    # for the accurate variants: two TwoSums per accumulator step, plus the
    # tail additions where four components can be out -- four emissions need
    # the steps of terms 2-5, so the tail starts at the sixth term at the
    # earliest and grows from the seventh; the FP64-pipe counters agree)
    OPS = (("dd", "add", 11), ("dd", "mul", 9), ("td", "add", 81), ("td", "addm", 45), ("td", "mul", 47),
           ("td", "mulq", 123), ("td", "mula", 148), ("qd", "add", 87), ("qd", "mul", 123),
           ("qd", "adda", 104))

    def __init__(self, torch, mm, I, rank, n=1 << 24):
        self.torch, self.mm, self.n = torch, mm, n
        rng = replica_rng(0, rank)
        self.dev = {}
        for prec in ("dd", "td", "qd"):
            P = I.P_OF[prec]
            x, y = I.random_mp(P, n, rng), I.random_mp(P, n, rng)
            self.dev[prec] = (torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(),
                              torch.empty((P, n), dtype=torch.float64, device="cuda"))
        self.mads = len(self.OPS) * n          # elements processed per step
        self.launches_per_step = len(self.OPS)
        self.config = {"workload": "elementwise DD/TD/QD add and mul and the TD/QD variants, n=%d elements per op"
                                   % n, "n": n}

    def timed_step(self, stream):
        evs = {}
        for prec, op, _ in self.OPS:
            x, y, r = self.dev[prec]
            e0, e1 = self.torch.cuda.Event(enable_timing=True), self.torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            self.mm.vec(prec, op, x, y, out=r)
            e1.record(stream)
            evs[prec + "_" + op] = (e0, e1)
        return evs

    def roofline(self, launch_ms, pk):
        per_op = {}
        for prec, op, ops in self.OPS:
            P = {"dd": 2, "td": 3, "qd": 4}[prec]
            ms = statistics.mean(launch_ms[prec + "_" + op])
            el_s = self.n / (ms * 1e-3)
            per_op[prec + "_" + op] = {"elements_s": el_s, "fp64_ops_per_element": ops,
                                       "frac_fp64": el_s * ops / pk["dfma"],
                                       "hbm_gb_s": el_s * 3 * P * 8 / 1e9}
        # the slowest op in FP64 throughput
        worst = min(per_op.items(), key=lambda kv: kv[1]["frac_fp64"])
        return {"bound": "alu", "kernel": "elementwise ops (one launch each)", "unit": "TFP64op/s",
                "achieved": worst[1]["elements_s"] * worst[1]["fp64_ops_per_element"] / 1e12,
                "peak": pk["dfma"] / 1e12, "frac": worst[1]["frac_fp64"], "frac_of": worst[0],
                "traffic": None, "per_op": per_op}


class Strassen(Workload):
    """The Strassen form (Sec. 3) beside the block algorithm: DD 4096^3 (the
    slicing forms' inputs) and QD 1024^3 (the main workload's inputs), one and
    two levels over the k-sequential kernel."""
    name = "strassen"
    CASES = (("dd", 1), ("dd", 2), ("qd", 1), ("qd", 2))

    def __init__(self, torch, mm, I, rank, n_dd=4096, n_qd=1024):
        self.torch, self.mm = torch, mm
        self.n = {"dd": n_dd, "qd": n_qd}
        self.dev, self.ws = {}, {}
        rng = replica_rng(2, rank)
        A, B = I.uniform(2, (n_dd, n_dd), rng), I.uniform(2, (n_dd, n_dd), rng)
        self.dev["dd"] = (torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                          torch.empty((2, n_dd, n_dd), dtype=torch.float64, device="cuda"))
        A, B = I.cancelling_pair(4, n_qd, n_qd, n_qd, replica_rng(1, rank))
        self.dev["qd"] = (torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                          torch.empty((4, n_qd, n_qd), dtype=torch.float64, device="cuda"))
        for prec, L in self.CASES:
            n = self.n[prec]
            self.ws[(prec, L)] = torch.empty(mm.workspace_size(prec, n, n, n, strassen=L), dtype=torch.uint8,
                                             device="cuda")
        self.mads = sum(self.n[p] ** 3 for p, _ in self.CASES)
        # per level: 18 block additions and 7 products, recursively; the leaves are one launch each
        self.launches_per_step = sum(18 * (7 ** L - 1) // 6 + 7 ** L for _, L in self.CASES)
        self.config = {"workload": "Strassen form: DD m=n=k=%d and QD m=n=k=%d, 1 and 2 levels" % (n_dd, n_qd),
                       "cases": ["%s L=%d" % c for c in self.CASES]}

    def timed_step(self, stream):
        evs = {}
        for prec, L in self.CASES:
            A, B, C = self.dev[prec]
            e0, e1 = self.torch.cuda.Event(enable_timing=True), self.torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            self.mm.gemm(prec, A, B, out=C, strassen=L, workspace=self.ws[(prec, L)])
            e1.record(stream)
            evs["%s_L%d" % (prec, L)] = (e0, e1)
        return evs

    def accuracy(self):
        """Errors of the DD Strassen products (the DD 4096^3 workload's inputs)
        against the bound 4^L n 2^-100."""
        n = self.n["dd"]
        A, B, C = self.dev["dd"]
        ref = exact_reference(("cfg2", n), host_of(A), host_of(B),
                              sample_entries(n, n, 256, np.random.default_rng(12)))
        out = {}
        for prec, L in self.CASES:
            if prec == "dd":
                self.mm.gemm(prec, A, B, out=C, strassen=L, workspace=self.ws[(prec, L)])
                out["dd_L%d" % L] = accuracy_of(ref, C, "dd", n, bound_factor=4.0 ** L)
        return out

    def roofline(self, launch_ms, pk):
        plain = {}
        for prec in ("dd", "qd"):
            A, B, C = self.dev[prec]
            plain[prec] = _time_call(self.torch, lambda: self.mm.gemm_plain(prec, A, B, out=C), 1)
        cases = {}
        for prec, L in self.CASES:
            n = self.n[prec]
            ms = statistics.mean(launch_ms["%s_L%d" % (prec, L)])
            # FP64 work actually done: 7^L leaf products of (n/2^L)^3 mads
            leaf_mads = 7 ** L * (n // 2 ** L) ** 3
            cases["%s_L%d" % (prec, L)] = {"ms": ms, "nominal_mad_s": n ** 3 / (ms * 1e-3),
                                           "speedup_vs_block": plain[prec] / ms,
                                           "leaf": kseq_roofline(prec, leaf_mads, ms, pk, self._leaf_tile(prec, L))}
        worst = min(cases.items(), key=lambda kv: kv[1]["leaf"]["frac"])
        w = worst[1]["leaf"]
        return {"bound": "alu", "kernel": "gemm_kseq_kernel leaves + mat_addsub_kernel", "unit": "TFP64op/s",
                "achieved": w["achieved"], "peak": w["peak"], "frac": w["frac"], "frac_of": worst[0],
                "peak_source": w["peak_source"], "traffic": None, "block_ms": plain, "cases": cases}

    def _leaf_tile(self, prec, L):
        m = self.n[prec] // 2 ** L
        return self.mm.tile_info(prec, self.mm.default_tile(prec, m, m, m))


class Batched(Workload):
    name = "batched"

    def __init__(self, torch, mm, I, rank, count=512):
        self.torch, self.mm = torch, mm
        rng = replica_rng(3, rank)
        self.shapes = I.batch_shapes(count, rng)
        self.plans = {}
        self.keep = []
        for prec in ("dd", "qd"):
            P = I.P_OF[prec]
            triples = []
            for (m, n, k) in self.shapes:
                A = torch.from_numpy(I.uniform(P, (m, k), rng)).cuda()
                B = torch.from_numpy(I.uniform(P, (k, n), rng)).cuda()
                C = torch.empty((P, m, n), dtype=torch.float64, device="cuda")
                triples.append((A, B, C))
            self.keep.append(triples)
            self.plans[prec] = mm.BatchPlan(prec, triples, policy=None, reps=1)
        self.mads_per = sum(m * n * k for (m, n, k) in self.shapes)
        self.mads = 2 * self.mads_per
        self.launches_per_step = 2
        self.config = {"workload": "batched DD + QD, %d problems each, m,n,k log-uniform [16,512], "
                                   "one persistent launch per precision replayed from a CUDA graph"
                                   % count, "problems": count, "sum_mnk": self.mads_per,
                       "policy": {p: self.plans[p].policy for p in self.plans},
                       "tiles": {p: self.plans[p].info()["tiles"] for p in self.plans}}

    def timed_step(self, stream):
        evs = {}
        for prec in ("dd", "qd"):
            e0, e1 = self.torch.cuda.Event(enable_timing=True), self.torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            self.plans[prec].run()
            e1.record(stream)
            evs[prec] = (e0, e1)
        return evs

    def roofline(self, launch_ms, pk):
        ms = statistics.mean(launch_ms["qd"])
        policy = self.plans["qd"].policy
        ints = self.mm.batch_int_ops("qd", policy)
        r = kseq_roofline("qd", self.mads_per, ms, pk, {"int_ops": ints})
        kern = "batched_int_kernel<4>" if ints else "batched_kernel<4>"
        return {**r, "kernel": "%s (QD, persistent, policy %d)" % (kern, policy), "traffic": None,
                "unit_of_work": "QD multiply-add", "units_per_launch": self.mads_per,
                "per_precision_mad_s": {p: self.mads_per / (statistics.mean(launch_ms[p]) * 1e-3)
                                        for p in ("dd", "qd")}}


class Autograd(Workload):
    name = "autograd"

    def __init__(self, torch, mm, I, rank, n=2048):
        from paper_2101_06584_gb300.autograd import dd_matmul
        self.torch, self.mm, self.n, self.f = torch, mm, n, dd_matmul
        rng = replica_rng(4, rank)
        self.A = torch.from_numpy(I.uniform(2, (n, n), rng)).cuda().requires_grad_(True)
        self.B = torch.from_numpy(I.uniform(2, (n, n), rng)).cuda().requires_grad_(True)
        self.W = torch.from_numpy(I.uniform(2, (n, n), rng)).cuda()
        self.mads = 3 * n ** 3
        self.launches_per_step = 3
        self.config = {"workload": "DDMatmul forward + backward (dA = dC B^T, dB = A^T dC), "
                                   "m=n=k=%d, loss = sum(W*C)" % n, "m": n, "n": n, "k": n}

    def timed_step(self, stream):
        torch = self.torch
        self.A.grad = None
        self.B.grad = None
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        C = self.f(self.A, self.B)
        e1.record(stream)
        C.backward(self.W)
        return {"fwd": (e0, e1)}

    def roofline(self, launch_ms, pk):
        n = self.n
        ti = self.mm.tile_info("dd", self.mm.default_tile("dd", n, n, n))
        r = kseq_roofline("dd", n ** 3, statistics.mean(launch_ms["fwd"]), pk, ti)
        return {**r, "kernel": "gemm_kseq_kernel<2,%d,%d,%d,%d,%d,ints=%d> (DD forward)" % (
                    ti["bm"], ti["bn"], ti["bk"], ti["tm"], ti["tn"], ti["int_ops"]),
                "traffic": None, "unit_of_work": "DD multiply-add", "units_per_launch": n ** 3}


class AutogradTc(Autograd):
    """DDMatmul forward + backward on the tcgen05 slicing form (default slices)."""
    name = "autograd_tc"

    def __init__(self, torch, mm, I, rank, n=2048):
        super().__init__(torch, mm, I, rank, n=n)
        from paper_2101_06584_gb300.autograd import dd_matmul
        self.f = lambda A, B: dd_matmul(A, B, algo="bf16")
        # per product: header clear, scale and slice of both operands, the product kernel
        self.launches_per_step = 3 * 6
        self.config = dict(self.config, workload=self.config["workload"] + ", tcgen05 slicing form", engine="tc")

    def roofline(self, launch_ms, pk):
        S = 14
        pairs = S * (S + 1) // 2
        ms = statistics.mean(launch_ms["fwd"])
        ach = 2.0 * pairs * self.n ** 3 / (ms * 1e-3)
        peak, src = bf16_peak()
        return {"bound": "tensor", "kernel": "ozaki_tc_pair_kernel (forward call incl. slicing)",
                "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s", "frac": ach / peak,
                "peak_source": src, "traffic": None, "ops_per_unit": 2 * pairs,
                "unit_of_work": "DD multiply-add (%d slice-pair MACs)" % pairs, "units_per_launch": self.n ** 3}


class AutogradCrt(Autograd):
    """DDMatmul forward + backward on the tcgen05 CRT form, 26 moduli: at
    k = 2048 that keeps 94 bits per scaled entry, so each gradient entry is
    within n 2^-100 of its own |W| |B| dot product (23 moduli meet the
    normwise bound at 4096^3 but not every entry's)."""
    name = "autograd_crt"
    MODULI = 26

    def __init__(self, torch, mm, I, rank, n=2048):
        super().__init__(torch, mm, I, rank, n=n)
        from paper_2101_06584_gb300.autograd import dd_matmul
        self.f = lambda A, B: dd_matmul(A, B, algo="crt_bf16", slices=self.MODULI)
        # per product: header clear, scale and residues of both operands, the products, the recovery
        self.launches_per_step = 3 * 7
        self.config = dict(self.config, workload=self.config["workload"] + ", tcgen05 CRT form, %d moduli"
                           % self.MODULI, engine="crt_tc", moduli=self.MODULI)

    def roofline(self, launch_ms, pk):
        N = self.MODULI
        ms = statistics.mean(launch_ms["fwd"])
        ach = 2.0 * N * self.n ** 3 / (ms * 1e-3)
        peak, src = bf16_peak()
        return {"bound": "tensor", "kernel": "crt_tc_kernel (forward call incl. residues and recovery)",
                "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s", "frac": ach / peak,
                "peak_source": src, "traffic": None, "ops_per_unit": 2 * N,
                "unit_of_work": "DD multiply-add (%d residue MACs)" % N, "units_per_launch": self.n ** 3}


WORKLOADS = {"td_qd": TdQd, "dd_small": DdSmall, "dd_int8": DdInt8, "dd_tc": DdTc, "dd_crt": DdCrt,
             "dd_crt_int8": DdCrtInt8, "td_crt": TdCrt, "qd_crt": QdCrt,
             "td_qd_int8": TdQdInt8, "td_qd_tc": TdQdTc, "batched": Batched, "autograd": Autograd,
             "elementwise": Elementwise, "strassen": Strassen, "autograd_tc": AutogradTc,
             "autograd_crt": AutogradCrt}


def host_of(t):
    return t.detach().cpu().numpy()


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


class L2Flush:
    """Between timed steps: write a buffer larger than L2 (evicting every
    line of the workload), then read a second one.  The read evicts the
    written lines, so their write-back to HBM happens here and not inside the
    next step's first kernel, and the step starts with a cold L2 that holds
    no dirty line."""

    def __init__(self, torch):
        self.w = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        self.r = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        self.sink = torch.empty((), dtype=torch.float32, device="cuda")
        self.torch = torch

    def __call__(self):
        self.w.zero_()
        self.torch.sum(self.r, dim=0, out=self.sink)


def measure(torch, w, steps, warmup, world, local, flush, sample_clocks=True):
    """Warm up, then time exactly `steps` steps (L2 flushed before each, not
    timed), with a barrier and a synchronize on both sides."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        w.timed_step(stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(local) if sample_clocks else None
    launch_ms, step_ms = {}, []
    barrier(world)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    t0 = time.perf_counter()
    for _ in range(steps):
        flush()
        evs = w.timed_step(stream)
        end = torch.cuda.Event(enable_timing=True)
        end.record(stream)
        torch.cuda.synchronize()
        start = next(iter(evs.values()))[0]          # first launch of the step
        step_ms.append(start.elapsed_time(end))
        for k, (a, b) in evs.items():
            launch_ms.setdefault(k, []).append(a.elapsed_time(b))
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - t0
    clocks = sampler.stop() if sampler else None
    total_ms = reduce_max(sum(step_ms), world)
    return total_ms, launch_ms, clocks, wall


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

    flush = L2Flush(torch)
    _ACC["enabled"] = rank == 0 and world == 1 and not args.no_accuracy
    if _ACC["enabled"]:
        _ACC["pool"] = error_pool()
    pk = peaks(torch, mm)
    kw = {} if args.size is None else {"n": args.size}
    if args.slices is not None and args.workload in ("dd_int8", "dd_tc", "dd_crt", "dd_crt_int8"):
        kw["S"] = args.slices
    w = WORKLOADS[args.workload](torch, mm, I, rank, **kw)
    total_ms, launch_ms, clocks, wall = measure(torch, w, args.steps, args.warmup, world, local, flush)
    value = aggregate_value(world, w.mads, args.steps, total_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded PCG64, shapes and value ranges of the workload)",
        "config": dict(w.config, l2="flushed between steps (256 MB write, then a 256 MB read of another buffer)",
                       mads_per_step=w.mads,
                       parallelism="%d independent replicas" % world if world > 1 else "single GPU"),
        "roofline": w.roofline(launch_ms, pk),
        "gpu_launches": w.launches_per_step * args.steps,
        "clocks": clocks,
        "peaks_measured": {k: v for k, v in pk.items()},
        "wall_s": wall,
    }
    if hasattr(w, "e2e"):
        line["e2e"] = w.e2e(args.steps, world)
    else:
        line["e2e"] = None
    if hasattr(w, "accuracy") and _ACC["enabled"]:
        line["accuracy"] = w.accuracy()
    if not args.no_extras and rank == 0 and args.workload == "td_qd":
        line["configs"] = extras(torch, mm, I, pk, flush)
        line["sliced_vs_plain"] = sliced_summary(line["configs"])
    if _ACC["pool"] is not None:
        _ACC["pool"].close()
        _ACC["pool"] = None
    if rank == 0 and world == 1 and not args.no_cpu and args.workload == "td_qd":
        import oracle
        rows = max(oracle.num_cpus(), w.n // 16)
        rate, cores, secs = cpu_sample_rate(w.precs, w.n, rows=rows)
        rate1, _, secs1 = cpu_sample_rate(w.precs, w.n, rows=4, threads=1)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "first %d rows of C for TD and QD at m=n=k=%d "
                                          "(%.1f s on %d threads)" % (rows, w.n, secs, cores),
                                "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                                  "sample": "first 4 rows of C for TD and QD at m=n=k=%d "
                                                            "(%.1f s on 1 thread)" % (w.n, secs1)},
                                "extrapolation": "rates are mads of the sampled rows over their time; "
                                                 "the whole product takes m / rows times as long"}
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def sliced_summary(configs):
    """The slicing form against the plain FP64-EFT kernel on the DD 4096^3
    workload, at the slice count chosen to meet the same bound n 2^-100 that
    the plain product meets, with the binary64-only product's error beside."""
    out = {}
    for name in ("dd_crt", "dd_tc", "dd_crt_int8", "dd_int8"):
        c = configs.get(name)
        if not c:
            continue
        acc = c.get("accuracy", {}).get("dd", {})
        out[name] = {"slices": c["config"]["slices"], "ms": c["ms_per_step"],
                     "fp64_eft_ms": c["roofline"]["fp64_eft_ms"],
                     "speedup_vs_fp64_eft": c["roofline"]["speedup_vs_fp64_eft"],
                     "bound": acc.get("bound"), "err_abs": acc.get("err_abs"),
                     "err_abs_fp64_eft": acc.get("fp64_eft", {}).get("err_abs"),
                     "err_abs_fp64_only": acc.get("fp64_only", {}).get("err_abs"),
                     "both_meet_bound": bool(acc.get("meets_bound") and acc.get("fp64_eft", {}).get("meets_bound"))}
    return out


def extras(torch, mm, I, pk, flush):
    """One short measurement of each other workload (rank 0, after the main one)."""
    out = {}
    for name in ("dd_small", "dd_int8", "dd_tc", "dd_crt", "dd_crt_int8", "td_qd_int8", "td_qd_tc", "td_crt",
                 "qd_crt", "batched", "autograd", "autograd_tc", "autograd_crt", "elementwise", "strassen"):
        w = WORKLOADS[name](torch, mm, I, 0)
        steps = {"dd_small": 10, "elementwise": 10, "strassen": 1}.get(name, 2)
        total_ms, launch_ms, _, _ = measure(torch, w, steps, 1, 1, 0, flush, sample_clocks=False)
        rate_key = "elements_s" if name == "elementwise" else "mad_s"
        out[name] = {"config": w.config, rate_key: w.mads * steps / (total_ms * 1e-3),
                     "ms_per_step": total_ms / steps, "roofline": w.roofline(launch_ms, pk)}
        if hasattr(w, "accuracy") and _ACC["enabled"]:
            out[name]["accuracy"] = w.accuracy()
        del w
        torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------ CPU baseline

def cpu_sample_rate(prec_list, size, rows, cfg=1, threads=None):
    """Oracle (as it stands) on all host cores (or ``threads``): mad/s over the
    first ``rows`` rows of C for each precision, same inputs as the GPU workload."""
    import oracle
    from paper_2101_06584_gb300 import inputs as I
    cores = threads or oracle.num_cpus()
    mads, secs = 0, 0.0
    for prec in prec_list:
        P = I.P_OF[prec]
        A, B = I.cancelling_pair(P, size, size, size, I.rng_for(cfg))
        A = np.ascontiguousarray(A[:, :rows, :])
        t0 = time.perf_counter()
        oracle.gemm(prec, A, B, nthreads=cores)
        secs += time.perf_counter() - t0
        mads += rows * size * size
    return mads / secs, cores, secs


def run_reference(args):
    """The oracle (CPU, as it stands) on a bounded sample of the td_qd workload."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    precs = ("td", "qd")
    n = args.size or 1024
    rows = max(oracle.num_cpus(), n // 64)
    for _ in range(args.warmup):
        cpu_sample_rate(precs, n, rows=1)
    rates, secs_all, cores = [], 0.0, 1
    for _ in range(args.steps):
        r, cores, secs = cpu_sample_rate(precs, n, rows=rows)
        rates.append(r)
        secs_all += secs
    value = statistics.mean(rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded PCG64; ill-scaled TD/QD entries with cancelling inner halves)",
            "config": {"workload": "TD GEMM + QD GEMM, m=n=k=%d, k-sequential (CPU oracle)" % n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "first %d rows of C for TD and QD at m=n=k=%d per step" % (rows, n)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def record_traffic(args):
    """Average DRAM bytes (read + write) per call of the kernels matching
    --kernel-regex in an ncu CSV log, stored with the current source hash."""
    import csv
    import re
    rows = list(csv.reader(open(args.record_traffic)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[hi]
    ki, ii, mi, vi = (hdr.index("Kernel Name"), hdr.index("ID"), hdr.index("Metric Name"),
                      hdr.index("Metric Value"))
    per_launch = {}
    pat = re.compile(args.kernel_regex)
    for r in rows[hi + 1:]:
        if len(r) > vi and pat.search(r[ki]) and r[mi] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            per_launch[r[ii]] = per_launch.get(r[ii], 0.0) + float(r[vi].replace(",", ""))
    if not per_launch:
        raise SystemExit("no matching launches with DRAM byte metrics in %s" % args.record_traffic)
    calls = len(per_launch) / args.per_call
    value = sum(per_launch.values()) / calls
    try:
        rec = json.load(open(TRAFFIC_FILE))
    except (OSError, ValueError):
        rec = {}
    rec[args.traffic_key] = {"bytes_per_launch": value, "launches": len(per_launch),
                             "per_call": args.per_call, "command": args.command,
                             "source_sha256": kernel_source_hash(args.traffic_key)}
    with open(TRAFFIC_FILE, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec[args.traffic_key]))


def main():
    args = parse_args()
    if args.record_traffic:
        record_traffic(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
