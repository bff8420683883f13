"""Host-side logic of the benchmark on CPU: DRAM traffic recorded from an ncu
CSV is stored with a hash of the kernel's sources and reported only while
those sources are unchanged; the committed records are well formed; the
per-kernel byte sums and per-call averages of a capture."""
import csv
import json
import os

import pytest

import bench


def test_committed_records_are_well_formed():
    """Each record names its capture command (with ncu's clocks left alone),
    its launches and a source hash; while the hash matches the sources the
    record is what the benchmark reports (a stale one is reported as null)."""
    with open(bench.TRAFFIC_FILE) as f:
        rec = json.load(f)
    assert rec
    for key, ent in rec.items():
        assert key.split("_")[0] + "_" + key.split("_")[1] in bench.TRAFFIC_SOURCES, key
        assert ent["bytes_per_launch"] > 0 and ent["launches"] >= ent["per_call"] >= 1, key
        assert ent["command"].startswith("ncu ") and "--clock-control none" in ent["command"], key
        assert len(ent["source_sha256"]) == 64 and int(ent["source_sha256"], 16) >= 0, key
        fresh = ent["source_sha256"] == bench.kernel_source_hash(key)
        assert bench.recorded_traffic(key) == (ent["bytes_per_launch"] if fresh else None), key


def _fake_csv(path, launches):
    """An ncu --csv log: per launch (id, kernel, read, write) three metric rows."""
    with open(path, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(["==PROF== a line before the table"])
        w.writerow(["ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value"])
        for i, name, rd, wr in launches:
            w.writerow([i, name, "dram__bytes_read.sum", "byte", "{:,}".format(rd)])
            w.writerow([i, name, "dram__bytes_write.sum", "byte", "{:,}".format(wr)])
            w.writerow([i, name, "gpu__time_duration.sum", "ns", "1000"])


def test_record_and_stale_hash(tmp_path, monkeypatch):
    traffic = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(traffic))
    log = tmp_path / "log.csv"
    # two calls of two kernels each; only the matching kernels count
    _fake_csv(log, [(0, "ozaki_slice(x)", 100, 50), (1, "ozaki_tc_pair_kernel<2>(y)", 1000, 10),
                    (2, "other_kernel(z)", 7, 7),
                    (3, "ozaki_slice(x)", 120, 30), (4, "ozaki_tc_pair_kernel<2>(y)", 1100, 20)])

    class Args:
        record_traffic = str(log)
        kernel_regex = "ozaki_"
        per_call = 2
        traffic_key = "dd_tc_4096_s13:call"
        command = "ncu ..."

    bench.record_traffic(Args)
    ent = json.load(open(traffic))["dd_tc_4096_s13:call"]
    # (150 + 1010 + 150 + 1120) bytes over 4 launches / 2 per call = 2 calls
    assert ent["bytes_per_launch"] == pytest.approx((150 + 1010 + 150 + 1120) / 2)
    assert ent["launches"] == 4 and ent["per_call"] == 2
    assert bench.recorded_traffic("dd_tc_4096_s13:call") == ent["bytes_per_launch"]
    # a record taken from other sources is not reported
    ent["source_sha256"] = "0" * 64
    json.dump({"dd_tc_4096_s13:call": ent}, open(traffic, "w"))
    assert bench.recorded_traffic("dd_tc_4096_s13:call") is None
    assert bench.recorded_traffic("td_qd_1024:qd") is None          # no record at all


def test_source_hash_follows_the_sources(tmp_path, monkeypatch):
    """The hash covers every listed source: changing one byte of one changes it."""
    src = os.path.join(bench.ROOT, "paper_2101_06584_gb300", "csrc")
    fake = tmp_path / "paper_2101_06584_gb300" / "csrc"
    fake.mkdir(parents=True)
    for name in bench.TRAFFIC_SOURCES["td_qd"]:
        (fake / name).write_bytes(open(os.path.join(src, name), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash("td_qd_1024:qd")
    for name in bench.TRAFFIC_SOURCES["td_qd"]:
        p = fake / name
        data = p.read_bytes()
        p.write_bytes(data + b" ")
        assert bench.kernel_source_hash("td_qd_1024:qd") != h0, name
        p.write_bytes(data)
    assert bench.kernel_source_hash("td_qd_1024:qd") == h0


@pytest.mark.parametrize("prec", ["dd", "td", "qd"])
def test_bench_errors_match_exact_arithmetic(prec):
    """The benchmark's error figures (exact products split into binary64 and
    peeled by math.fsum) agree with the oracle's rational arithmetic on the
    same entries, for the oracle's product, a perturbed copy of it and the
    leading plane alone (the FP64-only figure), on ordinary and cancelling
    inputs; whole rows and scattered entries both take their paths."""
    import numpy as np
    import oracle
    from oracle import exact as X
    from paper_2101_06584_gb300 import inputs as I
    P = I.P_OF[prec]
    rng = np.random.default_rng(700 + P)
    m, n, k = 70, 90, 37
    for A, B in ((I.uniform(P, (m, k), rng), I.uniform(P, (k, n), rng)),
                 I.cancelling_pair(P, m, n, k, rng)):
        ent = bench.sample_entries(m, n, 40, np.random.default_rng(5), full_rows=1)
        ref = bench.ExactReference(A, B, ent)
        C = oracle.gemm(prec, A, B, nthreads=2)
        bumped = C.copy()
        bumped[-1] *= 1.0 + 2.0 ** -20
        for cand in (C, bumped, C[:1], oracle.dgemm(A[0], B[0])):
            got = ref.errors(cand)
            want = X.gemm_error(cand if cand.ndim == 3 else cand[None], A, B, ent)
            for key in ("err_abs", "err_rel", "max_abs"):
                assert got[key] == pytest.approx(want[key], rel=1e-9, abs=1e-300), (key, got, want)


def test_bench_exact_products_refuse_extreme_ranges():
    """Products outside the range where the split products are exact raise."""
    import numpy as np
    A = np.full((1, 2, 3), 2.0 ** -500)
    B = np.full((1, 3, 2), 2.0 ** -500)
    with pytest.raises(ValueError):
        bench.ExactReference(A, B, [(0, 0)])


def test_eft_mix_adds_up_to_the_operation_counts():
    """(TwoSum, FastTwoSum, TwoProd, other) per multiply-add, weighted 6, 3, 2
    and 1 binary64 operations, give the implemented sequences' counts."""
    for prec, (ts, qts, tp, other) in bench.EFT_MIX.items():
        assert 6 * ts + 3 * qts + 2 * tp + other == bench.FP64_OPS_PER_MAD[prec]


def test_kseq_bound_and_roofline():
    """The bound of a tile is the larger of its FP64-pipe time and its
    integer-pipe time; with no transformation moved it is the DFMA time, and
    the roofline's peak is the algorithm's operations at that bound."""
    pk = {"dfma": 6.0e11, "int_two_sum": 1.5e11, "int_fast_two_sum": 1.8e11, "int_two_prod": 2.4e11}
    s, f64 = bench.kseq_bound("qd", 0, pk)
    assert f64 == 210 and s == pytest.approx(210 / 6.0e11)
    s, f64 = bench.kseq_bound("qd", 1, pk)                  # 22 TwoSums moved
    assert f64 == 78 and s == pytest.approx(max(78 / 6.0e11, 22 / 1.5e11))
    s, f64 = bench.kseq_bound("dd", 3, pk)                  # TwoSum + 2 FastTwoSums moved
    assert f64 == 8 and s == pytest.approx(max(8 / 6.0e11, 1 / 1.5e11 + 2 / 1.8e11))
    s, f64 = bench.kseq_bound("td", 7, pk)
    assert f64 == 8 and s == pytest.approx(14 / 1.5e11 + 10 / 1.8e11 + 3 / 2.4e11)
    r = bench.kseq_roofline("qd", 10 ** 9, 200.0, pk, {"int_ops": 1})
    ach = 10 ** 9 * 210 / 0.2
    assert r["achieved"] == pytest.approx(ach / 1e12)
    assert r["peak"] == pytest.approx(210 / (22 / 1.5e11) / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["frac_of_fp64_pipe_alone"] == pytest.approx(ach / 6.0e11)
    assert r["int_ops"] == 1 and r["fp64_pipe_ops_per_unit"] == 78
