"""Host arithmetic of the benchmark's measurement (no GPU): the algorithmic work the
rooflines divide by, the scan's latency model, the whole-job rate, and the committed DRAM
traffic record of the scan (it must belong to the committed scan source, else the bench
line reports no traffic)."""
import itertools
import json
import os
import shutil
import types

import bench


def brute_pairs(N):
    """Mode pairs (k, m) of the direct Fourier-Galerkin sum in 3-D: |k_i|, |m_i| and
    |k_i - m_i| at most h = N/2 - 1 in every dimension, counted one by one."""
    h = N // 2 - 1
    one = sum(1 for k, m in itertools.product(range(-h, h + 1), repeat=2) if abs(k - m) <= h)
    return one ** 3


def test_pairs_per_cell_counts_the_sum_terms():
    for N in (4, 6, 8, 16, 32):
        assert bench.pairs_per_cell(N) == brute_pairs(N), N


def test_sum_roofline_is_work_over_time_against_the_measured_peak():
    wl = types.SimpleNamespace(N=32, J=64)
    peaks = {"fp32_ffma_tflops": 77.0, "fp64_dfma_tflops": 1.05, "sms": 152}
    prof = {"sum": (3.0, 2, 64), "sum_fp64": (600.0, 1, 64), "sum_df64": (26.0, 1, 64)}
    r = bench.roofline("sum", prof, wl, 2070.0, peaks)
    flops = 10 * 0.5 * brute_pairs(32) * 64
    assert abs(r["achieved"] - flops / 3e-3 / 1e12) < 1e-9 * r["achieved"]
    assert r["bound"] == "alu" and r["peak"] == 77.0 and abs(r["frac"] - r["achieved"] / 77.0) < 1e-12
    r64 = bench.roofline("sum_fp64", prof, wl, 2070.0, peaks)
    assert r64["peak"] == 1.05
    rdf = bench.roofline("sum_df64", prof, wl, 2070.0, peaks)
    assert abs(rdf["achieved"] - 56 * 0.5 * brute_pairs(32) * 64 / 26e-3 / 1e12) < 1e-9 * rdf["achieved"]
    assert rdf["peak"] == 38.5  # one FP32-pipe operation per lane per clock: half the FFMA flop rate


def test_scan_latency_model_adds_up():
    stats = {"visits": 100, "inner_iters": 700, "newton_iters": 2500, "newton_solves": 1500}
    peaks = {"scan_cluster_reduce_us": 2.0, "scan_newton_iteration_us": 1.5}
    m = bench.scan_latency_model(160.0, stats, peaks)
    assert m["inner_updates_per_visit"] == 7.0
    assert m["cluster_reductions_per_visit"] == 9.0  # two per visit, then one per inner update
    assert m["newton_evaluations_per_visit"] == 40.0
    assert m["us_cluster_reductions"] == 18.0 and m["us_newton"] == 60.0
    assert m["modelled_fraction"] == round(78.0 / 160.0, 3)


def test_whole_job_rate_aggregates_the_ranks():
    assert bench.whole_job_rate(128 * 20, 1, 650.0) == 128 * 20 / 0.65
    assert bench.whole_job_rate(128 * 20, 4, 650.0) == 4 * 128 * 20 / 0.65


def test_scan_traffic_record_belongs_to_the_committed_scan(tmp_path, monkeypatch):
    per_visit = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))["k_sweep<dfloat,8>"]
    t = bench.kernel_traffic("k_sweep<dfloat,8>", 32)
    assert t == per_visit["dram_bytes_per_unit"] * 32, "profiles/traffic.json is stale: re-capture the scan's traffic"
    # a record whose sources hash differs from the sources is not used
    root = tmp_path / "repo"
    for src in per_visit["sources"]:
        (root / os.path.dirname(src)).mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, src), root / src)
    (root / "profiles").mkdir()
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    rec["k_sweep<dfloat,8>"]["sources_sha256"] = "0" * 64
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.kernel_traffic("k_sweep<dfloat,8>", 32) is None
