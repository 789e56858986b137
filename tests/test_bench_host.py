"""Host logic of bench.py that needs no GPU: the algorithmic units behind its roofline fields
and the arithmetic that turns event times into achieved rates and fractions of the peak."""
from __future__ import annotations

import pytest

import bench

M, N = 16384, 2048


def test_paired_iteration_bytes_at_the_dense_workload():
    # A_u in FP32 once, the triangle of R_H in FP16 for each of the two triangular products,
    # about 24 FP32 n-vectors: 142.8 MB at 16384 x 2048
    assert bench.paired_iteration_bytes(M, N) == 4 * M * N + 2 * N * (N + 1) + 24 * 4 * N
    assert bench.paired_iteration_bytes(M, N) == 142_807_040


def test_inner_loop_rate_from_event_time_and_iterations():
    peaks = {"hbm_gbs": 6800.0}
    prof = {"pcg_solve2": (30, 5.7811)}              # launches, device ms
    units = {"pcg_solve2": 135}                      # paired iterations in those launches
    r = bench._inner_loop(prof, units, peaks, M, N)
    per_s = 5.7811e-3 / 135
    assert r["us_per_iteration"] == pytest.approx(per_s * 1e6, rel=1e-12)
    assert r["achieved"] == pytest.approx(142_807_040 / per_s / 1e9, rel=1e-12)
    assert r["frac"] == pytest.approx(r["achieved"] / 6800.0, rel=1e-12)
    assert r["peak_source"] == "measured" and r["bound"] == "hbm"
    # ncu traffic belongs to the size it was captured at only
    assert r["traffic"] == bench.PCG_FUSED_TRAFFIC_PER_ITER_C2
    assert bench._inner_loop(prof, units, peaks, 8192, N)["traffic"] is None
    # no launches timed: no roofline
    assert bench._inner_loop({}, {}, peaks, M, N) == {}


def test_residual_and_gram_units():
    peaks = {"hbm_gbs": 6800.0, "bf16_tflops_sustained": 1700.0}
    avg_ms = 0.078
    r = bench._roofline({"resid_pass": (9, 9 * avg_ms)}, peaks, "resid_pass", M, N, variant64=4)
    # the pair A32 + Alo read once (8 B per entry of A), x and b in, per-SM FP64 partials out
    byts = 8 * M * N + 8 * M + 8 * N + 152 * 8 * N
    assert r["algorithmic_bytes"] == byts
    assert r["achieved"] == pytest.approx(byts / (avg_ms * 1e-3) / 1e9, rel=1e-12)
    assert r["frac"] == pytest.approx(r["achieved"] / 6800.0, rel=1e-12)
    # the FP64 pass is bounded by the FP64 FMA rate: 4 flops per entry of A
    r = bench._roofline({"resid_pass": (1, 0.152)}, peaks, "resid_pass", M, N, variant64=3)
    assert r["bound"] == "alu" and r["algorithmic_flops"] == 4.0 * M * N
    assert r["frac"] == pytest.approx(4.0 * M * N / 0.152e-3 / 1e12 / bench.FP64_PEAK)
    # the Gram: n(n+1)/2 entries of 2m flops each, against the sustained bf16 peak
    r = bench._roofline({"gram": (1, 0.08)}, peaks, "gram", M, N)
    assert r["algorithmic_flops"] == M * N * (N + 1)
    assert r["frac"] == pytest.approx(M * N * (N + 1) / 0.08e-3 / 1e12 / 1700.0)


def test_fallback_peaks_are_named_as_such():
    r = bench._roofline({"gram": (1, 0.08)}, {}, "gram", M, N)
    assert r["peak"] == 1700.0 and r["peak_source"].startswith("fallback")


def test_batch_residual_roofline_follows_the_working_precision():
    peaks = {"hbm_gbs": 6800.0}
    prof = {"resid_pass": (10, 20.0, 10 * 2.2e8)}    # launches, device ms, entries of A
    r = bench._batch_roofline(prof, peaks, "resid_pass")
    assert r["bound"] == "hbm" and "double-FP32" in r["kernel"]
    assert r["achieved"] == pytest.approx(8.0 * 2.2e9 / 20e-3 / 1e9, rel=1e-12)
    assert r["frac"] == pytest.approx(r["achieved"] / 6800.0, rel=1e-12)
    r = bench._batch_roofline(prof, peaks, "resid_pass", u64=True)
    assert r["bound"] == "alu" and r["peak"] == bench.FP64_PEAK
    assert r["achieved"] == pytest.approx(4.0 * 2.2e9 / 20e-3 / 1e12, rel=1e-12)


def _run_bench(args, env_extra=None):
    import json
    import os
    import subprocess
    import sys
    env = dict(os.environ)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(os.path.dirname(bench.__file__), "bench.py"),
                        *args], capture_output=True, text=True, timeout=300, env=env)
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    return r.returncode, [json.loads(ln) for ln in lines], r.stderr


def test_reference_arm_prints_the_contract_line():
    """`--impl reference` times the FP64 oracle on the host cores (here on a small case) and
    prints one JSON line with the keys the benchmark contract names."""
    rc, lines, err = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "1",
                                 "--m", "600", "--n", "60"])
    assert rc == 0, err
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "solves/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "dense_600x60_uf16_u32_ur64"


def test_reference_arm_runs_on_rank_zero_only():
    rc, lines, err = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "1",
                                 "--m", "600", "--n", "60"],
                                {"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"})
    assert rc == 0, err
    assert lines == []
