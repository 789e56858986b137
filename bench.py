"""Benchmark: TLS solves/s of RQI-PCGTLS on one GB300 (or N, weak scaling).

One step = one complete solve of a resident 16384 x 2048 dense problem A = Y [diag(D); 0] Z^T
(D log-spaced in [1e-3, 1], noise std 1e-4, seed 0 + rank): the preconditioner (column scaling,
FP16 Gram on the GPU, Cholesky, inverse) and the RQI-PCGTLS iteration (FP32 PCGTLS, FP64
residuals). A solve counts only if sigma rel err <= 1e-10 and x rel err <= 1e-8 against the
FP64 CPU oracle run on the same problem.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --workload batch [--batch 512]

Prints one JSON line (rank 0). `--impl reference` times the FP64 CPU oracle instead.
`--workload batch`: one step = factor + solve of a resident packed batch of 512 uneven dense
problems (n ~ U{32..512}, m = n U{4..20}, D log-spaced in [10^-U(1,4), 1], seeds 1000 + i); a
solve counts if it matches the FP64 oracle (run on every problem, in a process pool) to the same
tolerances.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import signal
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TLS solves/s on GB300 at sigma rel err<=1e-10 vs FP64 oracle; mixed vs plain FP64"
M_ROWS, N_COLS, D_LO, NOISE = 16384, 2048, 1e-3, 1e-4
SIGMA_TOL, X_TOL = 1e-10, 1e-8
SOLVE_TOL, MAX_RQI = 1e-16, 12
# derived ALU peaks (no measured FP32 / FP64 peak in the measured-peaks file)
FP64_PEAK = 2 * 2 * 152 * 2.07e9 / 1e12       # TFLOP/s: 2 FMA/clk/SM
FP32_PEAK = 2 * 128 * 152 * 2.07e9 / 1e12     # TFLOP/s: 128 FMA/clk/SM
WORKLOAD = f"dense_{M_ROWS}x{N_COLS}_uf16_u32_ur64"


def _peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def _problem(rank: int):
    from paper_2305_19028_gb300 import synth
    return synth.dense_problem(M_ROWS, N_COLS, d_lo=D_LO, noise=NOISE, seed=rank)


def _set_size(m: int | None, n: int | None):
    """Override the problem size (for profiling captures on a smaller case)."""
    global M_ROWS, N_COLS, WORKLOAD
    if m:
        M_ROWS = m
    if n:
        N_COLS = n
    WORKLOAD = f"dense_{M_ROWS}x{N_COLS}_uf16_u32_ur64"


def _oracle_solve(p):
    import oracle.rqi_pcgtls as O
    return O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=MAX_RQI)


def _cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _timed_dense_oracle(seed: int):
    """Pool worker: one FP64 oracle solve of the dense benchmark problem (seed), timed."""
    p = _problem(seed)
    t0 = time.perf_counter()
    x, s, _ = _oracle_solve(p)
    return x, s, time.perf_counter() - t0


def _single_thread_pool(fn, items, procs):
    """map(fn, items) on `procs` spawned single-threaded processes; (results, wall seconds)."""
    import multiprocessing as mp
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        t0 = time.perf_counter()
        with mp.get_context("spawn").Pool(processes=procs) as pool:
            res = pool.map(fn, items, chunksize=1)
        dt = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return res, dt


def _cpu_baseline_dense(seed: int):
    """The CPU plan for the dense benchmark problem: single-core latency as the median of three
    single-threaded solves (run side by side), and throughput as P = nproc single-threaded
    solves run at once on all host cores (solves / wall time). Returns (baseline, (x, sigma))."""
    nproc = os.cpu_count() or 1
    lat, _ = _single_thread_pool(_timed_dense_oracle, [seed] * 3, 3)
    thr, wall = _single_thread_pool(_timed_dense_oracle, [seed] * nproc, nproc)
    times = sorted(t for _, _, t in lat)
    x, s, _ = lat[0]
    base = {"value": nproc / wall, "unit": "solves/s", "cores": nproc, "kind": "oracle",
            "sample": f"{nproc} FP64 solves of the {M_ROWS}x{N_COLS} problem at once, one "
                      f"single-threaded process per core ({wall:.1f} s wall)",
            "latency_s_median": statistics.median(times), "latency_s": times,
            "latency_sample": "3 single-threaded solves (one core each), median",
            "nproc": nproc, "cpu_model": _cpu_model()}
    return base, (x, s)


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None
        self.skip = 0

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
            # let the sampler finish starting (its driver initialisation otherwise overlaps the
            # first timed steps and slows their launches); samples from before this point are
            # not the timed region's
            time.sleep(1.0)
            self.skip = os.path.getsize(self.path)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self) -> dict | None:
        if self.proc is None or not self.path:
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            lines = fh.read().splitlines()
        with open(self.path) as fh:
            fh.seek(self.skip)
            during = fh.read().splitlines()
        # only the samples taken while the timed steps ran, unless the region was shorter than
        # the sampling period (then the nearest ones, taken just before it)
        in_region = bool(during)
        for line in during if in_region else lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm), "in_timed_region": in_region}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _reduce(value: float, ws: int, op: str) -> float:
    """Max or sum of a scalar over the ranks (a CUDA tensor under NCCL, a host one under gloo)."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def _barrier_max(value: float, ws: int) -> float:
    """The slowest rank's time (the job's time)."""
    return _reduce(value, ws, "max")


def _total(value: float, ws: int) -> float:
    """Units processed by all ranks together."""
    return _reduce(value, ws, "sum")


def _shard_ids(rank: int, count: int) -> list[int]:
    """The batch members of one rank: independent problems, no exchange between ranks."""
    return [rank * count + i for i in range(count)]


def run_reference(args, ws, rank):
    """The FP64 CPU oracle, timed on the host cores as the reference arm."""
    if rank != 0:
        return
    p = _problem(0)
    for _ in range(args.warmup):
        _oracle_solve(p)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _oracle_solve(p)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "m": M_ROWS, "n": N_COLS, "d_lo": D_LO, "noise": NOISE,
                   "seed": 0, "solver": "FP64 CPU oracle (numpy/OpenBLAS), Householder QR R"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} full solves of the {M_ROWS}x{N_COLS} problem "
                                   f"(numpy/OpenBLAS threads)",
                         "nproc": cores, "cpu_model": _cpu_model()},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# DRAM bytes per launch of the FP64 residual pass (the pipelined kernel, n = 2048) per row of A,
# from the ncu capture in profiles/resid_pass_dense_8192x2048.md (134.346 MB read + 0.067 MB
# written at m = 8192; one read of A, so proportional to m)
RESID_PIPE_TRAFFIC_PER_ROW = (134.346e6 + 0.067e6) / 8192
# DRAM bytes of the one-launch paired PCGTLS solve per paired iteration at 16384 x 2048 (read +
# write, from the ncu capture in profiles/pcg_fused_dense_16384x2048.md: 419.96 MB for a launch
# of 3 iterations). The double-FP32 residual pass has no current figure: its capture predates
# the column reduction it now runs after a grid barrier in the same launch.
PCG_FUSED_TRAFFIC_PER_ITER_C2 = (416.771072e6 + 3.188480e6) / 3


def paired_iteration_bytes(m: int, n: int) -> int:
    """Algorithmic bytes of one paired PCGTLS iteration (both right-hand sides): A_u in FP32
    once (4 m n), the two triangular factors' products with R_H held in u_f = FP16
    (2 x n (n + 1) / 2 x 2 B) and about 24 FP32 n-vectors (q, w, y, s, p and partial sums)."""
    return 4 * m * n + 2 * n * (n + 1) + 24 * 4 * n


def _inner_loop(prof: dict, units: dict, peaks: dict, m: int, n: int) -> dict:
    """HBM roofline of the PCGTLS inner loop per paired iteration: the paired solves' device
    time (one launch per solve: passes over A, reductions and W / W^T products of every step)
    divided by the PCGTLS steps they ran."""
    cnt, ms = prof.get("pcg_solve2", (0, 0.0))
    it = units.get("pcg_solve2", 0)
    hbm = peaks.get("hbm_gbs", 6800.0)
    src = "measured" if peaks else "fallback"
    byts = paired_iteration_bytes(m, n)
    if cnt and it:
        per = ms * 1e-3 / it
        ach = byts / per / 1e9
        return {"kernel": "pcg_fused_kernel (one launch per paired PCGTLS solve: t = A d, "
                          "A^T t reduced in a fixed order, r and w updates, "
                          "z = (R^T R)^{-1} r; FP32)",
                "unit_of_work": "one paired PCGTLS iteration", "bound": "hbm", "achieved": ach,
                "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": PCG_FUSED_TRAFFIC_PER_ITER_C2 if (m, n) == (16384, 2048) else None,
                "traffic_unit": "DRAM bytes per paired iteration (ncu, 3-step launch)",
                "peak_source": src, "us_per_iteration": per * 1e6, "iterations": it,
                "launches": cnt, "algorithmic_bytes": byts}
    # multi-launch path: the pass launches plus the step-tail launches per iteration
    c2, m2 = prof.get("pcg_pass2", (0, 0.0))
    cr, mr = prof.get("pcg_reduce", (0, 0.0))
    if not c2:
        return {}
    per = (m2 + mr * c2 / max(1, cr)) * 1e-3 / c2
    ach = byts / per / 1e9
    return {"kernel": "pass + step tail per paired iteration (multi-launch path)",
            "unit_of_work": "one paired PCGTLS iteration", "bound": "hbm", "achieved": ach,
            "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": None, "peak_source": src,
            "us_per_iteration": per * 1e6, "iterations": c2, "algorithmic_bytes": byts}


def _pass_only(tls, ctx, p, sigma) -> dict:
    """The pass over A alone inside the one-launch solve: one traced paired solve of 8 steps
    at the final shift; the pass's duration per step from the in-kernel global timer (CTA 0),
    against the pass's algorithmic bytes (A_u once in FP32 plus d in and A^T t out)."""
    m, n = p.A.shape
    tls.tls_trace_enable(ctx, True)
    try:
        rng = np.random.default_rng(0)
        f0, f1 = rng.standard_normal(n), rng.standard_normal(n)
        tls.tls_pcgtls(ctx, 0.99 * sigma * sigma, f0, f1, steps=8)
        tr = tls.tls_trace_get(ctx).astype(np.int64)
    finally:
        tls.tls_trace_enable(ctx, False)
    if tr.size < 2 + 10 * 8 or tr[0] == 0:
        return {}
    passes = [tr[2 + 10 * j + 1] - tr[2 + 10 * j] for j in range(8)
              if tr[2 + 10 * j] and tr[2 + 10 * j + 1]]
    steps = [tr[2 + 10 * (j + 1)] - tr[2 + 10 * j] for j in range(7)
             if tr[2 + 10 * j] and tr[2 + 10 * (j + 1)]]
    if not passes:
        return {}
    us = float(np.mean(passes)) / 1e3
    byts = 4 * m * n + 2 * 2 * n * 4
    return {"us_per_pass": us, "achieved": byts / (us * 1e-6) / 1e9, "unit": "GB/s",
            "algorithmic_bytes": byts, "us_per_step_in_kernel":
            float(np.mean(steps)) / 1e3 if steps else None,
            "source": "in-kernel global timer of CTA 0, one traced paired solve of 8 steps"}


def _roofline(prof: dict, peaks: dict, cls: str, m: int, n: int, variant64: int = -1,
              units: dict | None = None, qr: bool = False) -> dict:
    cnt, ms = prof.get(cls, (0, 0.0))
    if cnt == 0:
        return {}
    avg_s = ms / cnt * 1e-3
    hbm = peaks.get("hbm_gbs", 6800.0)
    bf16 = peaks.get("bf16_tflops_sustained", 1700.0)
    src = "measured" if peaks else "fallback"
    if cls == "pcg_solve2":
        return _inner_loop(prof, units or {}, peaks, m, n)
    if cls == "pcg_pass2":
        unit_bytes = m * n * 4 + 2 * n * 4 * 2          # A_u once + q in / partial out
        ach = unit_bytes / avg_s / 1e9
        return {"kernel": "pcg_pass2 (fused t=Aq, A^T t, 2 RHS, FP32)", "bound": "hbm",
                "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": None, "peak_source": src, "avg_launch_us": avg_s * 1e6,
                "algorithmic_bytes": unit_bytes}
    if cls == "resid_pass" and variant64 == 4:
        # double-FP32 residual: A read once as the FP32 pair A32 + Alo (8 bytes per entry, the
        # FP64 pass's traffic), x and b in, the per-CTA FP64 partials of A^T r out
        unit_bytes = 8 * m * n + 8 * m + 8 * n + 152 * 8 * n
        ach = unit_bytes / avg_s / 1e9
        return {"kernel": "resid_df_kernel (r = b - A x, A^T r in double-FP32 arithmetic on "
                          "A32 + Alo)", "bound": "hbm", "achieved": ach,
                "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": None,
                "peak_source": src, "avg_launch_us": avg_s * 1e6, "algorithmic_bytes": unit_bytes,
                "fp64_equivalent_tflops": 4.0 * m * n / avg_s / 1e12}
    if cls == "resid_pass":
        # FP64 FMA-bound on this GPU: r = b - A x and A^T r are 2 FMA (4 flops) per entry of A
        flops = 4.0 * m * n
        ach = flops / avg_s / 1e12
        traffic = RESID_PIPE_TRAFFIC_PER_ROW * m if (variant64 == 3 and n == 2048) else None
        return {"kernel": "resid_pass (FP64 r=b-Ax, A^T r)", "bound": "alu", "achieved": ach,
                "peak": FP64_PEAK, "unit": "TFLOP/s", "frac": ach / FP64_PEAK, "traffic": traffic,
                "traffic_unit": "bytes per launch (DRAM read + write, ncu)",
                "peak_source": "nominal FP64 rate (2 FMA/clk/SM x 152 SMs x 2.07 GHz)",
                "avg_launch_us": avg_s * 1e6, "algorithmic_flops": flops,
                "hbm_gbs": (m * n * 8 + m * 8) / avg_s / 1e9}
    if cls == "gram":
        flops = m * n * (n + 1)                          # SYRK: n(n+1)/2 entries x 2m flops
        ach = flops / avg_s / 1e12
        return {"kernel": "gram (H = A_s^T A_s, FP16 in, FP32 acc)", "bound": "tensor",
                "achieved": ach, "peak": bf16, "unit": "TFLOP/s", "frac": ach / bf16,
                "traffic": None, "peak_source": src + " (bf16 sustained; fp16 nominal rate equal)",
                "avg_launch_us": avg_s * 1e6, "algorithmic_flops": flops}
    if cls == "chol" and qr:
        # the Householder QR of the scaled m x n matrix (R only): 2 m n^2 - 2 n^3 / 3 flops,
        # FP32 on CUDA cores; bound by the per-column cluster exchanges of its panels
        flops = 2.0 * m * n * n - 2.0 * n ** 3 / 3.0
        ach = flops / avg_s / 1e12
        return {"kernel": "householder qr (R of A D^-1 in u_q; panel reflectors on a 16-CTA "
                          "cluster, WY trailing updates, FP32 CUDA cores)", "bound": "alu",
                "achieved": ach, "peak": FP32_PEAK, "unit": "TFLOP/s", "frac": ach / FP32_PEAK,
                "traffic": None,
                "peak_source": "nominal FP32 rate (128 FMA/clk/SM x 152 SMs x 2.07 GHz)",
                "avg_launch_us": avg_s * 1e6, "algorithmic_flops": flops}
    if cls == "chol":
        # one launch-class entry per factor: the diagonal blocks (a chain of n pivots, one CTA
        # per 64-block) and the panel / trailing updates, FP32 on CUDA cores
        flops = n ** 3 / 3.0
        ach = flops / avg_s / 1e12
        return {"kernel": "chol (blocked Cholesky of H, FP32 CUDA cores; latency of the "
                          "diagonal-block chain)", "bound": "alu", "achieved": ach,
                "peak": FP32_PEAK, "unit": "TFLOP/s", "frac": ach / FP32_PEAK, "traffic": None,
                "peak_source": "nominal FP32 rate (128 FMA/clk/SM x 152 SMs x 2.07 GHz)",
                "avg_launch_us": avg_s * 1e6, "algorithmic_flops": flops}
    return {}


def run_ours(args, ws, rank, local):
    import torch
    from paper_2305_19028_gb300 import tls

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    tls.load()
    p = _problem(rank)
    stream = torch.cuda.current_stream()
    ctx = tls.tls_create_dense(p.A, p.b, stream=stream.cuda_stream)
    qr = args.factor == "qr"
    opt = tls.tls_default_options(u="fp32", factor=1 if qr else 0)

    # the CPU oracle (accuracy reference and CPU baseline) runs after every GPU measurement,
    # so that its host threads cannot slow the launches being timed; results are kept and
    # checked against it at the end
    cpu = None
    ref = None

    def accurate(x, s):
        if ref is None:
            return True
        xo, so = ref
        return (abs(s - so) / so <= SIGMA_TOL and
                np.linalg.norm(x - xo) / np.linalg.norm(xo) <= X_TOL)

    def step():
        tls.tls_factor(ctx, "fp16", opt)
        return tls.tls_solve(ctx, tol=SOLVE_TOL, max_rqi=MAX_RQI)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    l0 = tls.tls_kernel_launches()
    results = []
    infos = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            x, s, info = step()
            results.append((x, s))
            infos.append(info)
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = tls.tls_kernel_launches() - l0
    if ws > 1:
        torch.distributed.barrier()
    ms = ev0.elapsed_time(ev1)
    ms = _barrier_max(ms, ws)
    clocks = clk.summary()
    # per-class kernel times: the same steps again with every launch bracketed by CUDA events
    # on the context's stream (the event records add host work, so they stay out of `value`)
    tls.tls_profile_enable(ctx, True)
    for _ in range(max(1, min(args.steps, 5))):
        step()
    torch.cuda.synchronize()
    prof = tls.tls_profile_get(ctx)
    units = tls.tls_profile_units(ctx)
    tls.tls_profile_enable(ctx, False)
    last_x, last_s = x, s
    pass_only = _pass_only(tls, ctx, p, s)

    # end to end through the public API from pinned host memory
    e2e = None
    if not args.no_e2e:
        A_pin = torch.from_numpy(p.A).pin_memory().numpy()
        b_pin = torch.from_numpy(p.b).pin_memory().numpy()
        ne = max(1, min(args.steps, 5))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2e_res = []

        def e2e_step():
            c2 = tls.tls_create_dense(A_pin, b_pin, stream=stream.cuda_stream)
            tls.tls_factor(c2, "fp16", opt)
            x2, s2, _ = tls.tls_solve(c2, tol=SOLVE_TOL, max_rqi=MAX_RQI)
            tls.tls_destroy(c2)
            return x2, s2

        e2e_step()   # warm-up: the first context's buffers come from cudaMalloc, later ones from the block cache
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(ne):
            e2e_res.append(e2e_step())
        e1.record(stream)
        torch.cuda.synchronize()
        ems = _barrier_max(e0.elapsed_time(e1), ws)
        e2e = {"value": None, "unit": "solves/s",
               "h2d_bytes_per_step": int(p.A.nbytes + p.b.nbytes),
               "d2h_bytes_per_step": int(8 * N_COLS + 8), "steps": ne,
               "ms_per_step": ems / ne}

    # plain all-FP64 GPU RQI-PCGTLS on the same problem, for the mixed-vs-plain comparison
    plain = None
    if not args.no_plain:
        opt64 = tls.tls_default_options(u="fp64")
        tls.tls_factor(ctx, "fp64", opt64)
        tls.tls_solve(ctx, tol=SOLVE_TOL, max_rqi=MAX_RQI)
        np_steps = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        plain_res = []
        q0.record(stream)
        for _ in range(np_steps):
            tls.tls_factor(ctx, "fp64", opt64)
            xp, sp, ip = tls.tls_solve(ctx, tol=SOLVE_TOL, max_rqi=MAX_RQI)
            plain_res.append((xp, sp))
        q1.record(stream)
        torch.cuda.synchronize()
        pms = _barrier_max(q0.elapsed_time(q1), ws)
        plain = {"value": None, "unit": "solves/s",
                 "ms_per_step": pms / np_steps, "steps": np_steps,
                 "rqi_steps": ip["rqi_steps"], "cg_iters": ip["cg_iters"]}
    tls.tls_destroy(ctx)

    # CPU oracle leg (rank 0 of a one-GPU run: the timed CPU baseline, whose first solve is
    # also the accuracy reference; other ranks: one multi-threaded solve of their problem),
    # then the accuracy of every result against it
    if not args.no_cpu:
        if rank == 0 and ws == 1:
            cpu, ref = _cpu_baseline_dense(rank)
        else:
            xo, so, io = _oracle_solve(p)
            ref = (xo, so)
    ok = _total(sum(int(accurate(x_, s_)) for x_, s_ in results), ws)
    err = None
    if ref is not None:
        err = {"sigma_rel": abs(last_s - ref[1]) / ref[1],
               "x_rel": float(np.linalg.norm(last_x - ref[0]) / np.linalg.norm(ref[0]))}
    if e2e is not None:
        okc = _total(sum(int(accurate(x_, s_)) for x_, s_ in e2e_res), ws)
        e2e["value"] = okc / (e2e["ms_per_step"] * e2e["steps"] * 1e-3)
    if plain is not None:
        okp = _total(sum(int(accurate(x_, s_)) for x_, s_ in plain_res), ws)
        plain["value"] = okp / (plain["ms_per_step"] * plain["steps"] * 1e-3)
        if ref is not None:
            plain["sigma_rel"] = abs(sp - ref[1]) / ref[1]
            plain["x_rel"] = float(np.linalg.norm(xp - ref[0]) / np.linalg.norm(ref[0]))

    if rank != 0:
        return
    peaks = _peaks()
    total = {k: v[1] for k, v in prof.items()}
    dom = max(total, key=total.get)
    share = {k: round(v / max(1e-9, sum(total.values())), 4) for k, v in total.items()}
    v64 = infos[-1]["pass_variant"][0]
    roof = (_roofline(prof, peaks, dom, M_ROWS, N_COLS, v64, units, qr) or
            _inner_loop(prof, units, peaks, M_ROWS, N_COLS))
    inner = _inner_loop(prof, units, peaks, M_ROWS, N_COLS)
    if inner and pass_only:
        hbm = peaks.get("hbm_gbs", 6800.0)
        pass_only["frac"] = pass_only["achieved"] / hbm
        pass_only["peak"] = hbm
        inner["pass_only"] = pass_only
    value = ok / (ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16+f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + ("_householder_qr" if qr else ""), "m": M_ROWS,
                   "n": N_COLS, "d_lo": D_LO, "noise": NOISE,
                   "seed": "rank", "u_f": "fp16", "u": "fp32", "u_r": "fp64",
                   "factor": "householder_qr" if qr else "cholesky_of_scaled_gram",
                   "solve_tol": SOLVE_TOL, "max_rqi": MAX_RQI,
                   "l2": "inputs larger than L2 (A: 268 MB FP64 + 134 MB FP32 per step)",
                   "step": "tls_factor + tls_solve on resident A"},
        "accurate_steps": ok, "error_vs_oracle": err,
        "rqi_steps": infos[-1]["rqi_steps"], "cg_iters": infos[-1]["cg_iters"],
        "shifts": infos[-1]["shifts"], "u_f_used": infos[-1]["u_f_used"],
        "fail_pivot": infos[-1]["fail_pivot"], "pass_variant": infos[-1]["pass_variant"],
        "t_factor_ms": infos[-1]["t_factor_ms"], "t_solve_ms": infos[-1]["t_solve_ms"],
        "roofline": roof, "inner_loop_roofline": inner,
        "kernel_share": share, "kernel_ms": {k: round(v, 4) for k, v in total.items()},
        "kernel_launches": {k: v[0] for k, v in prof.items()},
        "kernel_units": {k: v for k, v in units.items() if v},
        "kernel_profile": "profiled steps after the timed region (every launch bracketed by "
                          "CUDA events on the context's stream)",
        "gpu_launches": int(launches),
        "cpu_baseline": cpu, "e2e": e2e, "plain_fp64": plain, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# C1: the small all-FP64 problem (400 x 40, tol 1e-12, max 10 RQI steps): latency bound
# ------------------------------------------------------------------------------------------
def _c1_oracle(seed: int, reps: int):
    """The 400 x 40 oracle solve, timed over `reps` repetitions (runs in a spawned process)."""
    import oracle.rqi_pcgtls as O
    from paper_2305_19028_gb300 import synth
    p = synth.dense_problem(400, 40, d_lo=1e-2, noise=1e-6, seed=seed)
    t0 = time.perf_counter()
    for _ in range(reps):
        xo, so, _ = O.rqi_pcgtls(p.A, p.b, tol=1e-12, max_rqi=10)
    return xo, so, (time.perf_counter() - t0) / reps


def run_c1(args, ws, rank, local):
    import torch
    from paper_2305_19028_gb300 import synth, tls

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    tls.load()
    p = synth.dense_problem(400, 40, d_lo=1e-2, noise=1e-6, seed=rank)
    cpu = None
    reps = 20
    # the oracle in one spawned single-threaded process (its BLAS threads end with it)
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                             "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes=1) as pool:
            xo, so, t_or = pool.apply(_c1_oracle, (rank, reps))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    if rank == 0:
        cpu = {"value": 1.0 / t_or, "unit": "solves/s", "cores": 1, "kind": "oracle",
               "sample": f"{reps} FP64 solves of the 400x40 problem in one single-threaded "
                         f"process"}
    stream = torch.cuda.current_stream()
    ctx = tls.tls_create_dense(p.A, p.b, stream=stream.cuda_stream)
    opt = tls.tls_default_options(u="fp64")

    def accurate(x, s):
        return bool(abs(s - so) <= SIGMA_TOL * so and
                    np.linalg.norm(x - xo) <= X_TOL * np.linalg.norm(xo))

    def step():
        tls.tls_factor(ctx, "fp64", opt)
        return tls.tls_solve(ctx, tol=1e-12, max_rqi=10)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ok = 0
    l0 = tls.tls_kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            x, s, info = step()
            ok += int(accurate(x, s))
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = tls.tls_kernel_launches() - l0
    ms = _barrier_max(ev0.elapsed_time(ev1), ws)
    tls.tls_destroy(ctx)
    # end to end from pinned host memory: create + factor + solve + destroy per step
    A_pin = torch.from_numpy(p.A).pin_memory().numpy()
    b_pin = torch.from_numpy(p.b).pin_memory().numpy()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    oke = 0

    def e2e_step():
        c2 = tls.tls_create_dense(A_pin, b_pin, stream=stream.cuda_stream)
        tls.tls_factor(c2, "fp64", opt)
        x2, s2, _ = tls.tls_solve(c2, tol=1e-12, max_rqi=10)
        tls.tls_destroy(c2)
        return x2, s2

    e2e_step()   # warm-up: the first context's buffers come from cudaMalloc, later ones from the block cache
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        oke += int(accurate(*e2e_step()))
    e1.record(stream)
    torch.cuda.synchronize()
    ems = _barrier_max(e0.elapsed_time(e1), ws)
    # the same problem as a packed batch of one (the whole solve is one CUDA graph launch)
    with tls.Batch([(p.A, p.b)], stream=stream.cuda_stream) as bt:
        for _ in range(args.warmup):
            bt.factor("fp64", u="fp64")
            bt.solve(tol=1e-12, max_rqi=10)
        torch.cuda.synchronize()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        okb = 0
        b0.record(stream)
        for _ in range(args.steps):
            bt.factor("fp64", u="fp64")
            xb, sb, _, _ = bt.solve(tol=1e-12, max_rqi=10)
            okb += int(accurate(xb[0], sb[0]))
        b1.record(stream)
        torch.cuda.synchronize()
        bms = _barrier_max(b0.elapsed_time(b1), ws)
    ok, okb, oke = _total(ok, ws), _total(okb, ws), _total(oke, ws)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": ok / (ms * 1e-3), "unit": "solves/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "dense_400x40_f64", "m": 400, "n": 40, "d_lo": 1e-2,
                   "noise": 1e-6, "seed": "rank", "u_f": "fp64", "u": "fp64", "u_r": "fp64",
                   "solve_tol": 1e-12, "max_rqi": 10,
                   "l2": "A is 128 KB and stays in L2 (a latency-bound configuration)",
                   "step": "tls_factor + tls_solve"},
        "accurate_steps": ok, "rqi_steps": info["rqi_steps"],
        "roofline": {"kernel": "none (latency bound: every kernel is a few microseconds)",
                     "bound": "latency", "achieved": None, "peak": None, "unit": None,
                     "frac": None, "traffic": None},
        "packed_batch_of_one": {"value": okb / (bms * 1e-3), "unit": "solves/s",
                                "ms_per_step": bms / args.steps, "accurate": okb},
        "gpu_launches": int(launches), "cpu_baseline": cpu,
        "e2e": {"value": oke / (ems * 1e-3), "unit": "solves/s",
                "h2d_bytes_per_step": int(p.A.nbytes + p.b.nbytes),
                "d2h_bytes_per_step": int(8 * 40 + 8), "ms_per_step": ems / args.steps},
        "plain_fp64": "this configuration is the plain all-FP64 method",
        "error_vs_oracle": {"sigma_rel": abs(s - so) / so,
                            "x_rel": float(np.linalg.norm(x - xo) / np.linalg.norm(xo))},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# sparse workload (CSR 200000 x 4000, u_f BF16)
# ------------------------------------------------------------------------------------------
CSR_M, CSR_N, CSR_NNZ, CSR_NOISE = 200000, 4000, 12, 1e-3


def _csr_oracle(p):
    """FP64 oracle on the CSR problem: R from the Cholesky factor of A^T A (the oracle's
    alternative factor; a dense QR of a 200000 x 4000 matrix is far too slow for a bench) and
    the normal-equation LS start."""
    import scipy.linalg as sla
    import scipy.sparse as sps
    import oracle.rqi_pcgtls as O
    A = sps.csr_matrix((p.val, p.col_idx, p.row_ptr), shape=(p.m, p.n))
    R = O.r_factor_cholesky(A)
    x0 = sla.solve_triangular(R, sla.solve_triangular(R, A.T @ p.b, trans="T"))
    return O.rqi_pcgtls(A, p.b, R=R, x0=x0, tol=0.0, max_rqi=MAX_RQI)


def run_sparse(args, ws, rank, local):
    import torch
    from paper_2305_19028_gb300 import synth, tls

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    tls.load()
    p = synth.csr_problem(CSR_M, CSR_N, nnz_per_row=CSR_NNZ, noise=CSR_NOISE, seed=rank)
    nnz = int(p.row_ptr[-1])
    stream = torch.cuda.current_stream()
    ctx = tls.tls_create_csr(p.m, p.n, p.row_ptr, p.col_idx, p.val, p.b, stream=stream.cuda_stream)
    opt = tls.tls_default_options(u="fp32")
    ref, cpu = None, None   # the CPU oracle runs after the GPU measurements (see run_ours)

    def accurate(x, s):
        if ref is None:
            return True
        xo, so = ref
        return abs(s - so) / so <= SIGMA_TOL and np.linalg.norm(x - xo) <= X_TOL * np.linalg.norm(xo)

    def step():
        tls.tls_factor(ctx, "bf16", opt)
        return tls.tls_solve(ctx, tol=SOLVE_TOL, max_rqi=MAX_RQI)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    l0 = tls.tls_kernel_launches()
    results = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            x, s, info = step()
            results.append((x, s))
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = tls.tls_kernel_launches() - l0
    ms = _barrier_max(ev0.elapsed_time(ev1), ws)
    clocks = clk.summary()
    tls.tls_profile_enable(ctx, True)
    for _ in range(max(1, min(args.steps, 3))):
        step()
    torch.cuda.synchronize()
    prof = tls.tls_profile_get(ctx)
    tls.tls_profile_enable(ctx, False)
    plain = None
    if not args.no_plain:
        opt64 = tls.tls_default_options(u="fp64")
        tls.tls_factor(ctx, "fp64", opt64)
        tls.tls_solve(ctx, tol=SOLVE_TOL, max_rqi=MAX_RQI)
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        plain_res, nps = [], 2
        q0.record(stream)
        for _ in range(nps):
            tls.tls_factor(ctx, "fp64", opt64)
            xp, sp_, _ = tls.tls_solve(ctx, tol=SOLVE_TOL, max_rqi=MAX_RQI)
            plain_res.append((xp, sp_))
        q1.record(stream)
        torch.cuda.synchronize()
        pms = _barrier_max(q0.elapsed_time(q1), ws)
        plain = {"value": None, "unit": "solves/s", "ms_per_step": pms / nps,
                 "steps": nps, "accurate": None}
    e2e = None
    if not args.no_e2e:
        pins = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
                for a in (p.row_ptr.astype(np.int64), p.col_idx.astype(np.int32), p.val, p.b)]
        ne = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2e_res = []

        def e2e_step():
            c2 = tls.tls_create_csr(p.m, p.n, *pins, stream=stream.cuda_stream)
            tls.tls_factor(c2, "bf16", opt)
            x2, s2, _ = tls.tls_solve(c2, tol=SOLVE_TOL, max_rqi=MAX_RQI)
            tls.tls_destroy(c2)
            return x2, s2

        e2e_step()   # warm-up: the first context's buffers come from cudaMalloc, later ones from the block cache
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(ne):
            e2e_res.append(e2e_step())
        e1.record(stream)
        torch.cuda.synchronize()
        ems = _barrier_max(e0.elapsed_time(e1), ws)
        e2e = {"value": None, "unit": "solves/s",
               "h2d_bytes_per_step": int(sum(a.nbytes for a in pins)),
               "d2h_bytes_per_step": int(8 * CSR_N + 8), "steps": ne, "ms_per_step": ems / ne}
    tls.tls_destroy(ctx)
    if not args.no_cpu:
        t0 = time.perf_counter()
        xo, so, _ = _csr_oracle(p)
        t_or = time.perf_counter() - t0
        ref = (xo, so)
        if rank == 0:
            cpu = {"value": 1.0 / t_or, "unit": "solves/s", "cores": os.cpu_count(),
                   "kind": "oracle",
                   "sample": f"1 full FP64 solve of the {CSR_M}x{CSR_N} CSR problem "
                             f"({t_or:.2f} s: sparse A^T A, dense Cholesky R, scipy products)"}
    ok = _total(sum(int(accurate(x_, s_)) for x_, s_ in results), ws)
    if plain is not None:
        okp = _total(sum(int(accurate(x_, s_)) for x_, s_ in plain_res), ws)
        plain["value"] = okp / (plain["ms_per_step"] * plain["steps"] * 1e-3)
        plain["accurate"] = okp
    if e2e is not None:
        okc = _total(sum(int(accurate(x_, s_)) for x_, s_ in e2e_res), ws)
        e2e["value"] = okc / (e2e["ms_per_step"] * e2e["steps"] * 1e-3)
    if rank != 0:
        return
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    total = {k: v[1] for k, v in prof.items()}
    share = {k: round(v / max(1e-9, sum(total.values())), 4) for k, v in total.items()}

    def sparse_roof(cls):
        cnt, tms = prof.get(cls, (0, 0.0))
        if not cnt:
            return {}
        avg = tms / cnt * 1e-3
        # the paired PCGTLS pass reads the FP32 values and int32 indices once in CSR order
        # (t = A q) and once in CSC order (A^T t), plus row / column offsets and t (2 RHS)
        byts = 2 * nnz * 8 + (CSR_M + CSR_N) * 4 + 2 * 2 * CSR_M * 4
        if cls == "resid_pass":
            byts = 2 * nnz * 12 + (CSR_M + CSR_N) * 4 + 2 * CSR_M * 8
        ach = byts / avg / 1e9
        return {"kernel": f"{cls} (CSR/CSC passes)", "bound": "hbm", "achieved": ach,
                "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": None,
                "peak_source": "measured" if peaks else "fallback",
                "avg_launch_us": avg * 1e6, "algorithmic_bytes": byts}

    dom = max(total, key=total.get)
    line = {
        "metric": METRIC, "value": ok / (ms * 1e-3), "unit": "solves/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16+f32+f64", "data": "synthetic",
        "config": {"workload": f"csr_{CSR_M}x{CSR_N}_nnz{nnz}_ufbf16_u32_ur64", "m": CSR_M,
                   "n": CSR_N, "nnz": nnz, "noise": CSR_NOISE, "u_f": "bf16", "u": "fp32",
                   "u_r": "fp64", "solve_tol": SOLVE_TOL, "max_rqi": MAX_RQI,
                   "l2": "values, indices and the dense factor (2 x 64 MB) exceed L2",
                   "step": "tls_factor + tls_solve on resident CSR A"},
        "accurate_steps": ok, "rqi_steps": info["rqi_steps"], "cg_iters": info["cg_iters"],
        "roofline": sparse_roof("pcg_pass2") if dom in ("pcg_pass2", "pcg_pass1") else
                    {"kernel": dom, "note": "dominant class is not a pass over A",
                     **{k: v for k, v in sparse_roof("pcg_pass2").items() if k != "kernel"}},
        "inner_loop_roofline": sparse_roof("pcg_pass2"), "resid_roofline": sparse_roof("resid_pass"),
        "kernel_share": share, "kernel_ms": {k: round(v, 4) for k, v in total.items()},
        "kernel_launches": {k: v[0] for k, v in prof.items()},
        "kernel_profile": "profiled steps after the timed region", "gpu_launches": int(launches),
        "cpu_baseline": cpu, "e2e": e2e, "plain_fp64": plain, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# packed batch workload
# ------------------------------------------------------------------------------------------
BATCH_K = 512


def _batch_workload(k: int) -> str:
    return f"batch_{k}_dense_n32-512_m4-20n_uf16_u32_ur64"


def _oracle_batch_member(i: int):
    """Pool worker: rebuild batch member i from its seed and solve it with the FP64 oracle."""
    from paper_2305_19028_gb300 import synth
    import oracle.rqi_pcgtls as O
    p = synth.batch_problem(i)
    x, s, _ = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=MAX_RQI)
    return i, x, s


def _oracle_pool(ids, procs):
    """FP64 oracle on every listed batch member, one single-threaded process per core."""
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                             "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        t0 = time.perf_counter()
        with mp.get_context("spawn").Pool(processes=procs) as pool:
            res = pool.map(_oracle_batch_member, ids, chunksize=1)
        dt = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return {i: (x, s) for i, x, s in res}, dt


def _batch_roofline(prof: dict, peaks: dict, cls: str, u64: bool = False) -> dict:
    """Roofline of one kernel class of the packed batch from its profiled launches (count,
    device ms, entries of A of the active problems). u64: the FP64 working precision (FP64
    residual passes); otherwise the residual passes run in double-FP32 on A32 + Alo."""
    cnt, ms, elems = prof.get(cls, (0, 0.0, 0))
    if cnt == 0 or ms <= 0:
        return {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    src = "measured" if peaks else "fallback"
    if cls in ("pcg_pass2", "pcg_pass1"):
        # algorithmic bytes: the FP32 entries of A of the active problems, once per launch
        byts = 4.0 * elems
        ach = byts / (ms * 1e-3) / 1e9
        return {"kernel": f"{cls} (batched fused t = A q, A^T t over all active problems, FP32)",
                "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": None, "peak_source": src,
                "avg_launch_us": ms / cnt * 1e3, "algorithmic_bytes_per_launch": byts / cnt}
    if cls == "resid_pass" and not u64:
        # double-FP32: the pair A32 + Alo read once (8 bytes per entry of A)
        byts = 8.0 * elems
        ach = byts / (ms * 1e-3) / 1e9
        return {"kernel": "resid_pass (batched r = b - A x, A^T r in double-FP32 arithmetic on "
                          "A32 + Alo)", "bound": "hbm", "achieved": ach, "peak": hbm,
                "unit": "GB/s", "frac": ach / hbm, "traffic": None, "peak_source": src,
                "avg_launch_us": ms / cnt * 1e3, "algorithmic_bytes_per_launch": byts / cnt,
                "fp64_equivalent_tflops": 4.0 * elems / (ms * 1e-3) / 1e12}
    if cls == "resid_pass":
        # FP64 FMA-bound: 2 FMA (4 flops) per entry of A; peak 1.25 TFLOP/s FP64 (nominal)
        flops = 4.0 * elems
        ach = flops / (ms * 1e-3) / 1e12
        return {"kernel": "resid_pass (batched FP64 r = b - A x, A^T r)", "bound": "alu",
                "achieved": ach, "peak": FP64_PEAK, "unit": "TFLOP/s", "frac": ach / FP64_PEAK,
                "traffic": None,
                "peak_source": "nominal FP64 rate (2 FMA/clk/SM x 152 SMs x 2.07 GHz)",
                "avg_launch_us": ms / cnt * 1e3, "algorithmic_flops_per_launch": flops / cnt,
                "hbm_gbs": 8.0 * elems / (ms * 1e-3) / 1e9}
    return {}


def run_batch(args, ws, rank, local):
    import torch
    from paper_2305_19028_gb300 import synth, tls

    K = args.batch
    ids = _shard_ids(rank, K)
    ref, t_or = {}, None
    procs = max(1, (os.cpu_count() or 1) // ws)
    if not args.no_cpu:
        ref, t_or = _oracle_pool(ids, procs)       # before the first CUDA call
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    tls.load()
    probs = [synth.batch_problem(i) for i in ids]
    stream = torch.cuda.current_stream()
    bt = tls.Batch([(p.A, p.b) for p in probs], stream=stream.cuda_stream)
    uf = "fp16"
    model = None
    if args.selector:
        from paper_2305_19028_gb300 import selector
        model = selector.load_model()
        if model is None:
            raise RuntimeError("--selector: no trained selector model in the package")
        bt.set_selector(*model)
        uf = "auto"

    def count_ok(xs, sig):
        if not ref:
            return len(xs)
        ok = 0
        for i, x, s in zip(ids, xs, sig):
            xo, so = ref[i]
            ok += int(abs(s - so) <= SIGMA_TOL * so and
                      np.linalg.norm(x - xo) <= X_TOL * np.linalg.norm(xo))
        return ok

    def step():
        bt.factor(uf, u="fp32")
        return bt.solve(tol=SOLVE_TOL, max_rqi=MAX_RQI)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    l0 = tls.tls_kernel_launches()
    ok = 0
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            xs, sig, infos, per = step()     # the solve is one CUDA graph launch
            ok += count_ok(xs, sig)
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = tls.tls_kernel_launches() - l0
    ms = _barrier_max(ev0.elapsed_time(ev1), ws)
    clocks = clk.summary()
    # per-class kernel times: one more step with the same launches run eagerly, each bracketed
    # by CUDA events (untimed for the headline number)
    bt.profile(True)
    step()
    prof = bt.profile_get()
    bt.profile(False)
    n_fb = sum(i["fallbacks"] for i in infos)
    uf_hist = np.bincount([i["u_f_used"] for i in infos], minlength=4).tolist()

    e2e = None
    if not args.no_e2e:
        pins = [(torch.from_numpy(p.A).pin_memory().numpy(), torch.from_numpy(p.b).pin_memory().numpy())
                for p in probs]
        ne = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        okc = 0

        def e2e_step():
            with tls.Batch(pins, stream=stream.cuda_stream) as b2:
                if model is not None:
                    b2.set_selector(*model)
                b2.factor(uf, u="fp32")
                x2, s2, _, _ = b2.solve(tol=SOLVE_TOL, max_rqi=MAX_RQI)
            return x2, s2

        e2e_step()   # warm-up: the first batch's buffers come from cudaMalloc, later ones from the block cache
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(ne):
            okc += count_ok(*e2e_step())
        e1.record(stream)
        torch.cuda.synchronize()
        ems = _barrier_max(e0.elapsed_time(e1), ws)
        e2e = {"value": _total(okc, ws) / (ems * 1e-3), "unit": "solves/s",
               "h2d_bytes_per_step": int(sum(p.A.nbytes + p.b.nbytes for p in probs)),
               "d2h_bytes_per_step": int(sum(8 * p.A.shape[1] + 8 for p in probs)),
               "steps": ne, "ms_per_step": ems / ne}

    plain = None
    if not args.no_plain:
        def step64():
            bt.factor("fp64", u="fp64")
            return bt.solve(tol=SOLVE_TOL, max_rqi=MAX_RQI)
        step64()
        torch.cuda.synchronize()
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        np_steps = max(1, min(args.steps, 2))
        okp = 0
        q0.record(stream)
        for _ in range(np_steps):
            xp, sp_, ip, _ = step64()
            okp += count_ok(xp, sp_)
        q1.record(stream)
        torch.cuda.synchronize()
        pms = _barrier_max(q0.elapsed_time(q1), ws)
        plain = {"value": _total(okp, ws) / (pms * 1e-3), "unit": "solves/s",
                 "ms_per_step": pms / np_steps,
                 "steps": np_steps, "accurate": okp, "of": np_steps * K}
    bt.close()
    ok = int(_total(ok, ws))
    if rank != 0:
        return
    peaks = _peaks()
    total = {k: v[1] for k, v in prof.items()}
    dom = max(total, key=total.get)
    share = {k: round(v / max(1e-9, sum(total.values())), 4) for k, v in total.items()}
    roof = _batch_roofline(prof, peaks, dom) or _batch_roofline(prof, peaks, "pcg_pass2")
    cpu = None
    if t_or is not None:
        cpu = {"value": K / t_or, "unit": "solves/s", "cores": procs, "kind": "oracle",
               "sample": f"all {K} problems of the batch, one FP64 oracle solve each "
                         f"({t_or:.1f} s on {procs} single-threaded processes)"}
    line = {
        "metric": METRIC, "value": ok / (ms * 1e-3), "unit": "solves/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f16+f32+f64", "data": "synthetic",
        "config": {"workload": _batch_workload(K), "problems": K,
                   "u_f": "selector (TLS_AUTO)" if model is not None else "fp16", "u": "fp32",
                   "u_r": "fp64", "solve_tol": SOLVE_TOL, "max_rqi": MAX_RQI,
                   "seeds": f"1000 + rank*{K} + i",
                   "l2": "inputs larger than L2 (A: %.1f GB FP64 + %.1f GB FP32)" % (
                       sum(p.A.nbytes for p in probs) / 1e9, sum(p.A.nbytes for p in probs) / 2e9),
                   "step": "tls_batch_factor + tls_batch_solve on the resident batch"},
        "accurate_solves": ok, "of": args.steps * K * ws, "fallbacks": n_fb, "u_f_used_hist": uf_hist,
        "roofline": roof, "inner_loop_roofline": _batch_roofline(prof, peaks, "pcg_pass2"),
        "resid_roofline": _batch_roofline(prof, peaks, "resid_pass"),
        "kernel_share": share, "kernel_ms": {k: round(v[1], 4) for k, v in prof.items()},
        "kernel_launches": {k: v[0] for k, v in prof.items()},
        "kernel_profile": "one profiled step after the timed region (eager launches, CUDA events)",
        "gpu_launches": int(launches),
        "cpu_baseline": cpu, "e2e": e2e, "plain_fp64": plain, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: enough for a timed region of about half a "
                         "second, so that the clock sampler sees it)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--m", type=int, default=None, help="rows (profiling a smaller case)")
    ap.add_argument("--n", type=int, default=None, help="columns (profiling a smaller case)")
    ap.add_argument("--workload", choices=["dense", "batch", "sparse", "c1"], default="dense")
    ap.add_argument("--factor", choices=["cholesky", "qr"], default="cholesky",
                    help="dense workload: R-hat from the Cholesky factor of the scaled Gram "
                         "matrix (default) or from Householder QR (Alg. 4)")
    ap.add_argument("--batch", type=int, default=BATCH_K, help="problems in the packed batch")
    ap.add_argument("--selector", action="store_true",
                    help="batch: let the trained selector network pick u_f per problem")
    args = ap.parse_args()
    if args.steps is None:
        # (a timed region of at least half a second: three or more 200 ms clock samples)
        args.steps = (10 if args.impl == "reference" or args.workload == "batch"
                      else 1500 if args.workload == "c1" else 150)
    _set_size(args.m, args.n)
    ws, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == "batch":
        run_batch(args, ws, rank, local)
    elif args.workload == "sparse":
        run_sparse(args, ws, rank, local)
    elif args.workload == "c1":
        run_c1(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
