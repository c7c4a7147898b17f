#!/usr/bin/env python3
"""Benchmark of the SGS-PFP solver on GB300: cell updates per second.

Workload: planar heat transfer, 64 cells on [0, 1], 32^3 velocities on [-8, 8]^3, Maxwell
molecules (B = 1/(4 pi)), eps = 0.01, diffuse walls with seeded temperatures
T_L ~ U[0.8, 1.2], T_R ~ U[1.5, 2.5] (seed 0), synthetic initial state.

A step is one SGS iteration of the mixed solver: forward scan, collision, backward scan,
mass rescale, collision (the collision sums in FP32, moments/Newton/residual in FP64), with
the FP64 defect-correction evaluation (FP64 collision + FP64 residual + right-hand side)
every --dc-every steps. One cell update is one cell visit of a scan; a step makes 2 x 64.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference] [--workload heat|shock]

--workload cavity runs them on the 2-D lid-driven cavity (64 x 64 cells on [0, 1]^2, 24^3
velocities on [-6, 6]^3, Maxwell molecules, eps = 0.05, lid speed 0.5, walls at T = 1,
four orderings per SGS iteration, V-cycles on 64^2/32^2/16^2 cells).
--workload shock runs the same measurements on the Mach-2 normal shock (128 cells on
[-20, 20], 32^3 velocities on [-10, 10]^3, hard spheres, eps = 0.1, Rankine-Hugoniot inflow
data, two-level V-cycles on 128/64 cells: deeper ones go non-finite on this shock) and records
the shock position.

--conserve-proj 1|2 adds the FP64 conservation projection of Q (plain or Maxwellian-weighted;
not in the paper); --pin-mass holds the shock's total mass at its initial value (eq. (32));
--order 2 runs the second-order scheme (1-D workloads).

N > 1 runs independent replicas (one per GPU, launched by torchrun): the method is a
sequential scan per problem, so work is replicated, not sharded ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("cell-updates/s (mixed-precision SGS-PFP; time to residual 1e-8, mixed vs FP64, under "
          "time_to_residual_1e-8)")
UNIT = "cell-updates/s"
L2_BYTES = 129 * 2**20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--dc-every", type=int, default=10)
    ap.add_argument("--workload", choices=["heat", "shock", "cavity", "batch", "paper_bgk_cavity"], default="heat",
                    help="heat: 64-cell heat transfer (default); shock: 128-cell Mach-2 normal shock; "
                         "cavity: 64 x 64 lid-driven cavity (2-D space); batch: 64 independent heat-transfer "
                         "instances of uneven size, grid and eps (one CUDA graph per defect-correction cycle)")
    ap.add_argument("--batch-size", type=int, default=64, help="instances of the batch workload")
    ap.add_argument("--paper-eps", default="1,0.1,0.01,0.001,0.0001",
                    help="paper_bgk_cavity: Knudsen numbers to time (comma separated)")
    ap.add_argument("--lo-iters", type=int, default=10, help="SGS iterations per defect-correction cycle (batch)")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-t2tol", action="store_true", help="skip the time-to-residual runs")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default scan shape")
    ap.add_argument("--no-overlap", action="store_true",
                    help="sequential iterations (no collision steps pipelined behind the scans)")
    ap.add_argument("--t2tol-all", action="store_true", help="also time the plain FP64 SGS form to 1e-8")
    ap.add_argument("--t2tol-cap", type=float, default=150.0, help="seconds allowed per time-to-residual run")
    ap.add_argument("--t2tol-kinds", default="mixed_mg,mixed_sgs,fp64_mg",
                    help="comma-separated time-to-residual runs (mixed_mg, mixed_sgs, fp64_mg, fp64_sgs)")
    ap.add_argument("--batch-t2tol-cap", type=float, default=0.0,
                    help="batch: seconds of defect-correction cycles from the initial states to time every "
                         "instance to residual 1e-8 (0: off)")
    ap.add_argument("--conserve-proj", type=int, choices=[0, 1, 2], default=0,
                    help="conservation projection of Q: 0 the paper's operator, 1 plain, 2 Maxwellian-weighted")
    ap.add_argument("--order", type=int, choices=[1, 2], default=1,
                    help="spatial order of the 1-D scheme (2: linear reconstruction, eq. (slope))")
    ap.add_argument("--pin-mass", action="store_true",
                    help="shock: hold the total mass at the initial state's (eq. (32) rescale), pinning the shock")
    ap.add_argument("--case", choices=["sweep", "sum", "sum64", "sumdf", "sweep2d", "dft", "peaks", "steps", "fast"],
                    default=None,
                    help="run a small case of one kernel class (for profiler captures) and exit")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_barrier(world):
    """Barrier across the ranks around a timed region (N > 1)."""
    if world > 1:
        import torch

        torch.distributed.barrier()


def max_over_ranks(ms, world, device="cpu"):
    """The slowest rank's time: a timed region lasts until every rank is done."""
    if world <= 1:
        return float(ms)
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms_total):
    """Units processed by all ranks per second of the slowest rank's time (weak scaling:
    every rank runs the same independent work)."""
    return world * units_per_rank / (ms_total * 1e-3)


# ------------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------- native
WORKLOAD = "heat"
CONSERVE_PROJ = 0   # --conserve-proj
PIN_MASS = False    # --pin-mass (shock)
ORDER = 1           # --order


def workload():
    from paper_2409_01910_gb300 import inputs as I

    if WORKLOAD == "shock":
        return I.shock_128cells_32v()
    if WORKLOAD == "cavity":
        return I.cavity_64x64_24v()
    if WORKLOAD == "batch":
        return I.heat_batch(64, seed=0)[0]  # the oracle sample of the batch: its first instance
    return I.heat_64cells_32v(seed=0)


def is_shock(wl):
    return hasattr(wl, "up")


def is_cavity(wl):
    return hasattr(wl, "ny")


def visits_per_iteration(wl):
    """Cell visits of one SGS iteration: two scans in 1-D, four orderings in 2-D."""
    return (4 if is_cavity(wl) else 2) * wl.J


def shock_mass(wl):
    """Total mass of the shock's initial state, sum_j dx sum_k w f0 (the --pin-mass constant)."""
    dx = (wl.x_hi - wl.x_lo) / wl.J
    return float(wl.initial_state().sum()) * (2 * wl.L / wl.N) ** 3 * dx


def make_solver(wl, precision):
    from paper_2409_01910_gb300 import sgs

    if is_cavity(wl):
        p = sgs.Problem(space_dim=2, nx=wl.nx, ny=wl.ny, nv=wl.N, v_max=wl.L, eps=wl.eps,
                        bc_T=(wl.T_wall, wl.T_wall), bc_T_y=(wl.T_wall, wl.T_wall),
                        bc_u_y=((0.0, 0.0, 0.0), (wl.lid, 0.0, 0.0)), total_mass=wl.total_mass, precision=precision)
    elif is_shock(wl):
        (r1, u1, T1), (r2, u2, T2) = wl.up, wl.down
        p = sgs.Problem(nx=wl.J, x_lo=wl.x_lo, x_hi=wl.x_hi, nv=wl.N, v_max=wl.L, collision=sgs.HARD_SPHERE,
                        eps=wl.eps, bc_kind=(sgs.INFLOW, sgs.INFLOW), bc_rho=(r1, r2),
                        bc_u=((u1, 0.0, 0.0), (u2, 0.0, 0.0)), bc_T=(T1, T2),
                        total_mass=shock_mass(wl) if PIN_MASS else 0.0, precision=precision)
    else:
        p = sgs.Problem(nx=wl.J, x_lo=wl.x_lo, x_hi=wl.x_hi, nv=wl.N, v_max=wl.L, eps=wl.eps,
                        bc_T=(wl.T_left, wl.T_right), total_mass=wl.total_mass, precision=precision)
    p.conserve_proj = CONSERVE_PROJ
    if ORDER != 1:
        p.order = ORDER
    return sgs.Solver(p)


def config_of(wl):
    c = _config_of(wl)
    if CONSERVE_PROJ:
        c["conserve_proj"] = ["plain", "maxwellian_weighted"][CONSERVE_PROJ - 1]
    if PIN_MASS and is_shock(wl):
        c["total_mass_pinned"] = True
    if ORDER != 1:
        c["order"] = ORDER
    return c


def _config_of(wl):
    if is_cavity(wl):
        return {"workload": wl.name, "cells": [wl.nx, wl.ny], "domain": [[0.0, 1.0], [0.0, 1.0]], "nv": wl.N,
                "v_max": wl.L, "eps": wl.eps, "collision": "maxwell", "lid_speed": wl.lid, "T_walls": wl.T_wall,
                "orderings": 4, "multigrid_levels": 3}
    if is_shock(wl):
        return {"workload": wl.name, "cells": wl.J, "x": [wl.x_lo, wl.x_hi], "nv": wl.N, "v_max": wl.L,
                "eps": wl.eps, "collision": "hard spheres", "inflow_up": [round(float(x), 6) for x in wl.up],
                "inflow_down": [round(float(x), 6) for x in wl.down], "multigrid_levels": 4}
    return {"workload": wl.name, "cells": wl.J, "nv": wl.N, "v_max": wl.L, "eps": wl.eps,
            "T_walls": [round(wl.T_left, 6), round(wl.T_right, 6)], "collision": "maxwell"}


def pairs_per_cell(N):
    h = N // 2 - 1
    return (3 * h * h + 3 * h + 1) ** 3


def run_native(args, rank, world, local):
    import torch

    from paper_2409_01910_gb300 import sgs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    wl = workload()
    f0 = torch.from_numpy(wl.initial_state().reshape(-1)).to(dev)
    s = make_solver(wl, sgs.FP32)
    if args.no_overlap:
        s.set_overlap(False)
    f = f0.clone()
    Q, P = s.field(), s.field()
    res_hi = torch.zeros(1, dtype=torch.float64, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    visits_per_step = visits_per_iteration(wl)

    # scan-shape autotuner (untimed, on a scratch copy of the state): keeps the fastest shape
    tuning = None
    if not args.no_autotune:
        g, Qt, Pt = f0.clone(), s.field(), s.field()
        s.collide(g, Qt, Pt)
        tuning = s.autotune(g, Pt, reps=1)
        del g, Qt, Pt
        s.reset_stats()

    def step(i):
        if i % args.dc_every == 0:
            s.dc_step(f, Q, P, 0, res=res_hi)
        s.iterate(f, Q, P, flags=sgs.IT_P_VALID | sgs.IT_EVAL)

    # measured denominators of the rooflines (FMA pipes, SM count, scan latencies), untimed
    peaks = measure_peaks(wl, s.sweep_shape(), local)

    # warm-up (untimed): the first DC evaluation also initialises P
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    rank_barrier(world)
    # the state after the warm-up (fields and the handle's workspace, which holds the
    # defect-correction reference and the Maxwellians): the profiled and end-to-end passes
    # start from it again, so that all three time the same iterations
    snap = [x.clone() for x in (f, Q, P, s.workspace)]

    def restore():
        for x, y in zip((f, Q, P, s.workspace), snap):
            x.copy_(y)
        torch.cuda.synchronize()

    def timed_pass(first, profiled):
        """K steps from step index `first`, each bracketed by CUDA events on the launching
        stream, an L2 flush between steps; the library's per-class event profiler on or off."""
        s.profile(profiled)
        s.profile_read()
        n0 = s.launch_count()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (outside the events)
            ev[i][0].record(stream)
            step(first + i)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        prof = s.profile_read(with_work=True)
        s.profile(False)
        return [a.elapsed_time(b) for a, b in ev], s.launch_count() - n0, prof

    # the headline: profiler off
    with ClockSampler(local) as clk:
        ms_steps, launches, _ = timed_pass(args.warmup, False)
        rank_barrier(world)
    ms_total = max_over_ranks(sum(ms_steps), world, dev)
    value = whole_job_rate(visits_per_step * args.steps, world, ms_total)
    # the per-class split: the same K steps again with every launch group bracketed by events
    restore()
    ms_prof_steps, _, prof_w = timed_pass(args.warmup, True)
    prof = {k: (v[0], v[1]) for k, v in prof_w.items()}
    status = s.read_status()

    # dominant kernel class and its roofline
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    dom = max(prof, key=lambda k: prof[k][0])
    roofs = {k: roofline(k, prof_w, wl, sm_mhz, peaks, status) for k in ("sweep", "sum", "sum_fp64", "sum_df64")
             if prof[k][1] > 0}
    roof = roofs.get(dom) or roofline(dom, prof_w, wl, sm_mhz, peaks, status)

    # end to end through the C ABI with host buffers: H2D of the state (f, P), one step,
    # D2H of the step's residual
    e2e = None
    if rank == 0 or world > 1:
        restore()
        e2e = end_to_end(s, f, Q, P, wl, args, stream, restore)

    # plain FP64 GPU form for comparison (same step, FP64 collision sum and FP64 scan)
    fp64 = fp64_form(wl, args, f0, dev, stream) if args.fp64_steps > 0 else None

    # time to FP64 residual 1e-8 from the initial state, mixed against FP64 (one GPU only)
    t2tol = None
    if world == 1 and not args.no_t2tol:
        kinds = [k for k in args.t2tol_kinds.split(",") if k] + (["fp64_sgs"] if args.t2tol_all else [])
        t2tol = {k: time_to_tol(wl, f0, dev, k, args.t2tol_cap, shape=s.sweep_shape()) for k in kinds}

    out = None
    if rank == 0:
        out = {
            "metric": METRIC,
            "value": value,
            "unit": UNIT,
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_total / args.steps,
            "ms_steps": [round(x, 3) for x in ms_steps],
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32+f64",
            "data": "synthetic",
            "config": {**config_of(wl),
                       "precision": ("mixed: FP32 direct spectral sums in increment form against the last "
                                     "high-precision evaluation; defect-correction sums in double-float (FP32 "
                                     "pairs); double-float scans with FP64 scalar decisions; FP64 moments, "
                                     "transforms and residual"),
                       "dc_every": args.dc_every, "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roof,
            "roofline_kernels": roofs,
            "pipelined": s.overlap(),
            "scan_shape": {"nodes_per_thread": s.sweep_shape()[0], "ctas_per_cluster": s.sweep_shape()[1],
                           "threads_per_cta": s.sweep_shape()[2],
                           "chosen_by": "autotuner" if tuning else "default", "tuning": tuning},
            "kernels_ms": {k: round(v[0], 3) for k, v in prof.items()},
            "kernels_ms_from": (f"a second pass of the same {args.steps} steps with the library's event profiler on "
                                f"({sum(ms_prof_steps) / args.steps:.3f} ms per step there); the headline pass "
                                "runs without it"),
            "measured_peaks": peaks,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": int(launches),
            "fp64": fp64,
            "time_to_residual_1e-8": t2tol,
            "device_status": status["status"],
            "inner_iters_per_visit": status["inner_iters"] / max(1, status["visits"]),
        }
    return out


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path)), "of measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "of fallback"


def kernel_traffic(name, units):
    """DRAM bytes per launch from the committed ncu summary, scaled by the units (cell visits)
    of one launch; None when the kernel's sources changed since the capture."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(name)
    if not rec:
        return None
    h = hashlib.sha256()
    for src in rec["sources"]:
        h.update(open(os.path.join(ROOT, src), "rb").read())
    if h.hexdigest() != rec["sources_sha256"]:
        return None
    return rec["dram_bytes_per_unit"] * units


def measure_peaks(wl, shape, local=0):
    """Denominators measured on this device, untimed, before the timed region: the FFMA and
    DFMA throughput of the CUDA cores (sgs_peak_fma: independent FMA chains on every SM), the
    SM count, the SM clock sampled while the FFMA probe runs, and the latencies of the
    scan's building blocks in the scan's launch shape (sgs_probe_scan: a cluster reduction,
    a Newton iteration of the discrete Maxwellian)."""
    from paper_2409_01910_gb300 import sgs

    with ClockSampler(local) as clk:
        t_end = time.perf_counter() + 1.0
        fp32 = []
        while time.perf_counter() < t_end:  # about a second of FFMA load for the clock samples
            fp32.append(sgs.peak_fma(sgs.FP32, iters=1 << 20))
    fp64 = max((sgs.peak_fma(sgs.FP64, iters=1 << 14) for _ in range(3)), key=lambda x: x["tflops"])
    packed = max((sgs.peak_fma(sgs.FP32 | sgs.PEAK_PACKED, iters=1 << 19) for _ in range(3)),
                 key=lambda x: x["tflops"])
    best32 = max(fp32, key=lambda x: x["tflops"])
    ept, cluster, threads = shape
    precision = sgs.FP32  # the mixed solver's scans run in double-float
    red = sgs.probe_scan(wl.N, wl.L, precision, cluster, threads, 0, reps=4000)
    newt = sgs.probe_scan(wl.N, wl.L, precision, cluster, threads, 1, reps=4000)
    cbar = sgs.probe_scan(wl.N, wl.L, precision, cluster, threads, 2, reps=4000)
    return {"fp32_ffma_tflops": round(best32["tflops"], 3), "fp64_dfma_tflops": round(fp64["tflops"], 4),
            "fp32_packed_ffma2_tflops": round(packed["tflops"], 3),
            "sms": best32["sms"], "sm_mhz_during_probe": clk.summary().get("sm_mhz"),
            "scan_cluster_reduce_us": round(red, 3), "scan_newton_iteration_us": round(newt, 3),
            "scan_cluster_barrier_us": round(cbar, 3),
            "scan_probe_shape": {"ctas_per_cluster": cluster, "threads_per_cta": threads, "arith": "double-float"},
            "how": ("sgs_peak_fma: 8 independent FMA chains per thread, every SM fully occupied, CUDA events; "
                    "sgs_probe_scan: 4000 dependent operations in one cluster minus an empty launch")}


def roofline(cls, prof, wl, sm_mhz, peaks, stats=None):
    """Roofline of one kernel class over the profiled pass: its algorithmic work (from the
    cells the library reports each bracketed launch group processed) over its time (CUDA
    events on the launching stream), against the measured peak of the pipe that bounds it
    (measure_peaks) or the measured HBM bandwidth. Per launch and over the pass the ratio is
    the same: both are sums over the same launches."""
    ms, n, cells = prof[cls]
    hbm, src = measured_peaks()
    K = wl.N ** 3
    if cls in ("sum", "sum_fp64"):
        # algorithmic work: 10 flops per mode pair over the Hermitian half, per cell evaluated
        flops = 10 * 0.5 * pairs_per_cell(wl.N) * cells
        ach = flops / (ms * 1e-3) / 1e12
        if cls == "sum":
            peak = peaks["fp32_ffma_tflops"]
            return {"kernel": "k_sum<float> (direct spectral sum, FP32)", "bound": "alu", "achieved": ach,
                    "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                    "peak_source": f"FFMA rate measured by sgs_peak_fma on {peaks['sms']} SMs (of measured)"}
        peak = peaks["fp64_dfma_tflops"]
        return {"kernel": "k_sum<double> (direct spectral sum, FP64)", "bound": "alu", "achieved": ach,
                "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                "peak_source": f"DFMA rate measured by sgs_peak_fma on {peaks['sms']} SMs (of measured)"}
    if cls == "sum_df64":
        # FP32-pipe operations of one pair in the double-float sum: 8 for w b (two
        # two-products with cross terms) + 4 x 12 for the products with a and their two-sum
        # accumulation; the pipe issues one operation per lane per clock, half the FFMA flop rate
        ops = 56 * 0.5 * pairs_per_cell(wl.N) * cells
        ach = ops / (ms * 1e-3) / 1e12
        peak = peaks["fp32_ffma_tflops"] / 2.0
        return {"kernel": "k_sum_df (direct spectral sum, double-float on the FP32 pipes)", "bound": "alu",
                "achieved": ach, "peak": peak, "unit": "T FP32-pipe op/s", "frac": ach / peak, "traffic": None,
                "peak_source": "half the FFMA flop rate measured by sgs_peak_fma (one op per lane per clock; "
                               "of measured)"}
    if cls == "sweep":
        # per visit: read the upwind/downwind neighbours, f_j and P_j, write f_j (1-D: 5 K
        # doubles; 2-D: 7 K doubles)
        byts = (7 if is_cavity(wl) else 5) * K * 8 * cells
        ach = byts / (ms * 1e-3) / 1e9
        out = {"kernel": "k_sweep<dfloat,8> (persistent SGS scan, one cluster per instance)", "bound": "hbm",
               "achieved": ach, "peak": hbm["hbm_gbs"], "unit": "GB/s", "frac": ach / hbm["hbm_gbs"],
               "traffic": kernel_traffic("k_sweep<dfloat,8>", cells / max(1, n)),
               "traffic_per": f"launch of {cells / max(1, n):.0f} cell visits",
               "peak_source": f"hbm_gbs ({src})",
               "note": "latency-bound: one visit is a chain of cluster reductions and Newton solves"}
        if stats and stats.get("visits") and not is_cavity(wl):
            out["latency_model"] = scan_latency_model(ms * 1e3 / cells, stats, peaks)
        return out
    byts = 2 * K * 8 * wl.J * n
    ach = byts / (ms * 1e-3) / 1e9
    return {"kernel": cls, "bound": "hbm", "achieved": ach, "peak": hbm["hbm_gbs"], "unit": "GB/s",
            "frac": ach / hbm["hbm_gbs"], "traffic": None, "peak_source": f"hbm_gbs ({src})"}


def scan_latency_model(us_per_visit, stats, peaks):
    """The scan's time per cell visit against the chain it runs: cluster reductions (two per
    visit, then one per inner update) and Newton iterations (each an evaluation of the
    separable Maxwellian with its combination and factorisation; one more evaluation per
    solve that starts without one), at the latencies measured by sgs_probe_scan."""
    v = stats["visits"]
    inner = stats["inner_iters"] / v
    reductions = 2.0 + inner
    evaluations = (stats["newton_iters"] + stats["newton_solves"]) / v
    t_red = reductions * peaks["scan_cluster_reduce_us"]
    t_newton = evaluations * peaks["scan_newton_iteration_us"]
    return {"us_per_visit_measured": round(us_per_visit, 2), "inner_updates_per_visit": round(inner, 3),
            "cluster_reductions_per_visit": round(reductions, 3),
            "newton_evaluations_per_visit": round(evaluations, 3),
            "us_cluster_reductions": round(t_red, 2), "us_newton": round(t_newton, 2),
            "modelled_fraction": round((t_red + t_newton) / us_per_visit, 3),
            "rest": "elementwise passes over the cell's nodes, loads of neighbours and P, the per-visit set-up"}


def time_to_tol(wl, f0, dev, kind, cap_s, tol=1e-8, shape=None):
    """Seconds from the initial state until the FP64 residual falls below tol.

    kinds: mixed_sgs (defect correction every 10 SGS iterations), mixed_mg (defect
    correction before every 2 two-level V-cycles), fp64_sgs (SGS iterations, FP64 sums and
    scans), fp64_mg (two-level V-cycles in FP64)."""
    import torch

    from paper_2409_01910_gb300 import sgs

    s = make_solver(wl, sgs.FP32 if kind.startswith("mixed") else sgs.FP64)
    if shape is not None and kind.startswith("mixed"):
        s.set_sweep_shape(*shape)  # the bench handle's autotuned shape (same arithmetic)
    # cavity 64^2/32^2/16^2; the shock two levels (128/64): deeper coarse grids put the shock
    # inside a few cells and their corrections drive coarse moments non-positive
    levels = 3 if is_cavity(wl) else 2
    f = f0.clone()
    Q, P = s.field(), s.field()
    res = torch.zeros(1, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r, iters, reached = float("nan"), 0, False
    while time.perf_counter() - t0 < cap_s:
        if kind == "mixed_sgs":
            s.dc_step(f, Q, P, 10, res=res)
            iters += 10
        elif kind == "mixed_mg":
            s.dc_step(f, Q, P, 0, res=res)
        elif kind == "fp64_sgs":
            s.iterate(f, Q, P, flags=sgs.IT_EVAL | (sgs.IT_P_VALID if iters else 0), res=res)
            iters += 1
        else:
            s.collide(f, Q, P)
            s.residual(f, Q, res)
        r = float(res.item())  # synchronises
        if r < tol or r != r:
            reached = r < tol
            break
        if kind == "mixed_mg" or kind == "fp64_mg":
            for _ in range(2 if kind == "mixed_mg" else 1):
                s.vcycle(f, levels, 1, 1, 4)
                iters += 1
    sec = time.perf_counter() - t0
    st = s.read_status()
    out = {"seconds": round(sec, 3), "reached": reached, "residual": r,
           ("V-cycles" if kind.endswith("mg") else "SGS iterations"): iters, "status": st["status"]}
    if is_shock(wl):
        # shock position: where the density crosses the mean of the two inflow densities
        K = wl.N ** 3
        rho = (f.view(wl.J, K).sum(1) * (2 * wl.L / wl.N) ** 3).cpu().numpy()
        mid = 0.5 * (wl.up[0] + wl.down[0])
        j = int(np.argmax(rho > mid))
        dx = (wl.x_hi - wl.x_lo) / wl.J
        if 0 < j < wl.J:
            out["shock_x"] = round(wl.x_lo + (j - 0.5) * dx + dx * (mid - rho[j - 1]) / (rho[j] - rho[j - 1]), 5)
    s.close()
    return out


def end_to_end(s, f, Q, P, wl, args, stream, restore):
    """The timed steps through the public API with host buffers: every step copies its
    input state (f, P) from pinned host memory, runs the same work as the timed step of the
    same index (the defect-correction evaluation every --dc-every steps, one SGS iteration
    with its residual) and reads the residual back; between steps (untimed) the new state
    goes back to the host buffers, so the steps follow the headline pass's iterations from
    the same post-warm-up state (`restore`)."""
    import torch

    from paper_2409_01910_gb300 import sgs

    hf = torch.empty(f.shape, dtype=f.dtype).pin_memory()
    hP = torch.empty(P.shape, dtype=P.dtype).pin_memory()
    hres = torch.zeros(1, dtype=torch.float64).pin_memory()
    res = torch.zeros(1, dtype=torch.float64, device=f.device)

    def step(i):
        f.copy_(hf, non_blocking=True)
        P.copy_(hP, non_blocking=True)
        if i % args.dc_every == 0:
            s.dc_step(f, Q, P, 0, res=res)
        s.iterate(f, Q, P, flags=sgs.IT_P_VALID | sgs.IT_EVAL, res=res)
        hres.copy_(res, non_blocking=True)

    def to_host():
        hf.copy_(f)
        hP.copy_(P)
        torch.cuda.synchronize()

    to_host()
    for i in range(2):  # warm-up of the copies (then back to the post-warm-up state)
        step(args.warmup + i)
        torch.cuda.synchronize()
    restore()
    to_host()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    total = 0.0
    steps = args.steps
    for i in range(steps):
        t0.record(stream)
        step(args.warmup + i)
        t1.record(stream)
        t1.synchronize()
        total += t0.elapsed_time(t1)
        to_host()
    ms = total / steps
    return {"value": visits_per_iteration(wl) / (ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": 2 * hf.numel() * 8,
            "d2h_bytes_per_step": 8, "ms_per_step": ms,
            "note": ("state (f, P) copied from pinned host memory and the residual read back every step, the "
                     "same steps as the timed region from the same post-warm-up state")}


def fp64_form(wl, args, f0, dev, stream):
    import torch

    from paper_2409_01910_gb300 import sgs

    s = make_solver(wl, sgs.FP64)
    f = f0.clone()
    Q, P = s.field(), s.field()
    res = torch.zeros(1, dtype=torch.float64, device=dev)
    s.iterate(f, Q, P, flags=sgs.IT_EVAL, res=res)
    torch.cuda.synchronize()
    s.profile(True)
    s.profile_read()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.fp64_steps):
        s.iterate(f, Q, P, flags=sgs.IT_P_VALID | sgs.IT_EVAL, res=res)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / args.fp64_steps
    prof = s.profile_read()
    s.close()
    return {"value": visits_per_iteration(wl) / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": args.fp64_steps,
            "kernels_ms": {k: round(v[0], 3) for k, v in prof.items()}}


# ------------------------------------------------------------------------------- oracle
def oracle_sample(wl, n_collide_cells=None, n_visits=2):
    """Times the FP64 oracle on a bounded sample of the workload: the collision step of a
    few cells (threads over cells) and a few cell visits. Returns seconds per cell update
    (one cell visit plus one cell's collision evaluation)."""
    from oracle import oracle as O

    O.build()
    cores = os.cpu_count() or 1
    S = n_collide_cells or min(8, cores)
    if is_cavity(wl):
        # the cell solve of a 2-D visit costs what a 1-D one costs on the same velocity grid
        prob = O.Problem(N=wl.N, L=wl.L, J=wl.nx, eps=wl.eps, bc_T=(wl.T_wall, wl.T_wall),
                         total_mass=wl.total_mass)
    elif is_shock(wl):
        (r1, u1, T1), (r2, u2, T2) = wl.up, wl.down
        prob = O.Problem(N=wl.N, L=wl.L, J=wl.J, x_lo=wl.x_lo, x_hi=wl.x_hi, eps=wl.eps, kernel=O.HARD_SPHERE,
                         bc_kind=(O.INFLOW, O.INFLOW), bc_rho=(r1, r2), bc_u=((u1, 0.0, 0.0), (u2, 0.0, 0.0)),
                         bc_T=(T1, T2), total_mass=0.0)
    else:
        prob = O.Problem(N=wl.N, L=wl.L, J=wl.J, eps=wl.eps, bc_T=(wl.T_left, wl.T_right),
                         total_mass=wl.total_mass)
    f = wl.initial_state()
    O.collide(prob, f[:1])  # builds the weight table (not timed)
    t = time.perf_counter()
    Qc, Pc, nu = O.collide(prob, f[:S])
    t_coll = (time.perf_counter() - t) / S
    dx = prob.dx
    V = (np.arange(wl.N) - wl.N // 2 + 1) * (2 * wl.L / wl.N)
    f = f[: max(S, n_visits + 2)]
    vp = np.maximum(V, 0)[:, None, None]
    vm = np.minimum(V, 0)[:, None, None]
    t = time.perf_counter()
    for j in range(1, 1 + n_visits):
        r = (-vp * f[j - 1] + vm * f[j + 1]) / dx - Pc[j] / wl.eps
        O.cell_solve(prob, dx, r, nu[j], f[j])
    t_visit = (time.perf_counter() - t) / n_visits
    return t_coll + t_visit, cores, S, n_visits, t_coll, t_visit


def cpu_baseline(wl):
    sec, cores, S, nv, tc, tv = oracle_sample(wl)
    return {"value": 1.0 / sec, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"FP64 C oracle: collision step of {S} cells (OpenMP over cells, {tc:.2f} s/cell) + "
                       f"{nv} cell visits ({tv:.2f} s/visit) of the same workload; value = 1/(per-cell collision + "
                       f"per-visit time)")}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    wl = workload()
    times = []
    for i in range(args.warmup + args.steps):
        sec, cores, S, nv, tc, tv = oracle_sample(wl, n_visits=1)
        if i >= args.warmup:
            times.append(sec)
    sec = sum(times) / len(times)
    value = 1.0 / sec
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(wl),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "per step: collision step of min(8, cores) cells + 1 cell visit, FP64 C oracle"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_batch(args, rank, world, local):
    """The batch workload: independent heat-transfer problems (cells uniform in 32..256, grid
    24^3 or 32^3, eps log-uniform in [1e-3, 1], seeded walls), one handle and stream per
    velocity grid, one CUDA graph holding a defect-correction cycle of every group (the
    double-float evaluation, deactivation of converged problems, --lo-iters mixed SGS
    iterations). A step is one replay of that graph."""
    import torch

    from paper_2409_01910_gb300 import inputs as I
    from paper_2409_01910_gb300 import sgs

    torch.cuda.set_device(local)
    wls = I.heat_batch(args.batch_size, seed=0)
    probs = [sgs.Problem(nx=w.J, nv=w.N, v_max=w.L, eps=w.eps, bc_T=(w.T_left, w.T_right),
                         total_mass=w.total_mass, precision=sgs.FP32) for w in wls]
    b = sgs.Batch(probs)
    peaks = measure_peaks(wls[0], next(iter(b.solvers.values())).sweep_shape(), local)
    states = [w.initial_state() for w in wls]
    b.load(states)
    tuning = None if args.no_autotune else b.autotune(reps=1)
    b.load(states)  # the autotuner advanced the iterates: start again from the initial states
    cells = sum(w.J for w in wls)
    visits_per_step = 2 * args.lo_iters * cells
    t_cap = time.perf_counter()
    b.capture(args.lo_iters)  # one eager warm-up cycle, then the recorded one
    torch.cuda.synchronize()
    capture_s = time.perf_counter() - t_cap
    for _ in range(max(0, args.warmup - 1)):
        b.step()
    torch.cuda.synchronize()
    rank_barrier(world)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stream = torch.cuda.current_stream()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for i in range(args.steps):
            ev[i][0].record(stream)
            b.step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        rank_barrier(world)
    ms_total = max_over_ranks(sum(a.elapsed_time(c) for a, c in ev), world, torch.device("cuda", local))
    res = b.residuals()
    # per-kernel timings and launch count of one eager cycle (a replay runs exactly the
    # kernels the captured cycle enqueued; replays themselves are not profiled), every
    # instance active so that every cell is evaluated
    for s in b.solvers.values():
        s.activate_all()
        s.profile(True)
        s.profile_read()
    launches0 = sum(s.launch_count() for s in b.solvers.values())
    b._cycle(args.lo_iters, 0.0)
    torch.cuda.synchronize()
    launches_per_cycle = sum(s.launch_count() for s in b.solvers.values()) - launches0
    prof = {}
    flops = 0.0
    for nv, s in b.solvers.items():
        for k, (ms, n, done) in s.profile_read(with_work=True).items():
            a = prof.setdefault(k, [0.0, 0])
            a[0] += ms
            a[1] += n
            if k == "sum":
                # FP32 spectral sums: 10 flops per mode pair over the Hermitian half per cell
                flops += 10 * 0.5 * pairs_per_cell(nv) * done
        s.profile(False)
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    ach = flops / (prof["sum"][0] * 1e-3) / 1e12 if prof["sum"][0] else None
    peak = peaks["fp32_ffma_tflops"]
    roof = {"kernel": "k_sum<float> (direct spectral sum, FP32), all groups", "bound": "alu", "achieved": ach,
            "peak": peak, "unit": "TFLOP/s", "frac": ach / peak if ach else None, "traffic": None,
            "peak_source": f"FFMA rate measured by sgs_peak_fma on {peaks['sms']} SMs (of measured)",
            "from": "one eager cycle (graph replays are not profiled)"}
    shapes = {str(nv): dict(zip(("nodes_per_thread", "ctas_per_cluster", "threads_per_cta"), s.sweep_shape()))
              for nv, s in b.solvers.items()}
    # end to end: states copied in from pinned host memory, one replay, residuals read back
    hostf = {nv: b.f[nv].cpu().pin_memory() for nv in b.groups}
    hostP = {nv: b.P[nv].cpu().pin_memory() for nv in b.groups}
    hres = {nv: torch.zeros(len(idx), dtype=torch.float64).pin_memory() for nv, idx in b.groups.items()}
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_ms = 0.0
    for i in range(args.steps):
        t0.record(stream)
        for nv in b.groups:
            b.f[nv].copy_(hostf[nv], non_blocking=True)
            b.P[nv].copy_(hostP[nv], non_blocking=True)
        b.step()
        for nv in b.groups:
            hres[nv].copy_(b.res[nv], non_blocking=True)
        t1.record(stream)
        t1.synchronize()
        e2e_ms += t0.elapsed_time(t1)
    e2e_ms /= args.steps
    h2d = sum(2 * hostf[nv].numel() * 8 for nv in b.groups)
    d2h = sum(hres[nv].numel() * 8 for nv in b.groups)
    # time from the initial states until each instance's FP64 residual falls below 1e-8
    t2tol = None
    if args.batch_t2tol_cap > 0:
        b.load(states)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reached = [None] * len(probs)
        cycles = 0
        while time.perf_counter() - t0 < args.batch_t2tol_cap:
            b.step()
            cycles += 1
            rr = b.residuals()  # the evaluation at the start of this cycle (synchronises)
            t = time.perf_counter() - t0
            for i, r in enumerate(rr):
                if reached[i] is None and r < 1e-8:
                    reached[i] = round(t, 2)
            if all(x is not None for x in reached):
                break
        done = [x for x in reached if x is not None]
        t2tol = {"converged": len(done), "of": len(probs), "cycles": cycles, "lo_iters": args.lo_iters,
                 "seconds_all": max(done) if len(done) == len(probs) else None, "cap_s": args.batch_t2tol_cap,
                 "per_instance_s": reached,
                 "per_instance": [{"J": w.J, "N": w.N, "eps": round(w.eps, 5)} for w in wls]}
    out = {
        "metric": METRIC, "value": whole_job_rate(visits_per_step * args.steps, world, ms_total), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"heat1d_batch{args.batch_size}", "instances": args.batch_size, "cells": cells,
                   "grids": {str(nv): len(idx) for nv, idx in b.groups.items()},
                   "cells_per_grid": {str(nv): sum(probs[i].nx for i in idx) for nv, idx in b.groups.items()},
                   "eps_range": [min(w.eps for w in wls), max(w.eps for w in wls)],
                   "step": f"one CUDA-graph replay: defect-correction cycle with {args.lo_iters} SGS iterations",
                   "l2": "inputs (GBs of state) larger than L2", "parallelism": f"replicas x{world}",
                   "capture_s": round(capture_s, 2)},
        "roofline": roof,
        "scan_shape_per_grid": shapes, "autotune": tuning,
        "kernels_ms_eager_cycle": {k: round(v[0], 3) for k, v in prof.items()},
        "e2e": {"value": visits_per_step / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "note": "every group's (f, P) copied from pinned host memory, one replay, residuals read back"},
        "clocks": clocks, "gpu_launches": int(launches_per_cycle * args.steps), "measured_peaks": peaks,
        "residuals_after": {"max": max(res), "converged_1e-8": int(sum(r < 1e-8 for r in res))},
        "time_to_residual_1e-8": t2tol,
        "device_status": b.status(),
    }
    return out


# The computing times the paper reports for its 2-D BGK cavity (1st and 2nd order; seconds to
# an outer residual of 1e-5, hardware not stated; None: stopped after 48 hours), for context.
PAPER_BGK_CAVITY_S = {
    (1, "sgs_fp"): [2461.28, 18921.84, 162168.90, None, None],
    (1, "sgs_pfp"): [1876.55, 4684.12, 6144.21, 5490.00, 5502.58],
    (1, "mg_sgs_pfp"): [425.06, 1030.87, 1090.24, 971.69, 945.81],
    (2, "sgs_pfp"): [2934.51, 9504.34, 40256.89, 171357.22, None],
    (2, "mg_sgs_pfp"): [2255.97, 1542.45, 6122.38, 30216.12, 67737.60],
}
PAPER_EPS = [1.0, 0.1, 0.01, 1e-3, 1e-4]


def run_paper_cavity(args, local):
    """The paper's 2-D BGK heat-transfer cavity (40 x 40 cells, 20^3 velocities on [-6, 6]^3,
    top wall at T = 2, nu = 4 pi rho) timed on the GPU in FP64 to an outer residual of 1e-5
    (inner tolerance 1e-8), for each method and order of the paper's table: SGS-FP,
    SGS-PFP and MG-SGS-PFP (V-cycles down to 5 x 5 cells, 1 + 1 smoothing iterations at first
    order, 5 + 1 at second order, 10 iterations on the coarsest grid). Each run is capped at
    --t2tol-cap seconds. One JSON line with the table and the paper's times beside it."""
    import torch

    from paper_2409_01910_gb300 import inputs as I
    from paper_2409_01910_gb300 import sgs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    eps_list = [float(x) for x in args.paper_eps.split(",")]
    rows = []
    t_start = time.perf_counter()
    for order, method in PAPER_BGK_CAVITY_S:
        for eps in eps_list:
            wl = I.cavity_heat_bgk_40x40_20v(eps)
            p = sgs.Problem(space_dim=2, nx=wl.nx, ny=wl.ny, x_lo=-0.5, x_hi=0.5, y_lo=-0.5, y_hi=0.5, nv=wl.N,
                            v_max=wl.L, collision=sgs.BGK, b0=wl.b0, eps=eps, bc_T=(wl.T_wall, wl.T_wall),
                            bc_T_y=(wl.T_wall, wl.T_top), total_mass=wl.total_mass, precision=sgs.FP64,
                            inner_tol=1e-8, order=order, inner_method=sgs.FP if method == "sgs_fp" else sgs.PFP)
            s = sgs.Solver(p)
            f = torch.from_numpy(wl.initial_state().reshape(-1)).to(dev)
            Q, P = s.field(), s.field()
            res = torch.zeros(1, dtype=torch.float64, device=dev)
            levels = min(4, s.max_levels())
            pre = 1 if order == 1 else 5
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r, iters, reached = float("nan"), 0, False
            while time.perf_counter() - t0 < args.t2tol_cap:
                if method == "mg_sgs_pfp":
                    s.collide(f, Q, P)
                    s.residual(f, Q, res)
                else:
                    s.iterate(f, Q, P, flags=sgs.IT_EVAL | (sgs.IT_P_VALID if iters else 0), res=res)
                    iters += 1
                r = float(res.item())
                if r < wl.tol or r != r:
                    reached = r < wl.tol
                    break
                if method == "mg_sgs_pfp":
                    s.vcycle(f, levels, pre, 1, 10)
                    iters += 1
            sec = time.perf_counter() - t0
            st = s.read_status()
            paper = PAPER_BGK_CAVITY_S[(order, method)][PAPER_EPS.index(eps)] if eps in PAPER_EPS else None
            rows.append({"order": order, "method": method, "eps": eps, "seconds": round(sec, 3), "reached": reached,
                         "residual": r, ("V-cycles" if method.startswith("mg") else "SGS iterations"): iters,
                         "inner_iters_per_visit": round(st["inner_iters"] / max(1, st["visits"]), 3),
                         "status": st["status"], "paper_s": paper})
            s.close()
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    return {"metric": "seconds to outer residual 1e-5 (the paper's 2-D BGK cavity)", "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "cavity2d_heat_bgk_40x40_N20", "cells": [40, 40], "domain": [[-0.5, 0.5], [-0.5, 0.5]],
                       "nv": 20, "v_max": 6.0, "collision": "BGK, nu = 4 pi rho", "T_walls": "top 2, others 1",
                       "tol": 1e-5, "inner_tol": 1e-8, "cap_s": args.t2tol_cap, "multigrid": "4 levels (40^2 .. 5^2)"},
            "table": rows, "total_s": round(time.perf_counter() - t_start, 1),
            "paper_note": "paper_s: the paper's computing time for the same problem, method, order and eps "
                          "(hardware not stated)"}


def profile_case(which):
    """Small instance of one kernel class for ncu: the persistent scan on 4 cells, or the
    spectral sum on 32 cells (one lane group), both on the 32^3 grid of the workload; or
    one 2-D scan ordering of an 8 x 8 cavity on the 24^3 grid of the cavity workload."""
    import torch

    from paper_2409_01910_gb300 import inputs as I
    from paper_2409_01910_gb300 import sgs

    if which == "fast":
        # the fast spectral operator (hard spheres, tensor cores) on 64 cells of the shock's
        # 32^3 grid on [-10, 10]^3: one evaluation after a warm-up one
        J, N, L = 64, 32, 10.0
        # FP32 handle: its direct FP32 sum is the comparison (the fast operator ignores the
        # handle's precision)
        s = sgs.Solver(sgs.Problem(nx=J, nv=N, v_max=L, collision=sgs.HARD_SPHERE, eps=0.1, precision=sgs.FP32))
        fast = sgs.FastOperator(s, 8, 16, chunk=8)
        f = torch.from_numpy(I.initial_state(J, N, L, T=1.5).reshape(-1)).cuda()
        Q, P = s.field(), s.field()
        out = {"case": which, "cells": J, "nv": N, "v_max": L, "nodes": "8 x 16 + loss slot", "chunk": 8}
        runs = (("fast_terms3", lambda: fast.collide(f, Q, terms=3)), ("fast_terms1", lambda: fast.collide(f, Q, terms=1)),
                ("direct_fp32", lambda: s.collide(f, Q, P)))
        for name, fn in runs:
            fn()  # warm-up (the first fast evaluation is the one ncu skips past)
            torch.cuda.synchronize()
            s.profile(True)
            s.profile_read()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                fn()
            e1.record()
            torch.cuda.synchronize()
            prof = s.profile_read()
            s.profile(False)
            out[name] = {"ms": round(e0.elapsed_time(e1) / 3, 3),
                         "classes_ms": {k: round(v[0] / 3, 3) for k, v in prof.items() if v[0] > 0}}
        out["status"] = s.read_status()["status"]
        print(json.dumps(out))
        return
    if which == "steps":
        # the benchmark's step on the 64-cell heat workload: one defect-correction evaluation,
        # then three pipelined SGS iterations with their evaluation (the launch list's case)
        wl = I.heat_64cells_32v()
        s = make_solver(wl, sgs.FP32)
        f = torch.from_numpy(wl.initial_state().reshape(-1)).cuda()
        Q, P = s.field(), s.field()
        res = torch.zeros(1, dtype=torch.float64, device="cuda")
        s.dc_step(f, Q, P, 0, res=res)
        for _ in range(3):
            s.iterate(f, Q, P, flags=sgs.IT_P_VALID | sgs.IT_EVAL, res=res)
        torch.cuda.synchronize()
        print(json.dumps({"case": which, "status": s.read_status(), "launches": s.launch_count(),
                          "pipelined": s.overlap()}))
        return
    if which == "peaks":
        wl = I.heat_64cells_32v()
        s = make_solver(wl, sgs.FP32)
        print(json.dumps({"case": which, "peaks": measure_peaks(wl, s.sweep_shape())}))
        return
    if which == "dft":
        # the transforms of the mixed solver's increment-form collision on the 64-cell workload
        wl = I.heat_64cells_32v()
        s = make_solver(wl, sgs.FP32)
        f = torch.from_numpy(wl.initial_state().reshape(-1)).cuda()
        Q, P = s.field(), s.field()
        s.dc_step(f, Q, P, 0)
        s.collide(f, Q, P)
        torch.cuda.synchronize()
        print(json.dumps({"case": which, "status": s.read_status()}))
        return
    if which == "sweep2d":
        w = I.CavityWorkload("cavity2d_8x8_N24", nx=8, ny=8, N=24, L=6.0, eps=0.05)
        s = make_solver(w, sgs.FP32)
        f = torch.from_numpy(w.initial_state().reshape(-1)).cuda()
        Q, P = s.field(), s.field()
        s.collide(f, Q, P)
        s.sweep_ordering(f, P, 0)
        torch.cuda.synchronize()
        print(json.dumps({"case": which, "status": s.read_status()}))
        return

    J = 4 if which == "sweep" else 32
    p = sgs.Problem(nx=J, nv=32, v_max=8.0, eps=0.01, bc_T=(1.0, 1.8), total_mass=1.0,
                    precision=sgs.FP64 if which == "sum64" else sgs.FP32)
    s = sgs.Solver(p)
    f = torch.from_numpy(I.initial_state(J, 32, 8.0, T=1.4).reshape(-1)).cuda()
    Q, P = s.field(), s.field()
    s.collide(f, Q, P)
    for _ in range(2):
        if which == "sweep":
            g = f.clone()
            s.sweep_forward(g, P)
        elif which == "sumdf":
            s.collide(f, Q, P, precision=sgs.DF64)
        else:
            s.collide(f, Q, P)
    torch.cuda.synchronize()
    print(json.dumps({"case": which, "status": s.read_status()}))


def main():
    global WORKLOAD, CONSERVE_PROJ, PIN_MASS, ORDER
    args = parse()
    WORKLOAD = args.workload
    CONSERVE_PROJ = args.conserve_proj
    PIN_MASS = args.pin_mass
    ORDER = args.order
    if args.case:
        profile_case(args.case)
        return
    rank, world, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    import torch

    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload == "paper_bgk_cavity":
        if rank == 0:
            print(json.dumps(run_paper_cavity(args, local)), flush=True)
        return
    out = (run_batch if args.workload == "batch" else run_native)(args, rank, world, local)
    if rank == 0:
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(workload())
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
