#!/usr/bin/env python
"""Throughput of the LODIE2 RE+V solve on GB300 (LOD Mpoint-steps/s).

Workload (default): the largest single solve, the 20,000-atom random-walk molecule on a 257^3 grid
at h = 0.5 A, eps 1/80, kbar^2 = 0.84 A^-2, LODIE2 with dt = 0.4, alpha = 1/25, 40 steps,
Richardson extrapolation (dt/2 leg: 80 steps) and the LOD vacuum legs: 255^3 x 240 interior
point-steps per solve.  Sweeps in FP32, combination and energy in FP64; the plain FP64 path is
timed beside it, and both are compared with the FP64 oracle on the same molecule.

One "step" is one complete solve of that molecule with its atoms resident in HBM: the set-up
kernels (mask, charge list, face data), the four legs, and the energy reduction with its 8-byte
read-back.  Steps are timed with CUDA events on the solver's stream; the four leg states (4 x 68
MB) exceed L2, and a 256 MB write precedes every step, outside the event pair.

Beside the headline: the sweep roofline (each direction's launches timed as the solve issues
them), the protein_1k configuration (129^3), the batched workload (64 molecules), the Poisson
serving stream against the plain FP64 path served FIFO, end-to-end timing from pinned host
arrays, and the oracle on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload W]
Under torchrun (N > 1) every rank solves its own copy (weak scaling, no collective on
the data path); rank 0 prints the line with the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LOD Mpoint-steps/s"
UNIT = "Mpoint-steps/s"
DT, ALPHA, NSTEPS = 0.4, 1.0 / 25.0, 25


def workload(name: str):
    import npb_inputs as I

    if name == "protein_1k":
        return I.protein_1k(), dict(dt=DT, alpha=ALPHA, n=NSTEPS)
    if name == "large_20k":
        return I.large_20k(), dict(dt=DT, alpha=ALPHA, n=40)
    if name == "born":
        return I.born_sphere(0.84), dict(dt=0.1, alpha=1.0, n=200)
    raise SystemExit(f"unknown workload {name}")


def point_steps(problem, n: int) -> int:
    nx, ny, nz = problem.n
    return (nx - 2) * (ny - 2) * (nz - 2) * n * 6  # (n + 2n) steps x 2 media


def workload_config(args, problem, w) -> dict:
    """The workload part of the JSON line's config, the same for both arms."""
    nx, ny, nz = problem.n
    return {"workload": f"{args.workload} (LODIE2 RE+V, {nx}x{ny}x{nz}, {problem.n_atoms} atoms, "
                        f"dt={w['dt']}, alpha={w['alpha']:.4g}, {w['n']}+{2 * w['n']} steps x 2 media)",
            "grid": [nx, ny, nz], "atoms": problem.n_atoms, "energy_dtype": "f64",
            "point_steps_per_step": point_steps(problem, w["n"])}


# ----------------------------------------------------------------------------- distributed
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(local_seconds: float, local_units: float, world: int, group=None):
    """Job-level (max seconds over ranks, total units over ranks) for weak-scaled ranks."""
    if world <= 1:
        return local_seconds, local_units
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([local_seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([local_units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), float(u.item())


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock and throttle-reason samples every 20 ms, time-stamped on the host.  Started
    before the warm-up so that the sampler is running when the timed region begins; `stop` keeps
    the samples inside the timed window (`mark_start`/`mark_end`), or the two that bracket it when
    the window is shorter than the sampling period."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.samples = []
        self.t0 = self.t1 = None

    def start(self):
        import threading

        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "20",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, bufsize=1)
        except (OSError, FileNotFoundError):
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                self.samples.append((time.perf_counter(), line))

        self.th = threading.Thread(target=reader, daemon=True)
        self.th.start()

    def mark_start(self):
        self.t0 = time.perf_counter()

    def mark_end(self):
        self.t1 = time.perf_counter()

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.05)  # one more sample after the window
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        rows = []
        for t, line in self.samples:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((t, float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        t0 = self.t0 if self.t0 is not None else rows[0][0]
        t1 = self.t1 if self.t1 is not None else rows[-1][0]
        inside = [r for r in rows if t0 <= r[0] <= t1]
        window = "inside the timed region"
        if not inside:  # the region is shorter than the sampling period: the bracketing samples
            before = [r for r in rows if r[0] < t0][-1:]
            after = [r for r in rows if r[0] > t1][:1]
            inside = before + after
            window = "bracketing the timed region"
        reasons = set()
        for r in inside:
            for nm, v in zip(self.NAMES, r[3]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": sorted(reasons), "samples": len(inside), "window": window,
                "timed_region_s": round(t1 - t0, 4)}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle (plain FP64 C, OpenMP over lines) on the host cores, same metric.  Small workloads:
    one full RE+V solve (set-up included) per step.  large_20k, whose oracle set-up alone takes about
    ten seconds: the set-up runs once before the steps, and each step is one LOD step of both dt legs
    and two of both dt/2 legs (a bounded sample of the solve's stepping; the set-up is left out, which
    favours the oracle)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    problem, w = workload(args.workload)
    n = w["n"]
    tau = w["dt"] / w["alpha"]
    nx, ny, nz = problem.n
    if args.workload == "large_20k":
        st = {m: oracle.setup(problem, m) for m in (oracle.SOLVENT, oracle.VACUUM)}
        legs = {(m, half): st[m].u0.copy() for m in st for half in (0, 1)}

        def one():
            for (m, half), u in legs.items():
                oracle.lod_run(u, st[m], tau * (0.5 if half else 1.0), problem.h, 2 if half else 1)

        units = (nx - 2) * (ny - 2) * (nz - 2) * 6
        sample = (f"{args.workload}: set-up once, then per step 1 LOD step of both dt legs and 2 of both "
                  f"dt/2 legs (6 of the solve's {6 * n} leg-steps), set-up excluded")
    else:
        def one():
            oracle.energy(problem, tau, n)

        units = point_steps(problem, n)
        sample = f"{args.workload}: one full RE+V solve per step, set-up included"
    for _ in range(args.warmup):
        one()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        one()
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = units * args.steps / total / 1e6
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": dict(workload_config(args, problem, w), l2="host run (no device cache)",
                           step="a bounded sample of the oracle's RE+V solve (see cpu_baseline.sample)",
                           parallelism=f"{cores} host threads"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- our arm
def cpu_baseline(problem, w, full_solve_s: float | None = None, budget_s: float = 12.0):
    """The oracle (plain FP64 C, OpenMP over lines) on the host cores: all cores on the full RE+V
    solve when `full_solve_s` (its time, set-up included) is given, else on a bounded sample of
    it; and one thread on one LOD step of the solvent leg (set-up excluded)."""
    import oracle

    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    cores = oracle.get_threads()
    n = w["n"]
    if full_solve_s is not None:
        n_s, reps, el = n, 1, full_solve_s
    else:
        est_rate = 8e7 * cores  # conservative oracle point-steps/s
        n_s = n
        while n_s > 1 and point_steps(problem, n_s) / est_rate > budget_s:
            n_s = max(1, n_s // 2)
        t0 = time.perf_counter()
        reps = 0
        while True:
            oracle.energy(problem, w["dt"] / w["alpha"], n_s)
            reps += 1
            el = time.perf_counter() - t0
            if el > budget_s / 2 or reps >= 3:
                break
    value = point_steps(problem, n_s) * reps / el / 1e6
    st = oracle.setup(problem, oracle.SOLVENT)
    u = st.u0.copy()
    oracle.set_threads(1)
    t1 = time.perf_counter()
    oracle.lod_run(u, st, w["dt"] / w["alpha"], problem.h, 1)
    t1 = time.perf_counter() - t1
    oracle.set_threads(cores)
    nx, ny, nz = problem.n
    single = (nx - 2) * (ny - 2) * (nz - 2) / t1 / 1e6
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{reps} full RE+V solve(s) of the same molecule with {n_s} steps per dt leg, set-up included",
            "single_thread": {"value": single, "unit": UNIT,
                              "sample": "1 LOD step of the solvent leg on 1 thread, set-up excluded"},
            "cpu_model": cpu_model()}


def cpu_model() -> str:
    """The host CPU's model name (Linux /proc/cpuinfo; Arm boards report implementer/part)."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return platform.processor() or platform.machine()
    for key in ("model name", "Model", "Hardware"):
        for line in info:
            if line.split(":")[0].strip() == key:
                return line.split(":", 1)[1].strip()
    imp = [l.split(":", 1)[1].strip() for l in info if l.startswith("CPU implementer")]
    part = [l.split(":", 1)[1].strip() for l in info if l.startswith("CPU part")]
    return f"{platform.machine()} implementer {imp[0] if imp else '?'} part {part[0] if part else '?'}"


def batch_run(npb, count: int, reps: int = 3, tune: bool = True):
    """The batched workload: `count` seeded random-walk molecules of 200-5,000 atoms (log-uniform),
    grids 65^3-161^3 by the grid-size rule, RE+V with FP32 sweeps and FP64 energies.  Times
    npb_energy_batch (equal-size grids share persistent launches; one CUDA graph per batch) against
    the same grids solved one npb_energy call at a time, both after a warm-up call, with L2 flushed
    before every timed call (CUDA events on the context's stream)."""
    import torch

    import npb_inputs as I

    mols = I.batch_molecules(count)
    ctx = npb.npb_ctx_create(0, 0)
    stream = torch.cuda.Stream()
    npb.npb_ctx_set_stream(ctx, stream.cuda_stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    try:
        grids = [npb.npb_grid_create(ctx, p) for p in mols]
        o32 = npb.make_opts(DT, ALPHA, NSTEPS, precision=npb.NPB_FP32_SWEEP)
        pts = sum((p.n[0] - 2) * (p.n[1] - 2) * (p.n[2] - 2) for p in mols) * 6 * NSTEPS
        # the autotuner picks the line solver per (direction, grid size) on one grid of each size
        tuned = {}
        for p, g in zip(mols, grids):
            if tune and p.n[0] not in tuned:
                npb.npb_autotune(g, o32, reps=3)
                tuned[p.n[0]] = {("x", "y", "z")[d]: npb.npb_tune_get(ctx, npb.NPB_FP32_SWEEP, d, p.n[d])
                                 for d in range(3)}

        def timed(fn):
            ms = []
            with torch.cuda.stream(stream):
                fn()
                for _ in range(reps):
                    flush.zero_()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    fn()
                    b.record(stream)
                    torch.cuda.synchronize()
                    ms.append(a.elapsed_time(b))
            return sorted(ms)[len(ms) // 2]

        out_b = []
        t_batch = timed(lambda: out_b.append(npb.npb_energy_batch(grids, o32)))
        out_s = []
        t_seq = timed(lambda: out_s.append([npb.npb_energy(g, o32) for g in grids]))
        for g in grids:
            npb.npb_grid_destroy(g)
    finally:
        npb.npb_ctx_destroy(ctx)
    sizes = sorted({p.n[0] for p in mols})
    return {"molecules": count, "grids": sizes, "atoms": [min(p.n_atoms for p in mols), max(p.n_atoms for p in mols)],
            "point_steps": pts, "ms_batch": t_batch, "Mpoint_steps_per_s": pts / t_batch / 1e3,
            "solves_per_s": count / t_batch * 1e3, "ms_one_at_a_time": t_seq,
            "one_at_a_time_Mpoint_steps_per_s": pts / t_seq / 1e3,
            "same_results": bool(out_b[-1] == out_s[-1]),
            "tuned_shapes": {str(k): v for k, v in tuned.items()},
            "alg_gbs": 24 * pts / t_batch / 1e6, "frac_of_peak": 24 * pts / t_batch / 1e6 / measured_peaks()[0],
            "note": "median of %d calls; equal-size grids share one launch per direction per step" % reps}


def serving_run(npb, seconds: float, rate: float = 50.0, fifo_requests: int = 50):
    """Poisson arrivals (seeded stream of random-walk molecules, 100-20,000 atoms, h 0.25/0.5 A)
    through npb_submit/npb_poll with continuous batching, FP32 sweeps; then the first
    `fifo_requests` of the same stream through the plain FP64 single-solve path, one at a time
    in arrival order, with the same arrival times."""
    import threading

    import numpy as np

    import npb_inputs as I

    count = max(1, int(round(seconds * rate)))
    stream = list(I.serving_stream(count, rate_hz=rate))
    o32 = npb.make_opts(DT, ALPHA, NSTEPS, precision=npb.NPB_FP32_SWEEP)
    ctx = npb.npb_ctx_create(0, 0)
    tickets = [None] * count
    t0 = time.perf_counter()

    def submitter():
        for i, (ta, p) in enumerate(stream):
            dt = t0 + ta - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets[i] = npb.npb_submit(ctx, p, o32)

    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    res = [npb.npb_poll(ctx, t, 600000) for t in tickets]
    elapsed = time.perf_counter() - t0
    npb.npb_ctx_destroy(ctx)
    ok = [r for r in res if r.status == npb.NPB_OK]
    lat = np.array([r.wall_ms for r in ok])
    pts = sum(r.point_steps for r in ok)
    out = {"requests": count, "completed": len(ok), "rate_hz": rate, "seconds": elapsed,
           "solves_per_s": len(ok) / elapsed, "Mpoint_steps_per_s": pts / elapsed / 1e6,
           "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
           "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
           "grids": sorted({int(r.n[0]) for r in ok}), "precision": "f32 sweeps, f64 energy"}
    # the plain FP64 path, FIFO, on the first requests of the same stream
    k = min(fifo_requests, count)
    o64 = npb.make_opts(DT, ALPHA, NSTEPS, precision=npb.NPB_FP64)
    ctx = npb.npb_ctx_create(0, 0)
    lat64, dg64 = [], []
    tf = time.perf_counter()
    for i in range(k):
        ta, p = stream[i]
        now = time.perf_counter() - tf
        if now < ta:
            time.sleep(ta - now)
        g = npb.npb_grid_create(ctx, p)
        dg64.append(npb.npb_energy(g, o64))
        npb.npb_grid_destroy(g)
        lat64.append((time.perf_counter() - tf - ta) * 1e3)
    el64 = time.perf_counter() - tf
    npb.npb_ctx_destroy(ctx)
    out["fp64_fifo"] = {"requests": k, "solves_per_s": k / el64, "p50_ms": float(np.percentile(lat64, 50)),
                        "p99_ms": float(np.percentile(lat64, 99)),
                        "note": "plain FP64 single-solve path, one request at a time in arrival order, "
                                "the first %d requests of the same stream at their arrival times" % k}
    # each served FP32-sweep result against the FP64 path's (which equals the oracle to 1e-10)
    rel = [abs(res[i].dG_kcal_mol - dg64[i]) / abs(dg64[i]) for i in range(k)
           if res[i].status == npb.NPB_OK and dg64[i] != 0.0]
    out["dG_rel_error_fp32_vs_fp64"] = {"requests": len(rel), "max": max(rel) if rel else None,
                                        "median": float(np.median(rel)) if rel else None,
                                        "per_request": [float("%.3g" % r) for r in rel]}
    return out


# The sources of the FP32 interior-row sweeps (the kernels whose DRAM traffic profiles/ncu_traffic.json
# records) and of the FP64 line sweeps.
FP32_SWEEP_SOURCES = ("sweep_kernel.cuh", "sweep_tma.cuh", "sweep_inner.cuh", "sweep_inner_launch.cuh", "f32x2.cuh")
FP64_SWEEP_SOURCES = ("sweep_kernel.cuh", "sweep_line64.cu")


def _kernel_source_hash(files=FP32_SWEEP_SOURCES) -> str:
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_1410_2788_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def roofline_traffic(kernel: str, workload: str):
    """ncu DRAM bytes per launch, if a capture of the current kernel source is on file."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    e = d.get(f"{workload}/{kernel}")
    if not e or e.get("source_hash") != _kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


def fp64_roofline(point_steps_per_s, dfma_per_s, ddiv_per_s, peak, peak_kind):
    """The plain FP64 path's sweeps against HBM: the FP64 Thomas-per-line kernel moves 48 B per
    interior node per sweep (u read and written, the forward result written and read back, the
    precomputed multiplier read on the way down and on the way up), 144 B per point-step.  The whole
    step is timed, set-up (the FP64 faces) included, so the fraction understates the sweeps' own.  The
    FP64 units' measured rates (npb_measure_fp64) and, when profiles/ncu_fp64_ops.json matches the
    kernel source, the FP64 operations per point-step counted by ncu go beside it."""
    ach = 144.0 * point_steps_per_s / 1e9
    out = {"bound": "hbm", "unit": "GB/s", "achieved": ach, "peak": peak, "frac": ach / peak,
           "peak_source": peak_kind, "alg_bytes_per_point_step": 144,
           "measured_fp64_fma_per_s": dfma_per_s, "measured_fp64_div_per_s": ddiv_per_s}
    path = os.path.join(ROOT, "profiles", "ncu_fp64_ops.json")
    e = json.load(open(path)).get("protein_1k") if os.path.exists(path) else None
    if e and e.get("source_hash") == _kernel_source_hash(FP64_SWEEP_SOURCES):
        flops = sum(e["flops_per_node_sweep"].values())
        out["fp64"] = {"flops_per_point_step": flops, "achieved_gflops": flops * point_steps_per_s / 1e9,
                       "peak_gflops": 2 * dfma_per_s / 1e9, "frac": flops * point_steps_per_s / (2 * dfma_per_s),
                       "fp64_pipe_busy_ncu": e.get("fp64_pipe_busy")}
    return out


def sweep_roofline(npb, grid, opts, problem, w, elem, peak, peak_kind, workload_name):
    """The dominant sweep kernel against the HBM roofline, timed the way the solve runs it: each
    direction's 4-leg and 2-leg launches as graph-captured back-to-back launches (CUDA events on
    the solver's stream), with the solve's shapes and fused stages.  Per 4-leg launch the
    algorithmic bytes are 2 * elem * (interior nodes) * 4 legs (read + write of every interior
    node of every leg); the mask (1/8 B per node) and the charge entries are left out."""
    nx, ny, nz = problem.n
    interior = (nx - 2) * (ny - 2) * (nz - 2)
    names = ("sweep_x", "sweep_y", "sweep_z")
    t = {}
    for d in range(3):
        t[names[d]] = {4: npb.npb_sweep_time(grid, opts, d, 4), 2: npb.npb_sweep_time(grid, opts, d, 2)}
    n = w["n"]
    per_step = {k: n * (v[4] + v[2]) for k, v in t.items()}  # ms of each direction in one solve
    dom = max(per_step, key=per_step.get)
    alg4 = 2 * elem * interior * 4
    ms4 = t[dom][4]
    achieved = alg4 / (ms4 * 1e-3) / 1e9
    per_dir = {k: {"ms_4_legs": v[4], "ms_2_legs": v[2],
                   "achieved_gbs_4_legs": alg4 / (v[4] * 1e-3) / 1e9,
                   "frac_4_legs": alg4 / (v[4] * 1e-3) / 1e9 / peak} for k, v in t.items()}
    return {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_kind,
            "traffic": roofline_traffic(dom, workload_name),
            "launch": f"4 legs x {nx - 2}x{ny - 2}x{nz - 2} interior nodes, {alg4 / 1e6:.1f} MB algorithmic",
            "avg_launch_ms": ms4,
            "timing": "graph of 8 back-to-back launches replayed 5x, CUDA events on the solver stream",
            "per_direction": per_dir, "sweeps_ms_per_solve": sum(per_step.values())}


def fp32_errors(npb, grid, problem, shape):
    """The FP32-sweep legs of the last solve, read back for the comparison with the oracle."""
    return {leg: npb.npb_potential(grid, leg, shape) for leg in range(4)}


def error_report(legs32, dg32, dg64, problem, w):
    """FP32-sweep path and plain FP64 path against the FP64 oracle on the same molecule: the oracle
    solve of the CPU baseline (full RE+V), its dG and its four legs."""
    import numpy as np

    import oracle

    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    t0 = time.perf_counter()
    ref_dg, ref_legs, st = oracle.energy(problem, w["dt"] / w["alpha"], w["n"], return_legs=True)
    el = time.perf_counter() - t0
    names = {0: "solvent_tau", 1: "solvent_half", 2: "vacuum_tau", 3: "vacuum_half"}
    rep = {"dG_oracle": ref_dg, "dG_fp32_rel": abs(dg32 - ref_dg) / abs(ref_dg),
           "dG_fp64_rel": abs(dg64 - ref_dg) / abs(ref_dg), "legs": {}}
    charge = st.qt != 0
    for leg, got in legs32.items():
        ref = ref_legs[names[leg]]
        diff = np.abs(got - ref)
        rep["legs"][names[leg]] = {"linf_rel": float(diff.max() / np.abs(ref).max()),
                                   "abs_max_at_charge_nodes": float(diff[charge].max()),
                                   "abs_max_elsewhere": float(diff[~charge].max())}
    return rep, el, ref_dg


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_1410_2788_gb300 as npb
    from paper_1410_2788_gb300 import build

    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    npb.load_library()

    problem, w = workload(args.workload)
    units_per_step = point_steps(problem, w["n"])
    prec = npb.NPB_FP32_SWEEP if args.precision == "fp32" else npb.NPB_FP64
    stream = torch.cuda.Stream()
    ctx = npb.npb_ctx_create(local, 0)
    npb.npb_ctx_set_stream(ctx, stream.cuda_stream)
    grid = npb.npb_grid_create(ctx, problem)
    opts = npb.make_opts(w["dt"], w["alpha"], w["n"], precision=prec)
    opts64 = npb.make_opts(w["dt"], w["alpha"], w["n"], precision=npb.NPB_FP64)
    tuning = npb.npb_autotune(grid, opts, reps=5) if args.autotune else []
    shapes = {("x", "y", "z")[d]: dict(zip(("kind", "tx", "seg", "len"), npb.npb_tune_get(ctx, prec, d, problem.n[d])))
              for d in range(3)}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step(o):
        npb.npb_grid_refresh(grid)
        return npb.npb_energy(grid, o)

    def timed(o, k):
        ms = []
        dg = None
        with torch.cuda.stream(stream):
            for _ in range(k):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                dg = step(o)
                b.record(stream)
                ms.append((a, b))
            torch.cuda.synchronize()
        return [x.elapsed_time(y) for x, y in ms], dg

    clocks = ClockSampler(local)
    clocks.start()  # running before the timed region begins
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            step(opts)
        step(opts64)
    torch.cuda.synchronize()

    # ---- headline: K steps of the FP32-sweep path
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark_start()
    wall0 = time.perf_counter()
    step_ms, dg = timed(opts, args.steps)
    wall = time.perf_counter() - wall0
    torch.cuda.synchronize()
    clocks.mark_end()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    total_s, total_units = aggregate(sum(step_ms) / 1e3, units_per_step * args.steps, world)
    value = total_units / total_s / 1e6
    ms_per_step = 1e3 * total_s / args.steps
    want_errors = world == 1 and rank == 0 and args.cpu_baseline
    legs32 = fp32_errors(npb, grid, problem, npb.grid_shape(problem)) if want_errors else None

    # ---- the plain FP64 path on the same molecule, and the FP64 units' measured rates
    k64 = max(2, min(3, args.steps))
    ms64, dg64 = timed(opts64, k64)
    t64, u64 = aggregate(sum(ms64) / 1e3, units_per_step * k64, world)
    dfma_s, ddiv_s = npb.npb_measure_fp64(ctx)

    # ---- launches per step and per-kernel shares (events around every launch, no graph)
    npb.npb_ctx_profile(ctx, True)
    kp = 2
    with torch.cuda.stream(stream):
        for _ in range(kp):
            flush.zero_()
            step(opts)
    torch.cuda.synchronize()
    stats = npb.npb_ctx_kernel_stats(ctx)
    npb.npb_ctx_profile(ctx, False)
    mine = {k: v for k, v in stats.items() if v["launches"] > 0}
    launches_per_step = sum(v["launches"] for v in mine.values()) / kp
    share_total = sum(x["ms"] for x in mine.values())
    kernel_share = {k: round(v["ms"] / share_total, 4) for k, v in mine.items()}

    # ---- roofline of the dominant sweep, timed as the solve launches it
    elem = 4 if prec == npb.NPB_FP32_SWEEP else 8
    peak, peak_kind = measured_peaks()
    with torch.cuda.stream(stream):
        roofline = sweep_roofline(npb, grid, opts, problem, w, elem, peak, peak_kind, args.workload)
    roofline["kernel_share"] = kernel_share
    roofline["sweeps_share_of_step"] = roofline["sweeps_ms_per_solve"] / ms_per_step
    alg_step = 2 * elem * 3 * units_per_step  # 3 sweeps x (read + write) per interior point-step
    roofline["whole_step"] = {"achieved": alg_step / (ms_per_step * 1e-3) / 1e9, "unit": "GB/s",
                              "frac": alg_step / (ms_per_step * 1e-3) / 1e9 / peak,
                              "note": "24 B per interior point-step over the whole timed step (set-up included)"}

    # ---- end to end through the C ABI from pinned host buffers
    pin = {}
    for k in ("xyz", "q", "radius"):
        t = torch.from_numpy(np.ascontiguousarray(getattr(problem, k), dtype=np.float64)).pin_memory()
        pin[k] = t.numpy()

    class HostProblem:
        pass

    hp = HostProblem()
    for k in ("eps_in", "eps_out", "kappa2", "h", "n", "origin"):
        setattr(hp, k, getattr(problem, k))
    hp.xyz, hp.q, hp.radius = pin["xyz"], pin["q"], pin["radius"]
    ke = max(3, args.steps // 2)
    with torch.cuda.stream(stream):
        for _ in range(2):
            g2 = npb.npb_grid_create(ctx, hp)
            npb.npb_energy(g2, opts)
            npb.npb_grid_destroy(g2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            g2 = npb.npb_grid_create(ctx, hp)
            npb.npb_energy(g2, opts)
            npb.npb_grid_destroy(g2)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
    te, ue = aggregate(te, units_per_step * ke, world)
    h2d = sum(pin[k].nbytes for k in pin)

    npb.npb_grid_destroy(grid)
    npb.npb_ctx_destroy(ctx)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    base, errors = None, None
    if want_errors:
        errors, el, _ = error_report(legs32, dg, dg64, problem, w)
        del legs32
        base = cpu_baseline(problem, w, full_solve_s=el)
    extra = {}
    if world == 1 and args.workload != "protein_1k" and args.second_workload:
        extra["protein_1k"] = second_workload(npb, "protein_1k", prec, args)
    serving = serving_run(npb, args.serving_seconds, fifo_requests=args.fifo_requests) \
        if (world == 1 and args.serving_seconds > 0) else None
    batch = batch_run(npb, args.batch_count, tune=args.autotune) if (world == 1 and args.batch_count > 0) else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == npb.NPB_FP32_SWEEP else "f64",
        "data": "synthetic",
        "config": dict(workload_config(args, problem, w),
                       l2=("inputs larger than L2 (4 states of %.0f MB), and a 256 MB write before every step"
                           % (4 * problem.n[0] * problem.n[1] * problem.n[2] * elem / 1e6)),
                       step="set-up kernels + 4 legs + FP64 energy + 8-byte read-back",
                       parallelism=f"replicas x{world}"),
        "dG_kcal_mol": dg,
        "solves_per_s": args.steps * world / total_s,
        "fp64_path": dict({"value": u64 / t64 / 1e6, "unit": UNIT, "ms_per_step": 1e3 * t64 / k64,
                           "solves_per_s": k64 * world / t64, "dG_kcal_mol": dg64},
                          roofline=fp64_roofline(u64 / t64, dfma_s, ddiv_s, *measured_peaks())),
        "error_vs_oracle": errors,
        "wall_s_timed_region": wall,
        "roofline": roofline,
        "cpu_baseline": base,
        "e2e": {"value": ue / te / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 8,
                "call": "npb_grid_create + npb_energy + npb_grid_destroy from pinned host arrays"},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "solver_shapes": shapes,
        "autotune": tuning if args.verbose else sorted(tuning, key=lambda r: (r["dir"], r["ms"]))[:12],
        "other_workloads": extra,
        "serving": serving,
        "batch": batch,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def second_workload(npb, name, prec, args):
    """A shorter measurement of another configuration on the same GPU (throughput, sweep roofline)."""
    import torch

    problem, w = workload(name)
    units = point_steps(problem, w["n"])
    stream = torch.cuda.Stream()
    ctx = npb.npb_ctx_create(0, 0)
    npb.npb_ctx_set_stream(ctx, stream.cuda_stream)
    g = npb.npb_grid_create(ctx, problem)
    o = npb.make_opts(w["dt"], w["alpha"], w["n"], precision=prec)
    if args.autotune:
        npb.npb_autotune(g, o, reps=5)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ms = []
    with torch.cuda.stream(stream):
        for i in range(3 + args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            npb.npb_grid_refresh(g)
            npb.npb_energy(g, o)
            b.record(stream)
            if i >= 3:
                ms.append((a, b))
        torch.cuda.synchronize()
    t = [x.elapsed_time(y) for x, y in ms]
    ms_step = sum(t) / len(t)
    peak, kind = measured_peaks()
    with torch.cuda.stream(stream):
        roof = sweep_roofline(npb, g, o, problem, w, 4 if prec == npb.NPB_FP32_SWEEP else 8, peak, kind, name)
    shapes = {("x", "y", "z")[d]: npb.npb_tune_get(ctx, prec, d, problem.n[d]) for d in range(3)}
    npb.npb_grid_destroy(g)
    npb.npb_ctx_destroy(ctx)
    roof["sweeps_share_of_step"] = roof["sweeps_ms_per_solve"] / ms_step
    return {"workload": workload_config(args, problem, w)["workload"].replace(args.workload, name),
            "value": units / (ms_step * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms_step,
            "solves_per_s": 1e3 / ms_step, "roofline": roof, "solver_shapes": shapes,
            "l2": "states fit L2 (4 x 8.6 MB); 256 MB write before every step"}


def run_once(args):
    """One RE+V solve of the workload (grid set-up, legs, energy), untimed: the command profilers
    capture (ncu launch lists and kernel captures), with --once-steps LOD steps per dt leg."""
    import paper_1410_2788_gb300 as npb
    from paper_1410_2788_gb300 import build

    build.build()
    problem, w = workload(args.workload)
    prec = npb.NPB_FP32_SWEEP if args.precision == "fp32" else npb.NPB_FP64
    ctx = npb.npb_ctx_create(0, 0)
    try:
        g = npb.npb_grid_create(ctx, problem)
        try:
            n = args.once_steps if args.once_steps > 0 else w["n"]
            print("dG", npb.npb_energy(g, npb.make_opts(w["dt"], w["alpha"], n, precision=prec)))
        finally:
            npb.npb_grid_destroy(g)
    finally:
        npb.npb_ctx_destroy(ctx)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="large_20k", choices=["protein_1k", "large_20k", "born"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--batch-count", type=int, default=64,
                    help="molecules in the batched-workload measurement (0 skips it)")
    ap.add_argument("--serving-seconds", type=float, default=60.0,
                    help="length of the Poisson serving stream measured after the main line (0: skip)")
    ap.add_argument("--fifo-requests", type=int, default=50,
                    help="requests of the same stream served by the plain FP64 path, FIFO")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false",
                    help="skip the oracle timing and the error report against it")
    ap.add_argument("--no-second-workload", dest="second_workload", action="store_false",
                    help="skip the protein_1k measurement beside the headline workload")
    ap.add_argument("--once", action="store_true",
                    help="run one untimed solve of the workload and exit (for profilers)")
    ap.add_argument("--once-steps", type=int, default=0, help="LOD steps per dt leg of --once (0: the workload's)")
    args = ap.parse_args(argv)
    if args.once:
        return run_once(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
