"""Benchmark of one IDUGKS iteration (the whole hot path) on one GB300.

Workload (N=1): the 64 x 64 lid-driven cavity (Shakhov Pr=2/3, Kn=0.075, lid
0.15, 32 x 32 trapezoid velocities on [-4,4]^2, CFL 1000), mixed precision
(f in float32; moments, predictor, residual in float64).  A step is one
iteration: cell prep, interior and boundary faces, macroscopic LU-SGS
predictor, micro LU-SGS forward and backward sweeps.  The f state (33.6 MB)
fits in L2, so L2 is flushed (a 256 MB write) between timed steps.

The same run also times, per iteration, the workloads whose state lives in
HBM (--extra-workloads, default the 128^2 stretched cavity with 28^2
Gauss-Hermite velocities and the 121 x 81 Ma 5 cylinder with 89^2
velocities), each with its own roofline.

Prints one JSON line (metric: cell-velocity updates per second).  The
roofline divides the method's compulsory bytes (algorithmic_bytes) by the
measured device time of the dominant launch group, and of the whole
iteration, against the measured HBM copy bandwidth.
--impl reference times the FP64 CPU oracle on the host cores instead.
Under torchrun (N > 1) every rank solves its own copy of the cavity (the
method has no data-parallel exchange: replicas only) and rank 0 reports the
aggregate over ranks with the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1709_01819_gb300 import inputs as I  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
KERNELS = ["cell_prep", "face_moments", "face_flux", "macro", "k_sweep_fwd", "k_sweep_bwd"]
# launch groups timed by idg_iterate_profiled: cell_prep = k_cell_moments + k_cell_params + k_fbp;
# face_moments = k_face_moments + k_face_params; face_flux = k_face_flux + k_face_phi;
# macro = k_macro_pre + k_macro_sweep + k_macro_post


# point-relaxation sweeps per workload for the time-to-residual report (the
# fewest with the shortest time on GB300); the Ma 5 cylinder's impulsive start
# diverges under point relaxation and keeps LU-SGS only
RELAX_SWEEPS = {"cavity64": 9, "cavity128": 25, "couette64": 9}


def workload(name: str) -> I.Problem:
    if name == "cavity64":
        return I.cavity_c2()
    if name == "couette64":
        return I.couette_c1()
    if name == "cavity128":
        return I.cavity_c3()
    if name == "cylinder":
        return I.cylinder_c5()
    if name == "cavity64_tri":
        # the 64x64 cavity with every square split into two triangles (8192 cells);
        # implicit CFL 10: on these triangles the iteration diverges at 30 and
        # above (the oracle's as the library's)
        return I.tri_cavity(64, Kn=0.075, U=0.15, nv=32, vmax=4.0, cfl_imp=10.0)
    if name == "cylinder_hybrid":
        # the 121x81 cylinder as a hybrid mesh: quadrilaterals in the 41 rings next
        # to the wall, triangles outside (14641 cells), the ring closed by connectivity
        return I.hybrid_cylinder(ntheta=121, nr=81, nr_quad=41, cfl_imp=30.0)
    if name == "cylinder61x41":
        # the cylinder at a quarter of the cells (same velocities, f 158 MB):
        # the size for full ncu captures of its kernels
        return I.cylinder(ntheta=61, nr=41, cfl_imp=30.0, name="cylinder_61x41_ma5_kn0.1_v89")
    raise SystemExit(f"unknown workload {name}")


def algorithmic_bytes(prob: I.Problem, s: int):
    """Compulsory bytes of one IDUGKS iteration per launch group (s = bytes per
    scalar of f; every per-velocity array holds a G and an H scalar).  These
    are the method's own data movements, not this implementation's arrays:
    the per-(cell, velocity) state f~ must be read once before the
    macroscopic predictor (its moments and the face reconstructions), read
    again after it (the micro residual needs W^{n+1}), the forward sweep's
    increments Delta* written and read back, and f~ written by the update:
      cell_prep      read f~ (moments, fb+, face reconstructions)   2s per cell-velocity
      face_moments   face states from the moments                  O(faces)
      face_flux      flux moments Phi                              O(faces)
      macro          R_W, W read and written (float64)             64 B per cell
      k_sweep_fwd    read f~, write Delta*                         4s per cell-velocity
      k_sweep_bwd    read Delta* and f~, write f~                  6s per cell-velocity
    The face groups' per-face side data (a few float64 per face) is counted
    as 64 B per cell like the predictor's.  The whole iteration's lower bound
    is 10s per cell-velocity (ITER_SCALARS): the two reads of f~ by the
    residual and by the update can be one."""
    N, Nv = prob.ncells, prob.nvel
    cv = N * Nv
    return {
        "cell_prep": 2 * s * cv,
        "face_moments": 64 * N,
        "face_flux": 64 * N,
        "macro": 64 * N,
        "k_sweep_fwd": 4 * s * cv,
        "k_sweep_bwd": 6 * s * cv,
    }


# scalars of f per cell-velocity that one iteration must move at least
ITER_SCALARS = 10


def roofline(prob: I.Problem, s: int, kms, ms_iter: float, peak: float, traffic_of=None):
    """The dominant launch group (largest device time, every group a
    candidate) against the HBM copy peak, with its compulsory bytes; the
    whole iteration's compulsory bytes (ITER_SCALARS per cell-velocity)
    against the iteration's time beside it."""
    alg = algorithmic_bytes(prob, s)
    dom = max(KERNELS, key=lambda k: kms[KERNELS.index(k)])
    dom_ms = float(kms[KERNELS.index(dom)])
    achieved = alg[dom] / (dom_ms * 1e-3) / 1e9
    it_bytes = ITER_SCALARS * s * prob.ncells * prob.nvel
    it_ach = it_bytes / (ms_iter * 1e-3) / 1e9
    groups = {k: {"ms": float(kms[i]), "algorithmic_bytes": alg[k],
                  "achieved_gbs": alg[k] / (float(kms[i]) * 1e-3) / 1e9 if kms[i] > 0 else None}
              for i, k in enumerate(KERNELS)}
    for g in groups.values():
        g["frac"] = g["achieved_gbs"] / peak if g["achieved_gbs"] is not None else None
    return {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic_of(dom) if traffic_of else None,
            "algorithmic_bytes": alg[dom], "kernel_ms": dom_ms,
            "iteration": {"algorithmic_bytes": it_bytes, "ms": ms_iter, "achieved": it_ach,
                          "frac": it_ach / peak, "scalars_per_cell_velocity": ITER_SCALARS},
            "groups": groups}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def host_cores() -> int:
    """Threads the oracle's OpenMP loops use (OMP_NUM_THREADS, else every core)."""
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms: float, dist=None, device="cpu") -> float:
    """The slowest rank's timed milliseconds: the whole job ends with it
    (every rank runs its own replica; the collective only reduces timings)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_step: int, steps: int, world_size: int, max_ms: float) -> float:
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    return units_per_step * steps * world_size / (max_ms * 1e-3)


def run_reference(args, prob):
    """The FP64 oracle on the host cores: each step is one IDUGKS iteration of
    the same cavity."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    o = O.Oracle(prob)
    o.init_uniform()
    o.iterate(args.warmup)
    t0 = time.perf_counter()
    o.iterate(args.steps)
    dt = time.perf_counter() - t0
    ups = prob.ncells * prob.nvel * args.steps / dt
    cores = host_cores()
    line = {
        "impl": "reference", "metric": "cell-velocity updates/s", "value": ups,
        "unit": "cell-velocity updates/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": prob.name, "cells": prob.ncells, "velocities": prob.nvel,
                   "precision": "fp64-oracle"},
        "cpu_baseline": {"value": ups, "unit": "cell-velocity updates/s", "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(), "nproc": os.cpu_count(),
                         "sample": f"{args.steps} full IDUGKS iterations of {prob.name} after {args.warmup} warm-up"},
        "e2e": {"value": ups, "unit": "cell-velocity updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    # the oracle's own time to the residual 1e-6 from the uniform start, on the
    # workloads it converges in seconds (C1, C2); the larger ones would take
    # hours on the host cores
    if not args.no_ttr and args.workload in ("cavity64", "couette64"):
        o2 = O.Oracle(prob)
        o2.init_uniform()
        t0, hist = time.perf_counter(), []
        while len(hist) < 20000:
            hist.extend(o2.iterate(1))
            if hist[-1] <= 1e-6 * hist[0]:
                break
        n = len(hist)
        line["time_to_residual_1e-6"] = {
            "fp64_oracle": {"seconds": time.perf_counter() - t0, "iterations": int(n),
                            "residual": float(hist[-1] / hist[0]), "converged": bool(hist[-1] <= 1e-6 * hist[0]),
                            "cores": cores}}
    print(json.dumps(line), flush=True)


def cpu_baseline(prob, budget_s=15.0):
    """Time the oracle as it stands on a bounded sample: whole IDUGKS iterations
    of the same cavity until about budget_s seconds have passed."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_cpu_worker, args=(prob.name, budget_s, q))
    p.start()
    p.join(timeout=budget_s * 6 + 120)
    if p.is_alive():
        p.kill()
        return None
    return q.get() if not q.empty() else None


def _cpu_worker(name, budget_s, q):
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    prob = workload_by_name(name)
    o = O.Oracle(prob)
    o.init_uniform()
    o.iterate(1)
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s or n < 2:
        o.iterate(1)
        n += 1
    dt = time.perf_counter() - t0
    q.put({"value": prob.ncells * prob.nvel * n / dt, "unit": "cell-velocity updates/s",
           "cores": host_cores(), "kind": "oracle", "cpu_model": cpu_model(), "nproc": os.cpu_count(),
           "sample": f"{n} full FP64 IDUGKS iterations of {name} ({dt:.1f} s)"})


def workload_by_name(name):
    for w in ("cavity64", "couette64", "cavity128", "cylinder", "cylinder61x41", "cavity64_tri", "cylinder_hybrid"):
        p = workload(w)
        if p.name == name:
            return p
    raise KeyError(name)


def run_batch(args):
    """64 seeded cavities (Kn log-uniform in [1e-3, 10], lid speed in [0.05, 0.3],
    n in {32, 48, 64, 96}, 32 x 32 velocities), mixed precision, autotuned sweep
    tiles, one launch per kernel over all instances, graph-replayed.  A step is
    one iteration of every instance; the 2.2 GB state exceeds L2.  --tune
    default / an explicit shape replace the autotuner as for one instance."""
    import torch
    from paper_1709_01819_gb300 import build
    from paper_1709_01819_gb300.solver import BatchSolver
    build.build()
    probs = I.batch_c4()
    t0 = time.perf_counter()
    fixed = None
    if args.tune not in ("auto", "default"):
        fixed = {k: int(v) for k, v in (kv.split("=") for kv in args.tune.split(","))}
    bs = BatchSolver(probs, args.precision, autotune=args.tune == "auto", tuning=fixed)
    setup_s = time.perf_counter() - t0
    bs.iterate(args.warmup)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        a.record(stream)
        bs.iterate(args.steps)
        e.record(stream)
        torch.cuda.synchronize()
    ms = a.elapsed_time(e)
    cv = bs.cell_velocities
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    sb = 8 if args.precision == "fp64" else 4
    ib = ITER_SCALARS * sb * cv  # the whole iteration's algorithmic bytes, all instances
    ach = ib / (ms / args.steps * 1e-3) / 1e9
    tiles = {}
    for s in bs.solvers:
        t = s.tuning()
        tiles[f"{s.prob.ni}x{s.prob.nj}"] = t["sweep_tv"]
    line = {
        "metric": "cell-velocity updates/s", "value": cv * args.steps / (ms * 1e-3), "unit": "cell-velocity updates/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": "batch of 64 cavities (seed 170901819)", "instances": len(probs),
                   "cell_velocities": cv, "precision": args.precision, "l2": "state larger than L2",
                   "sweep_tv": tiles, "tuning": args.tune, "setup_and_tuning_s": setup_s},
        "roofline": {"bound": "hbm", "kernel": "whole iteration, all instances", "achieved": ach, "peak": peak,
                     "unit": "GB/s", "frac": ach / peak, "traffic": None, "algorithmic_bytes": ib,
                     "scalars_per_cell_velocity": ITER_SCALARS,
                     "peak_source": "measured" if peaks else "fallback"},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def profiled_group_ms(s, flush, nprof: int = 10):
    """Mean device ms of the six launch groups over nprof profiled iterations
    (CUDA events between the launches, L2 flushed before each)."""
    kms = np.zeros(6)
    for _ in range(nprof):
        flush.fill_(1)
        kms += s.iterate_profiled()
    return kms / nprof


def time_workload(prob, precision, local, flush, peak, tune="auto", steps=10, warmup=3, traffic_of=None):
    """ms per iteration (CUDA events around each, L2 flushed between), the
    update rate, the group times and the roofline of one workload from its
    uniform start after warm-up iterations; traffic_of(group) gives the
    group's DRAM bytes per launch from an ncu capture (or None)."""
    import torch
    from paper_1709_01819_gb300.solver import Autotuner, Solver
    s = Solver(prob, precision, device=local)
    s.init_uniform()
    if tune == "auto":
        Autotuner().tune(s)
    for _ in range(warmup):
        s.iterate(1)
    stream = torch.cuda.current_stream()
    a = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    b = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for q in range(steps):
            flush.fill_(q & 0xff)
            a[q].record(stream)
            s.iterate(1)
            b[q].record(stream)
        torch.cuda.synchronize()
    ms = sum(x.elapsed_time(y) for x, y in zip(a, b)) / steps
    kms = profiled_group_ms(s, flush)
    sb = 8 if precision == "fp64" else 4
    out = {"workload": prob.name, "cells": prob.ncells, "velocities": prob.nvel, "precision": precision,
           "ms_per_step": ms, "value": prob.ncells * prob.nvel / (ms * 1e-3), "unit": "cell-velocity updates/s",
           "steps": steps, "tuning": s.tuning(), "roofline": roofline(prob, sb, kms, ms, peak, traffic_of),
           "clocks": clk.summary()}
    del s
    torch.cuda.empty_cache()
    return out


def ttr_runs(prob, local, precisions=("mixed", "fp64"), max_iter=20000):
    """Wall-clock time from the uniform start to the relative residual 1e-6
    (idg_iterate stops at the crossing), per precision."""
    import torch
    from paper_1709_01819_gb300.solver import Solver
    out = {}
    for prec in precisions:
        s2 = Solver(prob, prec, device=local)
        s2.init_uniform()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ok, n, r = s2.iterate(max_iter, 1e-6)
        torch.cuda.synchronize()
        out[prec] = {"seconds": time.perf_counter() - t0, "iterations": n, "residual": r, "converged": ok}
        del s2
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cavity64")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ttr", action="store_true", help="skip the time-to-residual runs")
    ap.add_argument("--relax-sweeps", type=int, default=0,
                    help="macroscopic predictor of the timed solver: 0 LU-SGS (Eq. 30), n point relaxation with n sweeps")
    ap.add_argument("--implicit-wall", action="store_true",
                    help="timed solver with the linearised diffuse wall in the micro sweeps (Eq. 33-35)")
    ap.add_argument("--explicit-ttr", action="store_true",
                    help="also time explicit DUGKS (Eq. 21, same precision) to the residual 1e-6 (tens of seconds)")
    ap.add_argument("--extra-workloads", default="cavity128,cylinder",
                    help="comma-separated workloads timed per iteration after the main one (rank 0, N=1); "
                         "empty to skip")
    ap.add_argument("--ttr-extra", action="store_true",
                    help="also time the extra workloads to the residual 1e-6, mixed and FP64 (minutes)")
    ap.add_argument("--tune", default="auto",
                    help="auto: pick the sweep tiles and prefetch depths with the autotuner before timing; "
                         "default: the library's default shape; or an explicit shape such as "
                         "sweep_tv=4,sweep_vpt=2 (keys of Solver.set_tuning)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.workload == "batch64":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batch workload is timed on the GPU arm only"}))
            return
        run_batch(args)
        return
    prob = workload(args.workload)
    if args.relax_sweeps:
        import dataclasses
        prob = dataclasses.replace(prob, relax_sweeps=args.relax_sweeps)
    if args.implicit_wall:
        import dataclasses
        prob = dataclasses.replace(prob, implicit_wall=1)
    if args.impl == "reference":
        run_reference(args, prob)
        return

    ws, rank, local = dist_env()
    # the CPU baseline runs first, in a spawned process, before any GPU work
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(prob)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1709_01819_gb300 import build
    from paper_1709_01819_gb300.solver import Solver
    build.build()

    s = Solver(prob, args.precision, device=local)
    s.init_uniform()
    if args.tune not in ("auto", "default"):
        s.set_tuning(**{k: int(v) for k, v in (kv.split("=") for kv in args.tune.split(","))})
    elif args.tune == "auto":
        from paper_1709_01819_gb300.solver import Autotuner
        Autotuner().tune(s)
    tuning = s.tuning()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        s.iterate(1)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # timed region: K iterations, each bracketed by CUDA events on the launching
    # stream, with an L2 flush (outside the events) between them
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for q in range(args.steps):
            flush.fill_(q & 0xff)
            starts[q].record(stream)
            s.iterate(1)
            ends[q].record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total_ms = max_over_ranks(sum(step_ms), dist, f"cuda:{local}")
    ups = job_throughput(prob.ncells * prob.nvel, args.steps, ws, total_ms)

    # per-kernel device time (events between launches) for the roofline
    kms = profiled_group_ms(s, flush)
    sbytes = 8 if args.precision == "fp64" else 4
    peaks = {}
    if os.path.exists(PEAKS_FILE):
        peaks = json.load(open(PEAKS_FILE))
    peak = peaks.get("hbm_gbs", 6800.0)
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    tr = json.load(open(tfile)) if os.path.exists(tfile) else {}
    roof = roofline(prob, sbytes, kms, sum(step_ms) / args.steps, peak,
                    lambda g: tr.get(f"{args.workload}:{args.precision}:{g}"))
    roof["peak_source"] = "measured" if peaks else "fallback"

    # end to end through the C ABI with host buffers: per step upload the state
    # from pinned host memory (set_state), iterate once, read the moments back
    G, H, W = s.get_state()
    Gp = torch.from_numpy(G).pin_memory().numpy()
    Hp = torch.from_numpy(H).pin_memory().numpy()
    Wp = torch.from_numpy(W).pin_memory().numpy()
    e2e_steps = min(args.steps, 10)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.set_state(Gp, Hp, Wp)
        s.iterate(1)
        m = s.moments()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": prob.ncells * prob.nvel * e2e_steps / e2e_s, "unit": "cell-velocity updates/s",
           "h2d_bytes_per_step": int(G.nbytes + H.nbytes + W.nbytes), "d2h_bytes_per_step": int(m.nbytes),
           "steps": e2e_steps}

    # time to residual 1e-6 from the uniform start, mixed and FP64
    ttr = None
    if rank == 0 and not args.no_ttr:
        ttr = {}
        for prec in ("mixed", "fp64"):
            s2 = Solver(prob, prec, device=local)
            s2.init_uniform()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ok, n, r = s2.iterate(20000, 1e-6)
            torch.cuda.synchronize()
            ttr[prec] = {"seconds": time.perf_counter() - t0, "iterations": n, "residual": r, "converged": ok}
            del s2
        # the point-relaxation predictor (the paper's other predictor), where
        # it converges from the uniform start: Jacobi sweeps chosen per workload
        sweeps = RELAX_SWEEPS.get(args.workload)
        if sweeps:
            import dataclasses
            for prec in ("mixed", "fp64"):
                s2 = Solver(dataclasses.replace(prob, relax_sweeps=sweeps), prec, device=local)
                s2.init_uniform()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ok, n, r = s2.iterate(20000, 1e-6)
                torch.cuda.synchronize()
                ttr[f"{prec}_point_relaxation"] = {"seconds": time.perf_counter() - t0, "iterations": n,
                                                   "residual": r, "converged": ok, "sweeps": sweeps}
                del s2
        # the linearised diffuse wall in the micro sweeps (Eq. 33-35), LU-SGS
        # predictor, against the zero ghost increments above
        if not prob.implicit_wall and not prob.relax_sweeps:
            import dataclasses
            for prec in ("mixed", "fp64"):
                s2 = Solver(dataclasses.replace(prob, implicit_wall=1), prec, device=local)
                s2.init_uniform()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ok, n, r = s2.iterate(20000, 1e-6)
                torch.cuda.synchronize()
                ttr[f"{prec}_implicit_wall"] = {"seconds": time.perf_counter() - t0, "iterations": n,
                                                "residual": r, "converged": ok}
                del s2
        if args.explicit_ttr:
            # explicit DUGKS: physical step dt, residual ||(W^{n+1} - W^n)/dt||
            s2 = Solver(prob, args.precision, device=local, explicit=True)
            s2.init_uniform()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ok, n, r = s2.iterate(1000000, 1e-6)
            torch.cuda.synchronize()
            ttr["explicit_" + args.precision] = {"seconds": time.perf_counter() - t0, "iterations": n,
                                                 "residual": r, "converged": ok}
            del s2

    # the HBM-resident workloads (state above or near L2), per iteration, in
    # the same run: their roofline is the one the HBM bound speaks to
    extra = {}
    if rank == 0 and ws == 1 and args.extra_workloads:
        del s
        torch.cuda.empty_cache()
        for name in args.extra_workloads.split(","):
            extra[name] = time_workload(workload(name), args.precision, local, flush, peak, args.tune,
                                        steps=10, warmup=3,
                                        traffic_of=lambda g, n=name: tr.get(f"{n}:{args.precision}:{g}"))
            extra[name]["roofline"]["peak_source"] = roof["peak_source"]
            if args.ttr_extra:
                extra[name]["time_to_residual_1e-6"] = ttr_runs(workload(name), local, max_iter=40000)

    if rank == 0:
        line = {
            "metric": "cell-velocity updates/s", "value": ups, "unit": "cell-velocity updates/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": prob.name, "cells": prob.ncells, "velocities": prob.nvel,
                       "predictor": (f"point relaxation, {prob.relax_sweeps} sweeps" if prob.relax_sweeps
                                     else "LU-SGS (Eq. 30)"),
                       "wall_ghost": ("linearised diffuse wall (Eq. 34-35)" if prob.implicit_wall
                                      else "zero ghost increments"),
                       "precision": args.precision, "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": "replicas" if ws > 1 else "single", "tuning": tuning},
            "roofline": roof,
            "kernel_ms": {k: float(v) for k, v in zip(KERNELS, kms)},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "time_to_residual_1e-6": ttr,
            "hbm_workloads": extra,
            "clocks": clk.summary(),
            # per iteration: cell moments, cell params, fb+, [limited gradients],
            # face moments, face params, face flux, Phi, macro pre / sweep /
            # post, micro residual, forward and backward sweeps
            # (point relaxation: the residual record and n sweeps replace the
            # wavefront kernel)
            "gpu_launches": (13 + (1 if prob.limiter else 0) + prob.relax_sweeps) * args.steps,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
