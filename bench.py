#!/usr/bin/env python3
"""Throughput of the splitting random-choice dynamic relaxation (TL-SPH) on GB300.

Workload: the 3D cantilever plate 0.2 x 0.02 x 0.1 m at dp = 1 mm (200 x 20 x
100 body particles + 3 clamped layers = 406,000 particles, ~80 neighbours
each), neo-Hookean E = 2e6 Pa, nu = 0.3, gravity, random-choice p = 0.2, seed 1,
FP32-mixed precision.  A "step" is one relaxation time step of the whole hot
path: stress pass, force/update pass, the damping sweep over all 27 colours
forward and backward on the randomly chosen steps, and the FP64 kinetic-energy
reduction.  value = particles x steps / device time (particle-steps/s).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

N > 1 runs under torchrun as independent body replicas (one per GPU, no
collective on the data path); value is the aggregate over all ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/s"
WORKLOAD = "3D cantilever plate 0.2x0.02x0.1 m, dp=1 mm (406,000 particles), FP32-mixed, p=0.2, seed 1"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-l2-flush", action="store_true",
                    help="skip the l2_flushed record (steps timed one at a time after a 256 MB write)")
    ap.add_argument("--sweep-sync", choices=["auto", "barrier", "cells"], default="auto",
                    help="synchronisation of the damping sweep's colour phases (default: autotuned)")
    ap.add_argument("--workload", choices=["plate", "batched", "served", "block", "compare", "strength",
                                           "layout"], default="plate")
    ap.add_argument("--compare-cap", type=int, default=200000,
                    help="step cap of each relaxation in the compare and strength workloads")
    ap.add_argument("--rates", type=float, nargs="+", default=[10, 30, 100, 300, 1000])
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--served-max-n", type=float, default=2e4)
    ap.add_argument("--served-tol", type=float, default=1e-8)
    ap.add_argument("--served-max-steps", type=int, default=20000)
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched-vs-one-at-a-time solves/s record of the default line")
    ap.add_argument("--no-served", action="store_true",
                    help="skip the served-stream record of the default line")
    ap.add_argument("--batch-bodies", type=int, default=24,
                    help="bodies of the batched solves/s sample (the first of the 256-body workload)")
    ap.add_argument("--solve-cap", type=int, default=100000,
                    help="step cap of the solves in the batched and served records")
    ap.add_argument("--served-requests", type=int, default=24,
                    help="requests per rate in the served record of the default line")
    ap.add_argument("--served-rates", type=float, nargs="+", default=[10.0, 100.0])
    return ap.parse_args()


def max_over_ranks(x: float) -> float:
    """The largest x over all ranks (the slowest rank's time); x itself when
    torch.distributed is not initialised or has one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time
    (replicas: each rank relaxes its own copy of the workload)."""
    return world * units_per_rank * steps / (max_ms / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, flag in zip(names, parts[4:8]):
                if flag.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- roofline bookkeeping
def algorithmic_bytes(n, nnz, dim=3):
    """Algorithmic HBM bytes per launch of the 3D FP32-mixed passes: a
    neighbour stream of (col int32, s_ij fp32) = 8 B per pair, every
    per-particle array the pass needs touched once, neighbour gathers counted
    as L2 hits.  Pass A: u hi/lo read 24, B0 36, PB written 36, r0 12.
    Pass B: PB 36, u hi/lo read and written 48, v read and written 24, r0 12,
    mass 4, flags 1."""
    pairs = 8 * nnz
    return {"pass_a": pairs + n * (24 + 36 + 36 + 12),
            "pass_b": pairs + n * (36 + 48 + 24 + 12 + 4 + 1)}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------- CPU baseline (oracle)
def oracle_rate(spec, steps, seed_steps=0, threads=0):
    """Time the FP64 oracle on `steps` steps of `spec` (threads > 0: its
    OpenMP build on that many threads, the same bits); returns (p-steps/s, n,
    seconds, damped steps)."""
    from oracle import oracle as O
    from paper_2103_08932_gb300 import synth as S
    r0, flags, u0 = S.lattice(spec)
    b = O.OracleBody(O.Params(dim=spec.dim, material=spec.material, rho0=spec.rho0, E=spec.E,
                              nu=spec.nu, h=spec.h, gravity=spec.gravity, beta=spec.beta,
                              L_char=spec.L_char, alpha=spec.alpha, seed=spec.seed),
                     r0, vol_default=spec.vol, flags=flags, threads=threads)
    if seed_steps:
        b.step(seed_steps)
    t = time.perf_counter()
    b.step(steps)
    el = time.perf_counter() - t
    return b.n * steps / el, b.n, el, b.damped_steps


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def cpu_baseline():
    """The FP64 oracle on the host: its OpenMP build on every core (the
    reported value) and its serial build on one, on the same bounded sample."""
    from oracle import oracle as O
    from paper_2103_08932_gb300 import synth as S
    spec = S.cantilever_plate_3d()
    # bounded sample: the full 406,000-particle plate, steps 0..7 (step 7 is
    # the first damped step of seed 1): about 10-20 s of single-thread work
    cores = os.cpu_count() or 1
    rate_all, n, el_all, damped = oracle_rate(spec, 8, threads=cores)
    rate1, _, el1, _ = oracle_rate(spec, 8)
    return {"value": rate_all, "unit": METRIC, "cores": O.threads_available() if cores > 1 else 1,
            "kind": "oracle", "cpu_model": cpu_model(), "nproc": cores,
            "single_thread_value": rate1,
            "sample": f"full plate ({n} particles), 8 time steps incl. {damped} damped, FP64 C "
                      f"oracle: OpenMP build on {cores} threads {el_all:.1f} s, serial build "
                      f"{el1:.1f} s (identical bits)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2103_08932_gb300 import synth as S
    # each step: one oracle time step of a scaled copy of the plate (same dp,
    # same physics), sized so that W + K steps take about 90 s on one core
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    threads = cores if cores > 1 else 0
    full = S.cantilever_plate_3d()
    probe = S.scaled(full, 0.25)
    r_probe, n_probe, _, _ = oracle_rate(probe, 2, threads=threads)
    budget = 90.0 / max(1, args.steps + args.warmup)
    n_target = max(2000, min(406000, r_probe * budget))
    f = max(0.12, min(1.0, (n_target / 406000.0) ** (1.0 / 3.0)))
    spec = S.scaled(full, f)
    rate, n, el, damped = oracle_rate(spec, args.steps, seed_steps=args.warmup, threads=threads)
    ms = el / args.steps * 1e3
    used = O.threads_available() if threads else 1
    out = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "reference_sample": f"plate scaled x{f:.3f} ({n} particles)"},
        "cpu_baseline": {"value": rate, "unit": METRIC, "cores": used, "kind": "oracle",
                         "cpu_model": cpu_model(),
                         "sample": f"plate scaled x{f:.3f} ({n} particles), {args.steps} steps "
                                   f"({damped} damped) after {args.warmup} warm-up steps, "
                                   f"FP64 C oracle on {used} thread(s)"},
        "e2e": {"value": rate, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


# ---------------------------------------------------------------- GPU arm
def run_gpu(args):
    import numpy as np
    import torch

    from paper_2103_08932_gb300 import build, srdr
    from paper_2103_08932_gb300 import synth as S

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    build.build()
    srdr.lib()
    spec = S.cantilever_plate_3d()
    desc = srdr.make_desc(spec, precision=srdr.SRDR_FP32_MIXED)
    stream = torch.cuda.current_stream()
    body = srdr.Body(desc, stream=stream.cuda_stream)
    body.sweep_sync(SYNC_MODES[args.sweep_sync])

    body.step(args.warmup)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.2)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    st0 = body.stats()
    # per-kernel CUDA events on every 8th step of the timed region (the
    # events' own cost stays out of the other steps)
    body.profile(8)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    body.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    body.profile(False)
    kt = body.kernel_times()
    st1 = body.stats()
    clocks = sampler.stop()
    ms = max_over_ranks(ms)
    n = body.n
    value = aggregate_rate(n, args.steps, world, ms)
    launches = int(st1["launches"] - st0["launches"])
    damped = int(st1["damped_steps"] - st0["damped_steps"])

    # roofline of the dominant kernel class
    peak, peak_kind = load_peaks()
    ab = algorithmic_bytes(n, body.nnz)
    per = {k: (v["ms"] / max(v["intervals"], 1)) for k, v in kt.items()}
    # the sweep: both directions of S_d in one launch, the CSR stream and the
    # velocities read and written once per direction
    ab["sweep"] = 2 * (8 * body.nnz + 28 * n)
    dom = max(("pass_a", "pass_b", "sweep"), key=lambda k: kt[k]["ms"])
    achieved = ab[dom] / (per[dom] / 1e3) / 1e9
    traffic = None
    tf = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tf):
        try:
            with open(tf) as fh:
                traffic = json.load(fh).get(dom)
        except (OSError, ValueError):
            traffic = None

    # the same steps with L2 flushed before each one: 256 MB written on the
    # body's stream, then the step timed alone.  The passes' per-particle
    # arrays (about 150 B per particle) fit in L2 and may stay there between
    # undamped steps of the continuous run above; the sweep's slot records
    # (8 B per pair) pass through L2 on every damped step.  A step timed
    # alone also waits for its own launches, so this rate is a lower bound.
    l2f = None
    if not args.no_l2_flush:
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        nfl = min(args.steps, 400)
        d0 = body.stats()["damped_steps"]
        tot = 0.0
        for s in range(nfl):
            flush.fill_(s & 0xFF)
            e0.record(stream)
            body.step(1)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        l2f = {"steps": nfl, "damped_steps": int(body.stats()["damped_steps"] - d0),
               "ms_per_step": tot / nfl, "value": world * n / (tot / nfl / 1e3),
               "flush": "256 MB written before each step; each step timed alone on the body's stream"}
        del flush

    # end to end through the C ABI with host buffers: create the body from
    # host particle arrays (H2D), run the steps, read the displacement (D2H)
    e2e = None
    if not args.no_e2e:
        r0, flags, u0 = S.lattice(spec)
        r0p = torch.from_numpy(np.ascontiguousarray(r0)).pin_memory()
        flp = torch.from_numpy(np.ascontiguousarray(flags)).pin_memory()
        outp = torch.empty((n, 3), dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b2 = srdr.Body(desc, r0=r0p.numpy(), flags=flp.numpy(), stream=stream.cuda_stream)
        b2.sweep_sync(SYNC_MODES[args.sweep_sync])
        b2.step(args.steps)
        import ctypes
        srdr._check(srdr.lib().srdr_body_read_displacement(
            b2.h, ctypes.c_void_p(outp.data_ptr()), outp.numel()))
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        b2.close()
        h2d = r0p.numel() * 8 + flp.numel()
        d2h = outp.numel() * 8
        e2e = {"value": world * n * args.steps / el, "unit": METRIC,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "includes": "body build from host arrays + steps + displacement read-back"}

    # per-step cost of the two kinds of step, from the per-kernel events: an
    # undamped step is the stress and force passes; a damped step adds the
    # damping sweep and the finish pass.  value_at_alpha is the rate at the
    # expected damped fraction alpha = 0.2 (a short window damps a random
    # number of steps)
    ms_u = per["pass_a"] + per["pass_b"]
    ms_d = ms_u + per["sweep"] + per["finish"]
    alpha = spec.alpha
    step_mix = {"ms_undamped_step": ms_u, "ms_damped_step": ms_d,
                "damped_fraction": damped / args.steps, "alpha": alpha,
                "value_at_alpha": world * n / (((1 - alpha) * ms_u + alpha * ms_d) / 1e3)}

    batched = served = None
    if rank == 0 and not args.no_batched:
        batched = run_batched_solves(args.batch_bodies, args.solve_cap)
    if rank == 0 and not args.no_served:
        served = [run_served(r, args.served_requests, 1e3, 2e5, 1e-8, args.solve_cap, seed=4,
                             workload_note=SERVED_NOTE) for r in args.served_rates]

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline()

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "particles": n, "neighbour_pairs": body.nnz,
                       "damped_steps": damped, "parallelism": f"replicas{world}",
                       "pass_mapping": {1: "sliced-ELL", 2: "bricks", 3: "lattice stencil"}.get(st1.get("pass_mapping"), "?"),
                       "sweep_cells_per_warp": st1.get("sweep_cells_per_warp"),
                       "sweep_sync": {srdr.SRDR_SWEEP_CELLS: "cell-wise waits",
                                      srdr.SRDR_SWEEP_BARRIER: "grid barriers"}.get(st1.get("sweep_sync")),
                       "l2": (f"no flush in the timed region: body data {(150 * n + 8 * body.nnz) / 1e6:.0f} MB "
                              f"> 129 MB L2, of which the sweep's slot records ({8 * body.nnz / 1e6:.0f} MB) "
                              f"stream through L2 on every damped step while the passes' per-particle arrays "
                              f"({150 * n / 1e6:.0f} MB) may stay in L2 between undamped steps; `l2_flushed` "
                              f"times steps after a 256 MB write")},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": peak_kind, "algorithmic_bytes": ab[dom]},
            **step_mix,
            "kernels_ms_per_launch": per,
            "kernels_ms_total": {k: v["ms"] for k, v in kt.items()},
            "batched": batched,
            "served": served,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "l2_flushed": l2f,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(out))
    body.close()
    if world > 1:
        torch.distributed.destroy_process_group()


SYNC_MODES = {"auto": 0, "barrier": 1, "cells": 2}


def run_batched(nbodies, n_lo, n_hi, steps, seed=3, sync="auto"):
    """Uneven bodies (counts log-uniform in [n_lo, n_hi], box / beam / plate,
    aspect 1-20, E log-uniform 1e5-1e7, nu 0.2-0.45, gravity or end load):
    `steps` steps of all of them as one batch vs the same steps one body at a
    time, FP32-mixed, device time with CUDA events."""
    import torch

    from paper_2103_08932_gb300 import srdr
    from paper_2103_08932_gb300 import synth as S
    specs = S.random_bodies(nbodies, n_lo, n_hi, seed)
    descs = [srdr.make_desc(s, precision=srdr.SRDR_FP32_MIXED) for s in specs]
    bodies = [srdr.Body(d) for d in descs]
    for b in bodies:
        b.sweep_sync(SYNC_MODES[sync])
    n_total = sum(b.n for b in bodies)
    batch = srdr.Batch(bodies)
    batch.step(8)  # warm-up, autotuner, graph capture
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch.step(steps)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    info = batch.info()
    batch.close()
    t_alone = 0.0
    for b in bodies:
        b.step(8)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.step(steps)
        torch.cuda.synchronize()
        t_alone += time.perf_counter() - t0
        b.close()
    return {"workload": f"{nbodies} bodies, particles log-uniform {int(n_lo)}-{int(n_hi)} "
                        f"({n_total} in all), FP32-mixed, seed {seed}",
            "steps": steps, "particles": n_total,
            "batched_particle_steps_per_s": n_total * steps / t_batch,
            "one_at_a_time_particle_steps_per_s": n_total * steps / t_alone,
            "speedup": t_alone / t_batch, "launches_per_step": info["launches"] / max(1, info["steps"]),
            "sweep_cells_per_warp": info["sweep_cells_per_warp"], "pass_threads": info["pass_threads"]}


CONFIG4_NOTE = ("random box / beam / plate bodies, particles log-uniform 1e3-2e5, aspect 1-20, "
                "E log-uniform 1e5-1e7, nu 0.2-0.45, gravity or end load; narrowed as the "
                "method requires: at least 6 layers thick, loads capped at a 5 % linear tip "
                "deflection (thinner or harder-loaded bodies diverge, the oracle's too)")
SERVED_NOTE = ("served bodies drawn like the batched workload (particles log-uniform 1e3-2e5, "
               "not the 1e3-1e6 of the full served workload: a default run stays within minutes)")


def run_batched_solves(nbodies, cap, tol=1e-8, seed=3):
    """Whole solves of the batched workload's first `nbodies` bodies (FP32-mixed,
    KE/KE_max < tol, at most `cap` steps): relaxed together as one batch, and
    one body at a time through srdr_body_relax on the same GPU.  solves/s
    counts converged bodies only; both runs stop every body at its own
    criterion, so their results are bitwise the same."""
    import torch

    from paper_2103_08932_gb300 import srdr
    from paper_2103_08932_gb300 import synth as S
    specs = S.random_bodies(256, 1e3, 2e5, seed)[:nbodies]
    descs = [srdr.make_desc(s, precision=srdr.SRDR_FP32_MIXED) for s in specs]
    # shared launches take sliced-ELL bodies
    descs_sell = [srdr.make_desc(s, precision=srdr.SRDR_FP32_MIXED, pass_layout=srdr.SRDR_PASS_LAYOUT_SELL)
                  for s in specs]
    runs = {}
    for name, mode in (("shared", srdr.SRDR_BATCH_SHARED), ("streams", srdr.SRDR_BATCH_STREAMS)):
        bodies = [srdr.Body(d) for d in (descs_sell if mode == srdr.SRDR_BATCH_SHARED else descs)]
        n_total = sum(b.n for b in bodies)
        batch = srdr.Batch(bodies)
        batch.mode(mode)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        status, per, steps_b = batch.run(tol, cap)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
        info = batch.info()
        batch.close()
        runs[name] = {"t": t_batch, "conv": [int(x) == 0 for x in per], "steps": steps_b,
                      "u": [b.displacement() for b in bodies], "n": [b.n for b in bodies], "info": info}
        for b in bodies:
            b.close()
    t_batch = runs["streams"]["t"]
    conv_b = runs["streams"]["conv"]
    steps_b = runs["streams"]["steps"]
    u_b = runs["streams"]["u"]
    info = runs["shared"]["info"]
    t_alone = 0.0
    conv_a, steps_a, same = [], [], 0
    for k, d in enumerate(descs):
        b = srdr.Body(d)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, steps, _ = b.relax(tol, cap, check=False)
        torch.cuda.synchronize()
        t_alone += time.perf_counter() - t0
        conv_a.append(st == srdr.SRDR_OK)
        steps_a.append(steps)
        same += int(np.array_equal(b.displacement(), u_b[k]))
        b.close()
    ps_b = sum(int(s) * n for s, n in zip(steps_b, runs["streams"]["n"]))
    t_sh = runs["shared"]["t"]
    return {"workload": f"first {nbodies} bodies of the 256-body batched workload (seed {seed}; "
                        f"{n_total} particles), FP32-mixed, KE/KE_max < {tol:g}, cap {cap} steps",
            "bodies": CONFIG4_NOTE,
            "converged": sum(conv_b), "not_converged": nbodies - sum(conv_b),
            "batched_mode": "streams (every body on its own stream, all at once)",
            "batched_s": t_batch, "shared_launches_s": t_sh, "one_at_a_time_s": t_alone,
            "batched_solves_per_s": sum(conv_b) / t_batch,
            "shared_launches_solves_per_s": sum(runs["shared"]["conv"]) / t_sh,
            "one_at_a_time_solves_per_s": sum(conv_a) / t_alone,
            "speedup": t_alone / t_batch, "shared_launches_speedup": t_alone / t_sh,
            "batched_particle_steps_per_s": ps_b / t_batch,
            "steps_min_median_max": [int(min(steps_b)), int(np.median(steps_b)), int(max(steps_b))],
            "bitwise_equal_to_alone": same,
            "shared_launches_bodies": "sliced-ELL bodies (shared launches take no lattice-stencil body)",
            "shared_launches_per_step": info["launches"] / max(1, info["steps"]),
            "sweep_cells_per_warp": info["sweep_cells_per_warp"]}


def run_served(rate, count, n_lo, n_hi, tol, max_steps, seed=4, workload_note=None):
    """Poisson request stream of uneven bodies into the continuous-batching
    server: solves/s and p50/p99 submit-to-result latency."""
    from paper_2103_08932_gb300 import srdr
    from paper_2103_08932_gb300 import synth as S
    specs = S.random_bodies(count, n_lo, n_hi, seed)
    arrivals = S.poisson_arrivals(rate, count, seed)
    srv = srdr.Server(64 << 30, ke_ratio=tol, max_steps=max_steps, max_bodies=256, chunk_steps=256)
    t0 = time.perf_counter()
    tickets = []
    for s, ta in zip(specs, arrivals):
        delay = t0 + ta - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        st, t = srv.submit(srdr.make_desc(s, precision=srdr.SRDR_FP32_MIXED))
        if st == srdr.SRDR_OK:
            tickets.append(t)
    statuses = [srv.wait(t, 3600.0)[0] for t in tickets]
    rep = srv.stats()
    srv.close()
    out = {"rate_per_s": rate, "requests": count,
           "bodies": f"particles log-uniform {int(n_lo)}-{int(n_hi)}, KE/KE_max < {tol:g}, "
                     f"cap {max_steps} steps, FP32-mixed, seed {seed}",
           "solves_per_s": rep["solves_per_s"], "p50_latency_s": rep["p50_latency_s"],
           "p99_latency_s": rep["p99_latency_s"], "peak_concurrent": rep["peak_concurrent"],
           "converged": rep["completed"], "not_converged": rep["not_converged"],
           "failed": rep["failed"],
           "particle_steps_per_s": rep["particle_steps"] / max(1e-9, time.perf_counter() - t0),
           "latency": "submit to result, converged requests only"}
    assert out["converged"] == sum(1 for s in statuses if s == srdr.SRDR_OK)
    if workload_note:
        out["note"] = workload_note
    return out


def run_block(steps, tol=1e-8, cap=20000):
    """The 0.1 m neo-Hookean cube at dp = 0.8 mm (125^3 body particles plus
    3 fixed and 3 prescribed layers, 2.05 M particles), top face at -10 %:
    FP32-mixed against an all-FP64 GPU run of the same steps, then both
    relaxed to KE/KE_max < tol (the FP32-mixed state compared at the FP64
    run's stopping step)."""
    import torch

    from paper_2103_08932_gb300 import srdr
    from paper_2103_08932_gb300 import synth as S
    spec = S.compression_block_3d()
    out = {"workload": "compression block 0.1 m, dp = 0.8 mm, 125^3 + 6 layers, neo-Hookean "
                       "E = 1e6, nu = 0.45, top -10 %, seed 2", "steps": steps}
    us = {}
    for name, prec in (("fp32_mixed", srdr.SRDR_FP32_MIXED), ("fp64", srdr.SRDR_FP64)):
        b = srdr.Body(srdr.make_desc(spec, precision=prec))
        b.step(3)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        b.step(steps - 3)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        us[name] = b.displacement()
        out[name + "_particle_steps_per_s"] = b.n * (steps - 3) / (ms / 1e3)
        out["particles"] = b.n
        out["damped_steps"] = b.stats()["damped_steps"]
        b.close()
    d = us["fp32_mixed"] - us["fp64"]
    moved = us["fp64"] - S.lattice(spec)[2]  # displacement from the initial field
    out["max_rel_displacement_error_fp32_vs_fp64"] = float(np.abs(d).max() / np.abs(us["fp64"]).max())
    out["max_rel_error_of_displacement_change"] = float(np.abs(d).max() / max(np.abs(moved).max(), 1e-300))
    # relaxed to the KE criterion
    rel = {}
    for name, prec in (("fp64", srdr.SRDR_FP64), ("fp32_mixed", srdr.SRDR_FP32_MIXED)):
        b = srdr.Body(srdr.make_desc(spec, precision=prec))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, nsteps, ratio = b.relax(tol, cap, check=False)
        torch.cuda.synchronize()
        rel[name] = {"status": srdr.STATUS_NAMES.get(st, st), "steps": nsteps, "ke_ratio": ratio,
                     "seconds": time.perf_counter() - t0, "damped_steps": b.stats()["damped_steps"]}
        if name == "fp32_mixed" and nsteps != rel["fp64"]["steps"]:
            b.close()
            b = srdr.Body(srdr.make_desc(spec, precision=prec))
            b.step(rel["fp64"]["steps"])
        us[name] = b.displacement()
        b.close()
    d = us["fp32_mixed"] - us["fp64"]
    rel["max_rel_displacement_error_fp32_vs_fp64_at_fp64_stop"] = float(np.abs(d).max() / np.abs(us["fp64"]).max())
    rel["max_displacement_m"] = float(np.abs(us["fp64"]).max())
    out["relaxed"] = rel
    return out


def run_compare(tol=1e-8, cap=200000):
    """The paper's comparisons (Sec. 4.1, 4.2): relaxation of the same bodies
    to KE/KE_max < tol with the split random-choice scheme (alpha = 0.2),
    damping at every step (alpha = 1), the explicit viscous term under its
    time-step limit, and no damping; steps, time step, simulated time and
    device time of each run."""
    import torch

    from paper_2103_08932_gb300 import srdr
    from paper_2103_08932_gb300 import synth as S
    from dataclasses import replace
    cases = [("2D cantilever 0.2 x 0.02 m, dp = 2 mm, neo-Hookean, FP64", S.cantilever_2d(S.NEO_HOOKEAN),
              srdr.SRDR_FP64),
             ("3D plate 0.1 x 0.01 x 0.05 m, dp = 1 mm (plate scaled x0.5), FP32-mixed",
              S.scaled(S.cantilever_plate_3d(), 0.5), srdr.SRDR_FP32_MIXED),
             ("3D twisting cantilever 0.2 x 0.02 x 0.02 m, dp = 1 mm, rotational body force, "
              "FP32-mixed", S.twisting_cantilever_3d(), srdr.SRDR_FP32_MIXED)]
    variants = [("split alpha=0.2", srdr.SRDR_DAMP_PARTICLE, 0.2),
                ("split alpha=1", srdr.SRDR_DAMP_PARTICLE, 1.0),
                ("explicit viscosity", srdr.SRDR_DAMP_EXPLICIT, 0.2),
                ("no damping", srdr.SRDR_DAMP_NONE, 0.2)]
    out = []
    for name, spec, prec in cases:
        rows = []
        for vname, damping, alpha in variants:
            b = srdr.Body(srdr.make_desc(replace(spec, alpha=alpha), precision=prec, damping=damping))
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            status, steps, ratio = b.relax(tol, cap, check=False)
            e1.record()
            torch.cuda.synchronize()
            st = b.stats()
            u = b.displacement()
            rows.append({"scheme": vname, "converged": status == srdr.SRDR_OK, "steps": steps,
                         "ke_ratio": ratio, "dt": st["dt"], "simulated_time_s": steps * st["dt"],
                         "device_s": e0.elapsed_time(e1) / 1e3, "damped_steps": st["damped_steps"],
                         "max_abs_displacement_m": float(np.abs(u).max())})
            b.close()
            print(json.dumps({"impl": "gpu", "compare_run": {"case": name, **rows[-1]}}), flush=True)
        out.append({"case": name, "tol": tol, "step_cap": cap, "runs": rows})
    return out


def run_strength(tol=1e-8, cap=200000):
    """Sec. 4.1's damping-strength comparison: eta = eta0, 5 eta0 and 10 eta0
    (beta = 0.2, 1, 2 in Eq. viscous-parameter), each with the random choice
    (alpha = 0.2) and damped at every step (alpha = 1), for the
    particle-by-particle scheme (Sec. 3.1) and the pairwise scheme (Sec.
    3.2): steps to KE/KE_max < tol, device time, and the static state reached
    (or the divergence, reported as it happens)."""
    import torch

    from paper_2103_08932_gb300 import srdr
    from paper_2103_08932_gb300 import synth as S
    from dataclasses import replace
    cases = [("2D cantilever 0.2 x 0.02 m, dp = 2 mm, neo-Hookean, FP64", S.cantilever_2d(S.NEO_HOOKEAN),
              srdr.SRDR_FP64, (srdr.SRDR_DAMP_PARTICLE, srdr.SRDR_DAMP_PAIRWISE)),
             ("3D plate 0.06 x 0.006 x 0.03 m, dp = 1 mm (plate scaled x0.3), FP32-mixed",
              S.scaled(S.cantilever_plate_3d(), 0.3), srdr.SRDR_FP32_MIXED, (srdr.SRDR_DAMP_PARTICLE,))]
    names = {srdr.SRDR_DAMP_PARTICLE: "particle-by-particle", srdr.SRDR_DAMP_PAIRWISE: "pairwise"}
    out = []
    for name, spec, prec, schemes in cases:
        rows = []
        for damping in schemes:
            for mult in (1, 5, 10):
                for alpha in (0.2, 1.0):
                    b = srdr.Body(srdr.make_desc(replace(spec, beta=0.2 * mult, alpha=alpha),
                                                 precision=prec, damping=damping))
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    status, steps, ratio = b.relax(tol, cap, check=False)
                    e1.record()
                    torch.cuda.synchronize()
                    st = b.stats()
                    u = b.displacement()
                    rows.append({"scheme": names[damping], "eta": f"{mult} eta0", "alpha": alpha,
                                 "status": srdr.STATUS_NAMES.get(status, status), "steps": steps,
                                 "dt": st["dt"], "simulated_time_s": steps * st["dt"],
                                 "device_s": e0.elapsed_time(e1) / 1e3,
                                 "damped_steps": st["damped_steps"],
                                 "max_abs_displacement_m": float(np.abs(u).max())})
                    b.close()
                    print(json.dumps({"impl": "gpu", "strength_run": {"case": name, **rows[-1]}}), flush=True)
        out.append({"case": name, "tol": tol, "step_cap": cap, "eta0": "beta = 0.2", "runs": rows})
    return {"damping_strength": out}


def run_layout(steps=400, warmup=20):
    """The plate with the paper's sweep layout (cells of edge r_c, 3^d = 27
    colours, 53 colour phases per damped step) and with the 2^d layout (cells
    of edge 2 r_c, 8 colours, 15 phases): per-kernel CUDA-event times of the
    stress and force passes and of the sweep per damped step."""
    import torch

    from paper_2103_08932_gb300 import srdr
    from paper_2103_08932_gb300 import synth as S
    spec = S.cantilever_plate_3d()
    out = {"workload": WORKLOAD, "steps": steps}
    for name, layout in (("3d_colours", srdr.SRDR_SWEEP_LAYOUT_3D), ("2d_colours", srdr.SRDR_SWEEP_LAYOUT_2D)):
        b = srdr.Body(srdr.make_desc(spec, precision=srdr.SRDR_FP32_MIXED, sweep_layout=layout))
        b.step(warmup)
        torch.cuda.synchronize()
        b.profile(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        b.step(steps)
        e1.record()
        torch.cuda.synchronize()
        kt = b.kernel_times()
        b.profile(False)
        st = b.stats()
        per = {k: v["ms"] / max(v["intervals"], 1) for k, v in kt.items()}
        out[name] = {"ms_per_step": e0.elapsed_time(e1) / steps, "sweep_ms_per_damped_step": per["sweep"],
                     "pass_a_ms": per["pass_a"], "pass_b_ms": per["pass_b"], "cells": b.ncells,
                     "damped_steps": kt["sweep"]["intervals"],
                     "sweep_cells_per_warp": st["sweep_cells_per_warp"],
                     "sweep_sync": st["sweep_sync"]}
        b.close()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        print(json.dumps({"impl": "gpu", "batched": run_batched(256, 1e3, 2e5, args.steps, sync=args.sweep_sync)}))
    elif args.workload == "block":
        print(json.dumps({"impl": "gpu", "block": run_block(args.steps)}))
    elif args.workload == "compare":
        print(json.dumps({"impl": "gpu", "compare": run_compare(cap=args.compare_cap)}))
    elif args.workload == "strength":
        print(json.dumps({"impl": "gpu", **run_strength(cap=args.compare_cap)}))
    elif args.workload == "layout":
        print(json.dumps({"impl": "gpu", "layout": run_layout(args.steps, args.warmup)}))
    elif args.workload == "served":
        out = [run_served(r, args.requests, 1e3, args.served_max_n, args.served_tol,
                          args.served_max_steps) for r in args.rates]
        print(json.dumps({"impl": "gpu", "served": out}))
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
