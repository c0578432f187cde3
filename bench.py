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
    return ap.parse_args()


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
    """Compulsory HBM bytes per launch of the FP32-mixed kernels: every array
    the kernel must touch, once.  Neighbour gathers re-read arrays already
    counted (they are meant to hit L2)."""
    pairs = 16 * nnz  # sliced-ELL stream per pair: col int32 + V_j gradW (3 x fp32)
    pass_a = pairs + n * (32 + 36 + 48)  # u hi/lo (2 x float4), B0 (9 f32), PB out (3 x float4)
    pass_b = pairs + n * (48 + 12 + 24 + 64 + 1 + 4)  # PB, G, v r/w, u hi/lo r/w, flags, mass
    return {"pass_a": pass_a, "pass_b": pass_b}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------- CPU baseline (oracle)
def oracle_rate(spec, steps, seed_steps=0):
    """Time the FP64 oracle on `steps` steps of `spec`; returns (p-steps/s, n, seconds)."""
    from oracle import oracle as O
    from paper_2103_08932_gb300 import synth as S
    r0, flags, u0 = S.lattice(spec)
    b = O.OracleBody(O.Params(dim=spec.dim, material=spec.material, rho0=spec.rho0, E=spec.E,
                              nu=spec.nu, h=spec.h, gravity=spec.gravity, beta=spec.beta,
                              L_char=spec.L_char, alpha=spec.alpha, seed=spec.seed),
                     r0, vol_default=spec.vol, flags=flags)
    if seed_steps:
        b.step(seed_steps)
    t = time.perf_counter()
    b.step(steps)
    el = time.perf_counter() - t
    return b.n * steps / el, b.n, el, b.damped_steps


def cpu_baseline():
    from paper_2103_08932_gb300 import synth as S
    spec = S.cantilever_plate_3d()
    # bounded sample: the full 406,000-particle plate, steps 0..7 (step 7 is
    # the first damped step of seed 1), about 10-20 s of single-thread CPU work
    rate, n, el, damped = oracle_rate(spec, 8)
    return {"value": rate, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"full plate ({n} particles), 8 time steps incl. {damped} damped, "
                      f"FP64 single-thread C oracle, {el:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2103_08932_gb300 import synth as S
    # each step: one oracle time step of a scaled copy of the plate (same dp,
    # same physics), sized so that W + K steps take about 90 s on one core
    full = S.cantilever_plate_3d()
    probe = S.scaled(full, 0.25)
    r_probe, n_probe, _, _ = oracle_rate(probe, 2)
    budget = 90.0 / max(1, args.steps + args.warmup)
    n_target = max(2000, min(406000, r_probe * budget))
    f = max(0.12, min(1.0, (n_target / 406000.0) ** (1.0 / 3.0)))
    spec = S.scaled(full, f)
    rate, n, el, damped = oracle_rate(spec, args.steps, seed_steps=args.warmup)
    ms = el / args.steps * 1e3
    out = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "reference_sample": f"plate scaled x{f:.3f} ({n} particles)"},
        "cpu_baseline": {"value": rate, "unit": METRIC, "cores": 1, "kind": "oracle",
                         "sample": f"plate scaled x{f:.3f} ({n} particles), {args.steps} steps "
                                   f"({damped} damped) after {args.warmup} warm-up steps"},
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

    body.step(args.warmup)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.2)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    st0 = body.stats()
    body.profile(True)
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
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    n = body.n
    value = world * n * args.steps / (ms / 1e3)
    launches = int(st1["launches"] - st0["launches"])
    damped = int(st1["damped_steps"] - st0["damped_steps"])

    # roofline of the dominant kernel class
    peak, peak_kind = load_peaks()
    ab = algorithmic_bytes(n, body.nnz)
    per = {k: (v["ms"] / max(v["intervals"], 1)) for k, v in kt.items()}
    dom = max(("pass_a", "pass_b"), key=lambda k: kt[k]["ms"])
    achieved = ab[dom] / (per[dom] / 1e3) / 1e9
    traffic = None
    tf = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tf):
        try:
            with open(tf) as fh:
                traffic = json.load(fh).get(dom)
        except (OSError, ValueError):
            traffic = None

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
                       "l2": "working set ~0.9 GB > 129 MB L2 (no flush)"},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": peak_kind, "algorithmic_bytes": ab[dom]},
            "kernels_ms_per_launch": per,
            "kernels_ms_total": {k: v["ms"] for k, v in kt.items()},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(out))
    body.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
