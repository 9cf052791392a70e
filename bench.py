#!/usr/bin/env python
"""Benchmark of the RTM hot path on GB300.

Workload (one "step" = one pass of the whole path): reverse time migration of
96 shots over the 1701 x 351 layered/faulted model at 10 m (20-cell sponge),
10 Hz Ricker, dt = 1 ms, 5000 steps, FP32 source snapshots every 4 steps,
source-normalised imaging, Kahan stack, Laplacian filter.  Observed data are
modelled once (untimed) by the library with the true model; migration uses a
60 m Gaussian-smoothed model, as the paper's scalability runs migrate with a
smoothed velocity.  All data are synthetic (seeded).

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload instead.  Under torchrun every rank
migrates its own copy of the workload on its own GPU (weak scaling, no
data-path collective); rank 0 prints max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2001_06444_gb300.sharding import barrier, max_over_ranks  # noqa: E402

METRIC = "RTM shots/s & Gpt-updates/s vs HBM roofline; p50/p99 latency, mixed stream"
WORKLOAD = "rtm_1701x351_96shots_nt5000_isnap4_f32snap"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--batch", type=int, default=0, help="items in flight (0 = memory budget)")
    p.add_argument("--snap", default="f32", choices=["f32", "bf16", "f16"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    # smaller cases of the same workload, for profiler captures only
    p.add_argument("--shots", type=int, default=96)
    p.add_argument("--nt", type=int, default=5000)
    return p.parse_args()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")
    return world, rank, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profile_traffic():
    """Per-update DRAM bytes of the step kernel from the committed ncu summary,
    if it was taken on the current kernel source; else None."""
    import hashlib

    src = os.path.join(ROOT, "paper_2001_06444_gb300", "csrc", "rtm_prop.cu")
    summ = os.path.join(ROOT, "profiles", "k_step_full_size.md")
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        for line in open(summ):
            if line.startswith("traffic_bytes_per_update:"):
                parts = line.split()
                if len(parts) >= 4 and parts[3] == h:
                    return float(parts[1])
    except OSError:
        pass
    return None


class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 6:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[2:6]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(survey, vel_mig, nshot=2, nt=None):
    """The FP64 oracle, as it stands, migrating `nshot` shots of the workload
    (forward, backward, imaging every 4 steps, filter) over `nt` time steps
    (all of them by default).  Returns (shots/s, seconds, threads); with
    nt < survey.nt the rate is extrapolated linearly in steps."""
    import oracle

    nt = survey.nt if nt is None else nt
    g = oracle.grid(survey.nx, survey.nz, survey.nb, survey.dx, survey.dz, survey.dt, nt)
    seis = np.zeros((nshot, nt, survey.nrec))
    seis[:, :, survey.nrec // 2] = 1e-6 * np.sin(0.05 * np.arange(nt))[None, :]
    t = time.perf_counter()
    oracle.migrate(g, vel_mig, survey.src_ix[:nshot], survey.src_iz[:nshot], survey.rec_ix,
                   survey.rec_iz, survey.wavelet[:nt], seis, isnap=4)
    dt = time.perf_counter() - t
    return nshot * (nt / survey.nt) / dt, dt, oracle.threads()


def run_reference(args, world, rank):
    from paper_2001_06444_gb300 import inputs

    if rank != 0:
        return
    s = inputs.full_size()
    vm = inputs.smooth(s.vel, s.dx, s.dz, 60.0)
    for _ in range(args.warmup):
        cpu_baseline(s, vm, nshot=1, nt=100)
    secs, shots, cores = 0.0, 0, 1
    for _ in range(args.steps):
        _, dt, cores = cpu_baseline(s, vm, nshot=2)
        secs += dt
        shots += 2
    value = shots / secs
    sample = "2 of the 96 shots per step, all 5000 steps (fwd+bwd+imaging, FP64)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "shots/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD},
        "cpu_baseline": {"value": value, "unit": "shots/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "shots/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_native(args, world, rank, local):
    import torch

    from paper_2001_06444_gb300 import inputs, rtm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s = inputs.full_size(nshot=args.shots, nt=args.nt)
    vm = inputs.smooth(s.vel, s.dx, s.dz, 60.0)
    grid = rtm.make_grid(*s.grid_tuple())
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    snap = {"f32": rtm.SNAP_F32, "bf16": rtm.SNAP_BF16, "f16": rtm.SNAP_F16}[args.snap]
    opts = rtm.Opts(4, snap, 1e-6, 1)

    vel_true = torch.from_numpy(s.vel.astype(np.float32)).to(dev)
    vel_mig = torch.from_numpy(vm.astype(np.float32)).to(dev)
    seis = torch.empty((s.nshot, s.nt, s.nrec), dtype=torch.float32, device=dev)
    image = torch.empty((s.nz, s.nx), dtype=torch.float32, device=dev)
    ctx = rtm.Context(local)
    ctx.model(grid, vel_true, acq, -1, seis)  # observed data, untimed
    torch.cuda.synchronize()
    if args.batch:
        ctx.set_batch(args.batch)
    for _ in range(args.warmup):
        ctx.migrate(grid, vel_mig, acq, seis, opts, image)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    ctx.set_profiling(True)
    ctx.stats(reset=True)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        ctx.migrate(grid, vel_mig, acq, seis, opts, image)
    e1.record(st)
    torch.cuda.synchronize()
    barrier(world)
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    stats = ctx.stats(reset=True)
    ctx.set_profiling(False)
    ms = max_over_ranks(ms, world)

    shots = s.nshot * args.steps * world
    value = shots / (ms / 1e3)
    gpt = stats["point_updates"] * world / (ms / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    achieved = stats["step_bytes"] / (stats["step_ms"] / 1e3) / 1e9 if stats["step_ms"] else None
    per_update = profile_traffic()
    launches_step = stats["step_launches"]
    traffic = None
    if per_update is not None and launches_step:
        traffic = per_update * stats["point_updates"] / launches_step

    # end to end through the C ABI with host buffers: the call stages the
    # velocity and the data to the device and returns the image to the host
    e2e = None
    if not args.no_e2e:
        h_seis = seis.cpu().pin_memory()
        h_vel = vel_mig.cpu().pin_memory()
        h_img = torch.empty((s.nz, s.nx), dtype=torch.float32).pin_memory()
        barrier(world)
        t = time.perf_counter()
        for _ in range(args.steps):
            ctx.migrate(grid, h_vel, acq, h_seis, opts, h_img)
        dt = max_over_ranks(time.perf_counter() - t, world)
        e2e = {"value": shots / dt, "unit": "shots/s",
               "h2d_bytes_per_step": int(h_seis.numel() * 4 + h_vel.numel() * 4),
               "d2h_bytes_per_step": int(h_img.numel() * 4)}
        del h_seis

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt, cores = cpu_baseline(s, vm, nshot=2)
        cpu = {"value": v, "unit": "shots/s", "cores": cores, "kind": "oracle",
               "sample": f"2 of the {s.nshot} shots, all {s.nt} steps (fwd+bwd+imaging, FP64), "
                         f"{dt:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "shots/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if (s.nshot, s.nt) == (96, 5000)
                       else f"rtm_1701x351_{s.nshot}shots_nt{s.nt}_isnap4_{args.snap}snap", "grid": "1701x351 +20 sponge, 10 m", "shots": s.nshot,
                       "nt": s.nt, "isnap": 4, "snap_dtype": args.snap,
                       "items_in_flight": args.batch or "memory budget",
                       "l2": "inputs larger than L2 (3.0 GB snapshot store per shot)",
                       "parallelism": f"weak x{world}, independent migrations per GPU"},
            "gpt_updates_per_s": gpt,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                         "kernel": "k_step (forward+backward phases)",
                         "peak_kind": f"{peak_kind} hbm_gbs",
                         "algorithmic_bytes_per_launch": stats["step_bytes"] / max(1, launches_step),
                         "avg_launch_us": 1e3 * stats["step_ms"] / max(1, launches_step)},
            "e2e": e2e, "cpu_baseline": cpu, "clocks": ck,
            "gpu_launches": int(stats["launches"]),
        }
        print(json.dumps(line), flush=True)
    ctx.close()


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_native(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
