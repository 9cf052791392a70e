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
STEP_KERNEL_NAMES = {
    4: "k_step2a (two-step TMA kernel, one tile per block, v^{n+1} over v^n; forward+backward "
       "phases)",
    3: "k_step2p (persistent two-step TMA kernel, two-stage copy ring; forward+backward phases)",
    2: "k_step2 (two-step TMA kernel, one tile per block; forward+backward phases)",
    1: "k_step (single-step kernel; forward+backward phases)",
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--batch", type=int, default=0, help="items in flight (0 = memory budget)")
    # a fixed launch configuration instead of the autotuner's choice (for
    # comparisons and profiler captures of one kernel)
    p.add_argument("--kernel", type=int, default=0, choices=[0, 1, 2, 3, 4],
                   help="0 autotune; 1 single-step; 2 two-step, one tile per block; "
                        "3 persistent two-step; 4 two-step, one tile per block, v^{n+1} over v^n")
    p.add_argument("--tile-z", type=int, default=24, choices=[16, 24, 32],
                   help="with --kernel 3 (16, 24) or 4 (24, 32): centre rows of a tile")
    p.add_argument("--graphs", type=int, default=1, choices=[0, 1],
                   help="with --kernel 1-3: capture each phase in a CUDA graph")
    p.add_argument("--pdl", type=int, default=0, choices=[0, 1],
                   help="with --kernel 4: programmatic dependent launches")
    p.add_argument("--image-input", type=int, default=0, choices=[0, 1],
                   help="with --kernel 2-4: backward launches image their input field")
    p.add_argument("--l2-ahead", type=int, default=0, choices=[0, 1],
                   help="with --kernel 2: each block prefetches a later block's tile into L2")
    p.add_argument("--snap", default="f32", choices=["f32", "bf16", "f16"])
    p.add_argument("--checkpoint", type=int, default=0,
                   help="0 keep every snapshot; C>0 / -1 recompute from checkpoints")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-serve", action="store_true", help="skip the mixed-stream latency run")
    # smaller cases of the same workload, for profiler captures only
    p.add_argument("--shots", type=int, default=96)
    p.add_argument("--nt", type=int, default=5000)
    # other workloads of the method, each printing its own JSON line
    p.add_argument("--workload", default="migrate",
                   choices=["migrate", "ensemble", "serve", "codec", "eikonal", "stats", "born",
                            "lsrtm"])
    p.add_argument("--samples", type=int, default=64, help="ensemble: velocity samples")
    p.add_argument("--requests", type=int, default=64, help="serve: requests in the stream")
    p.add_argument("--rate", type=float, default=0.0, help="serve: arrivals/s (0 = 0.8 x capacity)")
    p.add_argument("--iters", type=int, default=2, help="lsrtm: CGLS iterations per step")
    p.add_argument("--serve-snap", default="f16", choices=["f16", "bf16"],
                   help="serve: snapshot format of the batched, served form")
    p.add_argument("--serve-plain", type=int, default=1, choices=[0, 1],
                   help="serve: also time the plain form (0 skips it; no batched/plain ratio)")
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


def step_sources_digest():
    """Hash of the propagation kernels' sources (the ncu summaries record it)."""
    import hashlib

    h = hashlib.sha256()
    for f in ("rtm_prop.cu", "rtm_prop2.cu", "rtm_prop2p.cu", "rtm_step2_dev.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2001_06444_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profile_traffic(kernel):
    """DRAM bytes per point update of step kernel `kernel` (e.g. "k_step2a")
    from the committed ncu summaries under profiles/, if one was taken on the
    current kernel sources; else None.  A summary carries the line
    `traffic_bytes_per_update: <B> <sources digest> <kernel>`."""
    import glob

    digest = step_sources_digest()
    for summ in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        try:
            for line in open(summ):
                if line.startswith("traffic_bytes_per_update:"):
                    parts = line.split()
                    if len(parts) >= 4 and parts[2] == digest and parts[3] == kernel:
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
    # a created stream: the library captures each phase of a batch as a CUDA
    # graph there (never on the legacy default stream)
    torch.cuda.set_stream(torch.cuda.Stream(dev))
    s = inputs.full_size(nshot=args.shots, nt=args.nt)
    vm = inputs.smooth(s.vel, s.dx, s.dz, 60.0)
    grid = rtm.make_grid(*s.grid_tuple())
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    snap = {"f32": rtm.SNAP_F32, "bf16": rtm.SNAP_BF16, "f16": rtm.SNAP_F16}[args.snap]
    opts = rtm.Opts(4, snap, 1e-6, 1, args.checkpoint)

    vel_true = torch.from_numpy(s.vel.astype(np.float32)).to(dev)
    vel_mig = torch.from_numpy(vm.astype(np.float32)).to(dev)
    seis = torch.empty((s.nshot, s.nt, s.nrec), dtype=torch.float32, device=dev)
    image = torch.empty((s.nz, s.nx), dtype=torch.float32, device=dev)
    if args.kernel:
        # the context's default launch configuration, read when it is created
        os.environ["RTM_STEP_KERNEL"] = str(args.kernel)
        os.environ["RTM_TILE_Z"] = str(args.tile_z)
        os.environ["RTM_GRAPHS"] = str(args.graphs)
        os.environ["RTM_L2_AHEAD"] = str(args.l2_ahead)
        os.environ["RTM_IMAGE_INPUT"] = str(args.image_input)
        os.environ["RTM_PDL"] = str(args.pdl)
    ctx = rtm.Context(local)
    ctx.model(grid, vel_true, acq, -1, seis)  # observed data, untimed
    torch.cuda.synchronize()
    if args.batch:
        ctx.set_batch(args.batch)
    if args.kernel:
        tuned = {"step_kernel": args.kernel, "max_items": args.batch, "graph": args.graphs,
                 "tile_z": args.tile_z if args.kernel in (3, 4) else 24,
                 "l2_ahead": args.l2_ahead if args.kernel == 2 else 0,
                 "image_input": args.image_input, "pdl": args.pdl, "fixed": True}
    else:
        tuned = ctx.autotune(grid, acq, opts, trial_steps=64)  # untimed: picks the launch config
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
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed launches
    e0.record(st)
    for _ in range(args.steps):
        ctx.migrate(grid, vel_mig, acq, seis, opts, image)
    e1.record(st)
    torch.cuda.nvtx.range_pop()
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
    kname = STEP_KERNEL_NAMES.get(tuned.get("step_kernel"), "k_step").split()[0]
    per_update = profile_traffic(kname)
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
        # one untimed call sizes the staging buffers in the context's pool
        ctx.migrate(grid, h_vel, acq, h_seis, opts, h_img)
        barrier(world)
        t = time.perf_counter()
        calls = []
        for _ in range(args.steps):
            c0 = time.perf_counter()
            ctx.migrate(grid, h_vel, acq, h_seis, opts, h_img)
            calls.append(round(time.perf_counter() - c0, 4))
        dt = max_over_ranks(time.perf_counter() - t, world)
        e2e = {"value": shots / dt, "unit": "shots/s",
               "h2d_bytes_per_step": int(h_seis.numel() * 4 + h_vel.numel() * 4),
               "d2h_bytes_per_step": int(h_img.numel() * 4), "call_s": calls}
        del h_seis

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        v, dt, cores = cpu_baseline(s, vm, nshot=2)
        cpu = {"value": v, "unit": "shots/s", "cores": cores, "kind": "oracle",
               "sample": f"2 of the {s.nshot} shots, all {s.nt} steps (fwd+bwd+imaging, FP64), "
                         f"{dt:.1f} s"}
        oracle.set_threads(1)
        v1, dt1, _ = cpu_baseline(s, vm, nshot=1, nt=300)
        oracle.set_threads(cores)
        cpu["single_thread_value"] = v1
        cpu["single_thread_sample"] = (f"1 shot, 300 of {s.nt} steps on 1 thread, {dt1:.1f} s, "
                                       f"extrapolated linearly in steps")

    ctx.close()
    serving = None
    if world == 1 and not args.no_serve:
        del seis, vel_true, vel_mig, image
        torch.cuda.empty_cache()
        sv = serve_measurement(local, 32, snap_name=args.serve_snap)
        serving = {"workload": "mixed stream: 32 Poisson requests, grids 201x101..2401x601, "
                               f"1-32 shots, 2000-6000 steps, {args.serve_snap.upper()} snapshots",
                   "p50_latency_s": sv["served"]["p50_latency_s"],
                   "p99_latency_s": sv["served"]["p99_latency_s"],
                   "arrival_rate_per_s": sv["arrival_rate_per_s"],
                   "served_shots_per_s": sv["served"]["shots_per_s"],
                   "batched_capacity_shots_per_s": sv["batched_capacity"]["shots_per_s"],
                   "batched_capacity_gpt_updates_per_s": sv["batched_capacity"]["gpt_updates_per_s"],
                   "plain_fp32_one_shot_shots_per_s": sv["plain_fp32_one_shot"]["shots_per_s"],
                   "batched_vs_plain": sv["speedup_batched_vs_plain"],
                   "failed_requests": sv["served"]["failed"] + sv["batched_capacity"]["failed"],
                   "image_rel_l2_vs_plain_max": sv["image_rel_l2_vs_plain_max"]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "shots/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if (s.nshot, s.nt) == (96, 5000)
                       else f"rtm_1701x351_{s.nshot}shots_nt{s.nt}_isnap4_{args.snap}snap", "grid": "1701x351 +20 sponge, 10 m", "shots": s.nshot,
                       "nt": s.nt, "isnap": 4, "snap_dtype": args.snap,
                       "checkpoint": args.checkpoint,
                       "items_in_flight": args.batch or "memory budget",
                       "launch_config": tuned,
                       "graph_launches_timed": int(stats["graph_launches"]),
                       "stream": "created (graph capture applies)",
                       "l2": "inputs larger than L2 (3.0 GB snapshot store per shot)",
                       "parallelism": f"weak x{world}, independent migrations per GPU"},
            "gpt_updates_per_s": gpt,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                         "kernel": STEP_KERNEL_NAMES.get(tuned.get("step_kernel"), "k_step"),
                         "peak_kind": f"{peak_kind} hbm_gbs",
                         "algorithmic_bytes_per_launch": stats["step_bytes"] / max(1, launches_step),
                         "avg_launch_us": 1e3 * stats["step_ms"] / max(1, launches_step)},
            "e2e": e2e, "cpu_baseline": cpu, "clocks": ck,
            "gpu_launches": int(stats["launches"]),
            "serving": serving,
        }
        print(json.dumps(line), flush=True)


def _survey_request(spec, snap, dev):
    """A request of the mixed stream: data modelled once with the true model,
    migrated with a 60 m smoothed one."""
    import torch

    from paper_2001_06444_gb300 import inputs, rtm

    s = inputs.scaled_survey(spec["nx"], spec["nz"], spec["nshot"], spec["nt"], spec["f"],
                             spec["seed"])
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    grid = rtm.make_grid(*s.grid_tuple())
    vt = torch.from_numpy(s.vel.astype(np.float32)).to(dev)
    vm = torch.from_numpy(inputs.smooth(s.vel, s.dx, s.dz, 60.0).astype(np.float32)).to(dev)
    seis = torch.empty((s.nshot, s.nt, s.nrec), dtype=torch.float32, device=dev)
    img = torch.zeros((s.nz, s.nx), dtype=torch.float32, device=dev)
    return dict(s=s, keep=keep, acq=acq, grid=grid, vt=vt, vm=vm, seis=seis, img=img,
                opts=rtm.Opts(4, snap, 1e-6, 1))


def serve_measurement(local, nreq, rate_arg=0.0, snap_name="f16", plain=True):
    """Poisson stream of mixed migration requests through rtm_submit/rtm_poll
    (continuous batching, half-precision snapshots: FP16 by default, which
    keeps the served images within 1e-2 of the plain form; BF16 does not on
    this mix), against the plain form: the same requests one after another,
    one shot per launch sequence, FP32 snapshots.  Returns a dict; the stream
    is the seeded one of inputs.request_stream."""
    import torch

    from paper_2001_06444_gb300 import inputs, rtm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    specs = inputs.request_stream(nreq, rate_hz=1.0)
    snap = {"bf16": rtm.SNAP_BF16, "f16": rtm.SNAP_F16}[snap_name]
    reqs = [_survey_request(sp, snap, dev) for sp in specs]
    # the context's default budget is a share of the memory free when it is
    # created: create it after the requests' data (86 GB at 256 requests)
    ctx = rtm.Context(local)
    for r in reqs:
        ctx.model(r["grid"], r["vt"], r["acq"], -1, r["seis"])
    torch.cuda.synchronize()
    total_shots = sum(r["s"].nshot for r in reqs)
    # padded point updates of the whole stream (forward + backward)
    total_upd = sum(2.0 * r["s"].nshot * r["s"].nt * (r["s"].nz + 2 * r["s"].nb) *
                    (r["s"].nx + 2 * r["s"].nb) for r in reqs)
    # plain form: one request at a time, one shot in flight, FP32 snapshots
    plain_s, plain_img = None, None
    if plain:
        ctx.set_batch(1)
        t = time.perf_counter()
        for r in reqs:
            ctx.migrate(r["grid"], r["vm"], r["acq"], r["seis"],
                        rtm.Opts(4, rtm.SNAP_F32, 1e-6, 1), r["img"])
        torch.cuda.synchronize()
        plain_s = time.perf_counter() - t
        ctx.set_batch(0)
        plain_img = [r["img"].clone() for r in reqs]

    def serve(gaps_s):
        """Submit request i after gaps_s[i] seconds; returns (wall, latencies).
        Outstanding requests are polled while later ones wait to be submitted,
        so a latency ends when its request ends, not when submitting does."""
        for r in reqs:
            r["img"].zero_()
        torch.cuda.synchronize()
        tickets = []
        done = {}
        errors = []
        pending = []

        def sweep():
            for item in list(pending):
                tk, sub = item
                st, _ = ctx.poll(tk, 0)
                if st in (rtm.REQ_DONE, rtm.REQ_FAILED):
                    done[tk] = (st, time.perf_counter() - sub)
                    pending.remove(item)
                    if st == rtm.REQ_FAILED:
                        errors.append(ctx.last_error())

        t0 = time.perf_counter()
        due = t0
        for r, gap in zip(reqs, gaps_s):
            due += gap
            while time.perf_counter() < due:
                sweep()
                time.sleep(0.0002)
            sub = time.perf_counter()
            req = rtm.Request(r["grid"], r["vm"].data_ptr(), r["acq"], r["seis"].data_ptr(),
                              r["opts"], r["img"].data_ptr())
            tickets.append((ctx.submit(req), sub))
            pending.append(tickets[-1])
        while pending:
            sweep()
            time.sleep(0.0002)
        wall = time.perf_counter() - t0
        torch.cuda.synchronize()
        failed = sum(1 for v in done.values() if v[0] != rtm.REQ_DONE)
        if errors:
            print(f"serve: {failed} requests failed, first: {errors[0]}", file=sys.stderr)
        subs = np.array([sub - t0 for _, sub in tickets])
        return wall, np.array([done[tk][1] for tk, _ in tickets]), failed, subs

    # batched capacity: every request submitted at once
    cap_wall, _, cap_failed, _ = serve(np.zeros(len(reqs)))
    capacity = len(reqs) / cap_wall
    rate = rate_arg or 0.8 * capacity
    unit_gaps = np.diff([0.0] + [sp["t"] for sp in specs])  # unit-rate Poisson gaps
    served_s, lat, failed, subs = serve(unit_gaps / rate)
    # the slowest requests: size, arrival and latency
    work = [2.0 * sp["nshot"] * sp["nt"] * (sp["nz"] + 40) * (sp["nx"] + 40) for sp in specs]
    slowest = [{"grid": f'{specs[i]["nx"]}x{specs[i]["nz"]}', "shots": specs[i]["nshot"],
                "nt": specs[i]["nt"], "gupdates": round(work[i] / 1e9, 1),
                "arrived_s": round(float(subs[i]), 2), "latency_s": round(float(lat[i]), 2)}
               for i in np.argsort(-lat)[:8]]
    errs = []
    for r, p in zip(reqs, plain_img or []):
        a, b = r["img"].double(), p.double()
        errs.append(float(torch.linalg.norm(a - b) / torch.linalg.norm(b)))
    line = {
        "workload": "serve_mixed_stream", "requests": len(reqs), "shots": total_shots,
        "arrival_rate_per_s": rate, "snap_dtype": snap_name,
        "batched_capacity": {"shots_per_s": total_shots / cap_wall, "wall_s": cap_wall,
                             "gpt_updates_per_s": total_upd / cap_wall / 1e9,
                             "failed": cap_failed},
        "served": {"shots_per_s": total_shots / served_s, "wall_s": served_s,
                   "p50_latency_s": float(np.percentile(lat, 50)),
                   "p99_latency_s": float(np.percentile(lat, 99)), "failed": failed},
        "slowest_requests": slowest,
        "plain_fp32_one_shot": ({"shots_per_s": total_shots / plain_s, "wall_s": plain_s,
                                 "gpt_updates_per_s": total_upd / plain_s / 1e9}
                                if plain_s else None),
        "speedup_batched_vs_plain": (plain_s / cap_wall) if plain_s else None,
        "image_rel_l2_vs_plain_max": max(errs) if errs else None,
        "grids": sorted({(sp["nx"], sp["nz"]) for sp in specs}),
    }
    ctx.close()
    del reqs
    torch.cuda.empty_cache()
    return line


def run_serve(args, local):
    print(json.dumps(serve_measurement(local, args.requests, args.rate, args.serve_snap,
                                       plain=bool(args.serve_plain))), flush=True)


def run_ensemble(args, world, rank, local):
    """All (sample, shot) migrations of a velocity ensemble in one call, then
    the per-pixel statistics of the images.  Under torchrun each rank
    migrates a contiguous share of the samples; the statistics then take the
    pixel-slab exchange (over gloo, through host copies)."""
    import torch

    from paper_2001_06444_gb300 import inputs, rtm
    from paper_2001_06444_gb300.sharding import share, sharded_ensemble_stats

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s = inputs.full_size(nshot=args.shots, nt=args.nt)
    vm = inputs.smooth(s.vel, s.dx, s.dz, 60.0)
    ens = inputs.ensemble(vm, s.dx, s.dz, args.samples)
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    grid = rtm.make_grid(*s.grid_tuple())
    snap = {"f32": rtm.SNAP_F32, "bf16": rtm.SNAP_BF16, "f16": rtm.SNAP_F16}[args.snap]
    ctx = rtm.Context(local)
    vt = torch.from_numpy(s.vel.astype(np.float32)).to(dev)
    seis = torch.empty((s.nshot, s.nt, s.nrec), dtype=torch.float32, device=dev)
    ctx.model(grid, vt, acq, -1, seis)
    a, b = share(args.samples, rank, world)
    vels = torch.from_numpy(ens[a:b].astype(np.float32)).to(dev)
    imgs = torch.empty((b - a, s.nz, s.nx), dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    ctx.set_profiling(True)
    ctx.stats(reset=True)
    barrier(world)
    t = time.perf_counter()
    ctx.migrate_ensemble(grid, vels, acq, seis, rtm.Opts(4, snap, 1e-6, 1), imgs)
    torch.cuda.synchronize()
    mig_s = max_over_ranks(time.perf_counter() - t, world)
    st = ctx.stats(reset=True)
    npix = s.nz * s.nx

    def gpu_stats(slab):
        d = slab.to(dev).contiguous()
        outs = [torch.empty(d.shape[1], dtype=tp, device=dev)
                for tp in (torch.float64, torch.float64, torch.float32, torch.float32)]
        ctx.ensemble_stats(d, *outs)
        return [o.cpu() if world > 1 else o for o in outs]

    barrier(world)
    t = time.perf_counter()
    local = imgs.reshape(b - a, npix)
    sharded_ensemble_stats(local.cpu() if world > 1 else local, args.samples, rank, world,
                           gpu_stats)
    torch.cuda.synchronize()
    stats_s = max_over_ranks(time.perf_counter() - t, world)
    peak, _ = measured_peaks()
    achieved = st["step_bytes"] / (st["step_ms"] / 1e3) / 1e9
    if rank == 0:
        line = {
            "workload": f"ensemble_{args.samples}x{s.nshot}_1701x351_nt{s.nt}_{args.snap}snap",
            "n_gpus": world, "migrations": args.samples * s.nshot, "migration_s": mig_s,
            "shots_per_s": args.samples * s.nshot / mig_s,
            "gpt_updates_per_s": st["point_updates"] * world / mig_s / 1e9,
            "step_kernel_gbs": achieved, "frac_of_measured_hbm": achieved / peak,
            "stats_ms": 1e3 * stats_s,
        }
        print(json.dumps(line), flush=True)
    ctx.close()


def paper_compression_tables():
    """{(array, tol): size / raw} as printed in §4.2, Tables 1-2 (a sorted
    pair where the paper gives the smallest and largest of 160 files), from
    the cited fixture tests/golden/paper_compression_tables.txt."""
    out = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "paper_compression_tables.txt")):
        f = line.split("#")[0].split()
        if f:
            out.setdefault((f[0], float(f[1])), []).append(float(f[3]) / float(f[2]))
    return {k: (v[0] if len(v) == 1 else tuple(sorted(v))) for k, v in out.items()}


def run_codec(args, local):
    """Throughput and ratios of the device codec on the workflow's arrays
    (§4.2, Tables 1-2): the survey's seismograms (96 x 5000 x 1701, modelled
    with the true model), a 64-sample velocity ensemble and migrated images
    (two samples' images, repeated to a batch of 64), at the paper's
    tolerances (1e-4, 1e-1) and lossless.  Kernel time from CUDA events
    around each codec launch; roofline bytes = floats read or written plus
    stream bytes written or read."""
    import torch

    from paper_2001_06444_gb300 import inputs, rtm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s = inputs.full_size(nshot=args.shots, nt=args.nt)
    vm = inputs.smooth(s.vel, s.dx, s.dz, 60.0)
    ens = inputs.ensemble(vm, s.dx, s.dz, 64).astype(np.float32)
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    grid = rtm.make_grid(*s.grid_tuple())
    ctx = rtm.Context(local)
    seis = torch.empty((s.nshot, s.nt, s.nrec), dtype=torch.float32, device=dev)
    ctx.model(grid, torch.from_numpy(s.vel.astype(np.float32)).to(dev), acq, -1, seis)
    vels = torch.from_numpy(ens).to(dev)
    two = torch.empty((2, s.nz, s.nx), dtype=torch.float32, device=dev)
    ctx.migrate_ensemble(grid, vels[:2].contiguous(), acq, seis, rtm.Opts(4, rtm.SNAP_F16, 1e-6, 1),
                         two)
    imgs = two.repeat(32, 1, 1).contiguous()
    torch.cuda.synchronize()
    peak, peak_kind = measured_peaks()
    paper = paper_compression_tables()  # Tables 1-2 (Marmousi2 files): context only
    cases = []
    clocks = Clocks(local)
    clocks.start()
    for kind, arr, tols in (("seismogram", seis, (1e-4, 0.0)), ("image", imgs, (1e-1, 1e-4, 0.0)),
                            ("velocity", vels, (1e-1, 1e-4, 0.0))):
        count, n0, n1 = arr.shape
        raw = arr.numel() * 4
        stride = (rtm.compress_bound(n0, n1) + 15) // 16 * 16
        out = torch.empty(count * stride, dtype=torch.uint8, device=dev)
        dec = torch.empty_like(arr)
        for tol in tols:
            for _ in range(args.warmup):
                _, _, sizes = ctx.compress(arr, tol, out, stride)
                ctx.decompress(out, stride, count, n0, n1, dec)
            torch.cuda.synchronize()
            ctx.set_profiling(True)
            ctx.stats(reset=True)
            for _ in range(args.steps):
                _, _, sizes = ctx.compress(arr, tol, out, stride)
            enc = ctx.stats(reset=True)
            for _ in range(args.steps):
                ctx.decompress(out, stride, count, n0, n1, dec)
            decs = ctx.stats(reset=True)
            ctx.set_profiling(False)
            err = float((dec - arr).abs().max()) if tol > 0 else None
            exact = bool(torch.equal(dec.view(torch.int32), arr.view(torch.int32))) if tol == 0 \
                else None
            comp = float(sum(sizes))
            frac = comp / raw
            enc_s = enc["codec_ms"] / 1e3 / args.steps
            dec_s = decs["codec_ms"] / 1e3 / args.steps
            c = {"array": kind, "shape": [count, n0, n1], "tol": tol,
                 "size_frac": frac, "ratio": raw / comp,
                 "paper_size_frac": paper.get((kind, tol)),
                 "compress_gbs": raw / enc_s / 1e9, "decompress_gbs": raw / dec_s / 1e9,
                 "compress_roofline_frac": (raw + comp) / enc_s / 1e9 / peak,
                 "decompress_roofline_frac": (raw + comp) / dec_s / 1e9 / peak,
                 "max_abs_err": err, "lossless_exact": exact}
            cases.append(c)
    ck = clocks.stop()

    # the paper's compression-error experiment (§4.2): migrate the survey from
    # seismograms and velocity passed through the codec (lossless, then
    # fixed accuracy 1e-4) and compare with the migration of the originals
    # (relative L2 of the images, in %; the paper reports 2.0e-6 % and
    # 4.3e-5 % NRMS on Marmousi2)
    vm_t = torch.from_numpy(vm.astype(np.float32)).to(dev)[None].contiguous()
    opts = rtm.Opts(4, rtm.SNAP_F32, 1e-6, 1)
    ref = torch.empty((s.nz, s.nx), dtype=torch.float32, device=dev)
    ctx.migrate(grid, vm_t[0], acq, seis, opts, ref)
    through = {}
    for tol in (0.0, 1e-4):
        rt = []
        for arr in (seis, vm_t):
            count, n0, n1 = arr.shape
            stride = (rtm.compress_bound(n0, n1) + 15) // 16 * 16
            out = torch.empty(count * stride, dtype=torch.uint8, device=dev)
            back = torch.empty_like(arr)
            ctx.compress(arr, tol, out, stride)
            ctx.decompress(out, stride, count, n0, n1, back)
            rt.append(back)
            del out
        img = torch.empty_like(ref)
        ctx.migrate(grid, rt[1][0], acq, rt[0], opts, img)
        torch.cuda.synchronize()
        through["lossless" if tol == 0 else f"tol_{tol:g}"] = {
            "image_rel_l2_pct": 100.0 * float(torch.linalg.norm((img - ref).double()) /
                                              torch.linalg.norm(ref.double())),
            "seismogram_rel_l2_pct": 100.0 * float(torch.linalg.norm((rt[0] - seis).double()) /
                                                   torch.linalg.norm(seis.double()))}
        del rt
    head = cases[0]
    line = {
        "workload": f"codec_seis{s.nshot}x{s.nt}x{s.nrec}_img64_vel64",
        "metric": "codec GB/s of float data (compress) at the paper's tolerances",
        "value": head["compress_gbs"], "unit": "GB/s", "steps": args.steps,
        "warmup": args.warmup, "peak": peak, "peak_kind": f"{peak_kind} hbm_gbs",
        "l2": "inputs larger than L2 (3.3 GB of seismograms; 153 MB of images, velocities)",
        "cases": cases, "clocks": ck, "migration_through_codec": through,
        "data": "synthetic",
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def run_eikonal(args, local):
    """First-arrival traveltime panels of the tomography stage (§2.1 Eq. 1,
    §3): the 17 km x 3.5 km layered/faulted model generated on a 40 m grid
    (426 x 88), a velocity ensemble of --samples (default 64) samples, 34
    surface sources every 480 m (the paper's 34 traveltime panels),
    receivers at every surface node.  One step = one rtm_eikonal call over
    the whole ensemble, timed with CUDA events; both field storages."""
    import torch

    import oracle
    from paper_2001_06444_gb300 import inputs, rtm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nz, nx, h = 88, 426, 40.0
    base = inputs.layered_faulted(nz, nx, h, h, seed=20010644)
    ens = inputs.ensemble(base, h, h, args.samples).astype(np.float32)
    src_ix = (6 + 12 * np.arange(34)).astype(np.int32)
    src_iz = np.zeros(34, np.int32)
    rec_ix = np.arange(nx, dtype=np.int32)
    rec_iz = np.zeros(nx, np.int32)
    ctx = rtm.Context(local)
    vel = torch.from_numpy(ens).to(dev)
    times = torch.empty((args.samples, 34, nx), dtype=torch.float32, device=dev)
    solves = args.samples * 34
    res = {}
    clocks = Clocks(local)
    clocks.start()
    for storage in ("shared", "offchip", "auto"):
        for _ in range(args.warmup):
            iters = ctx.eikonal(vel, h, h, src_iz, src_ix, rec_iz, rec_ix, times=times,
                                storage=storage)
        torch.cuda.synchronize()
        ctx.set_profiling(True)
        ctx.stats(reset=True)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            iters = ctx.eikonal(vel, h, h, src_iz, src_ix, rec_iz, rec_ix, times=times,
                                storage=storage)
        e1.record(st)
        torch.cuda.synchronize()
        stt = ctx.stats(reset=True)
        ctx.set_profiling(False)
        ms = e0.elapsed_time(e1) / args.steps
        kms = stt["eik_ms"] / args.steps
        res[storage] = {
            "solves_per_s": solves / (ms / 1e3), "kernel_solves_per_s": solves / (kms / 1e3),
            "ms_per_step": ms, "kernel_ms_per_step": kms,
            "node_updates_per_s": stt["eik_updates"] / (stt["eik_ms"] / 1e3),
            "iterations_mean": float(np.mean(iters)), "iterations_max": int(np.max(iters))}
    # one sampler step of the tomography: one model, its 34 sources (latency)
    lat = {}
    for storage in ("shared", "offchip", "auto"):
        one, t1 = vel[:1].contiguous(), times[:1].contiguous()
        for _ in range(args.warmup):
            ctx.eikonal(one, h, h, src_iz, src_ix, rec_iz, rec_ix, times=t1, storage=storage)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(args.steps):
            ctx.eikonal(one, h, h, src_iz, src_ix, rec_iz, rec_ix, times=t1, storage=storage)
        lat[storage] = 1e3 * (time.perf_counter() - t) / args.steps
    ck = clocks.stop()
    best = "auto"
    # end to end with host buffers: velocities in, panels out
    h_vel = torch.from_numpy(ens).pin_memory()
    h_times = torch.empty((args.samples, 34, nx), dtype=torch.float32).pin_memory()
    t = time.perf_counter()
    for _ in range(args.steps):
        ctx.eikonal(h_vel, h, h, src_iz, src_ix, rec_iz, rec_ix, times=h_times)
    e2e = solves * args.steps / (time.perf_counter() - t)
    # the oracle (fast marching, FP64) on one sample's 34 sources
    t = time.perf_counter()
    for k in range(34):
        oracle.eikonal(ens[0].astype(np.float64), h, h, 0, src_ix[k])
    cpu_dt = time.perf_counter() - t
    line = {
        "workload": f"eikonal_426x88_40m_{args.samples}samples_34src",
        "metric": "traveltime solves/s (one source x one velocity sample)",
        "value": res[best]["solves_per_s"], "unit": "solves/s", "steps": args.steps,
        "warmup": args.warmup, "storage": best, "variants": res,
        "sampler_step_ms": lat,
        "e2e": {"value": e2e, "unit": "solves/s",
                "h2d_bytes_per_step": int(h_vel.numel() * 4),
                "d2h_bytes_per_step": int(h_times.numel() * 4)},
        "cpu_baseline": {"value": 34 / cpu_dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": f"34 fast-marching solves (FP64) of one sample, {cpu_dt:.2f} s"},
        "clocks": ck, "data": "synthetic",
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def run_stats(args, local):
    """Per-pixel ensemble statistics (mean, std, 5/95 % quantiles) of
    --samples seeded normal images of the 351 x 1701 grid, device buffers;
    CUDA events around --steps calls after --warmup calls."""
    import torch

    from paper_2001_06444_gb300 import rtm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, npix = args.samples, 351 * 1701
    g = torch.Generator(device=dev).manual_seed(2001064)
    x = torch.randn((n, npix), generator=g, device=dev, dtype=torch.float32)
    outs = [torch.empty(npix, dtype=t, device=dev)
            for t in (torch.float64, torch.float64, torch.float32, torch.float32)]
    ctx = rtm.Context(local)
    for _ in range(args.warmup):
        ctx.ensemble_stats(x, *outs)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        ctx.ensemble_stats(x, *outs)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    nbytes = n * npix * 4 + npix * 24
    peak, kind = measured_peaks()
    print(json.dumps({"workload": f"ensemble_stats_{n}x{npix}", "ms_per_call": ms,
                      "algorithmic_gbs": nbytes / ms / 1e6, "frac_of_hbm": nbytes / ms / 1e6 / peak,
                      "peak_kind": kind, "data": "synthetic"}), flush=True)
    ctx.close()


def run_born(args, local):
    """Born modelling of the full-size survey (the forward operator of
    least-squares migration): --shots shots of the 1701 x 351 model,
    reflectivity = the relative contrast of the true model against the 60 m
    smoothed one, FP32 snapshots every 4 steps; CUDA events around --steps
    calls after --warmup calls."""
    import torch

    from paper_2001_06444_gb300 import inputs, rtm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s = inputs.full_size(nshot=args.shots, nt=args.nt)
    vm = inputs.smooth(s.vel, s.dx, s.dz, 60.0)
    refl = ((s.vel - vm) / s.vel).astype(np.float32)
    grid = rtm.make_grid(*s.grid_tuple())
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    opts = rtm.Opts(4, rtm.SNAP_F32, 1e-6, 0, 0)
    ctx = rtm.Context(local)
    vel = torch.from_numpy(vm.astype(np.float32)).to(dev)
    m = torch.from_numpy(refl).to(dev)
    seis = torch.empty((s.nshot, s.nt, s.nrec), dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        ctx.born(grid, vel, acq, m, opts, seis)
    torch.cuda.synchronize()
    ctx.set_profiling(True)
    ctx.stats(reset=True)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        ctx.born(grid, vel, acq, m, opts, seis)
    e1.record(st)
    torch.cuda.synchronize()
    stt = ctx.stats(reset=True)
    ms = e0.elapsed_time(e1) / args.steps
    peak, _ = measured_peaks()
    print(json.dumps({
        "workload": f"born_1701x351_{s.nshot}shots_nt{s.nt}_isnap4_f32snap",
        "shots_per_s": s.nshot / (ms / 1e3), "ms_per_step": ms,
        "gpt_updates_per_s": stt["point_updates"] / args.steps / (ms / 1e3) / 1e9,
        "step_kernel_gbs": stt["step_bytes"] / (stt["step_ms"] / 1e3) / 1e9,
        "frac_of_measured_hbm": stt["step_bytes"] / (stt["step_ms"] / 1e3) / 1e9 / peak,
        "data": "synthetic"}), flush=True)
    ctx.close()


def run_lsrtm(args, local):
    """Least-squares migration of the full-size survey: --iters CGLS
    iterations (one Born modelling and one adjoint migration each, plus the
    first adjoint) over --shots shots, data = Born data of the relative
    contrast between the true and the 60 m smoothed model (modelled untimed),
    FP32 snapshots every 4 steps; CUDA events around --steps solves after
    --warmup."""
    import torch

    from paper_2001_06444_gb300 import inputs, rtm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s = inputs.full_size(nshot=args.shots, nt=args.nt)
    vm = inputs.smooth(s.vel, s.dx, s.dz, 60.0)
    refl = ((s.vel - vm) / s.vel).astype(np.float32)
    grid = rtm.make_grid(*s.grid_tuple())
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    opts = rtm.Opts(4, rtm.SNAP_F32, 1e-6, 0, 0)
    ctx = rtm.Context(local)
    vel = torch.from_numpy(vm.astype(np.float32)).to(dev)
    seis = torch.empty((s.nshot, s.nt, s.nrec), dtype=torch.float32, device=dev)
    ctx.born(grid, vel, acq, torch.from_numpy(refl).to(dev), opts, seis)  # the data, untimed
    out = torch.empty((s.nz, s.nx), dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        ctx.lsrtm(grid, vel, acq, seis, opts, args.iters, out)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        mis = ctx.lsrtm(grid, vel, acq, seis, opts, args.iters, out)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({
        "workload": f"lsrtm_1701x351_{s.nshot}shots_nt{s.nt}_{args.iters}iters_f32snap",
        "s_per_solve": ms / 1e3, "s_per_iteration": ms / 1e3 / (args.iters + 0.5),
        "operator_shots_per_s": s.nshot * (2 * args.iters + 1) / (ms / 1e3),
        "misfit_ratio": mis[-1] / mis[0], "misfits": mis, "data": "synthetic"}), flush=True)
    ctx.close()


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "serve":
        run_serve(args, local)
    elif args.workload == "ensemble":
        run_ensemble(args, world, rank, local)
    elif args.workload == "codec":
        run_codec(args, local)
    elif args.workload == "eikonal":
        run_eikonal(args, local)
    elif args.workload == "stats":
        run_stats(args, local)
    elif args.workload == "born":
        run_born(args, local)
    elif args.workload == "lsrtm":
        run_lsrtm(args, local)
    else:
        run_native(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
