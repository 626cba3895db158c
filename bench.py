#!/usr/bin/env python
"""Throughput of the landscape-evolution time step on GB300, in cell-steps/s.

A step is one full time step of the method (receivers, donors, levels,
accumulation, uplift + erosion) over the whole synthetic grid.  Default
workload: the paper's 10000 x 10000 size, FP32 elevations with FP64 slope
tests and int64 cell counts, seeded [0,10) noise, dx = 100 m, K = 2e-5 /yr,
m = 0.45, U = 1e-3 m/yr, dt = 500 yr; the timed window ends at the
configuration's 100th step (earlier steps run untimed first).

Its working set (~0.6 GB of elevations, codes and masks) is larger than the
129 MB L2; the L2 is also flushed (a 512 MiB write) between timed steps,
outside the CUDA events that bracket each step on the launching stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the CPU oracle on the host cores
  python bench.py --sweep                # edge 100 .. 16000, O(N^x) per region

Under torchrun each rank advances its own replica of the grid (one grid does
not shard: its level order is global); the reported value is the sum over
ranks divided by the slowest rank's time.  The batch of realizations (a form
measured beside the main line) shards by LPT over the ranks.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "cell-steps/s"
# algorithmic bytes per cell-step by phase (elevation bytes P, count bytes Ab):
#   receivers+donors P+2 (read h, write receiver code and donor mask),
#   levels 10 (mask, frontier read, queue write, sink scan),
#   accumulate 5+2Ab (queue, mask, donor counts, count write),
#   erode 5+Ab+3P (queue, receiver code, count, h_c, h_r, h write)
PHASES = ("receivers", "levels", "accumulate", "erode")


def algo_bytes(P, Ab):
    return {"receivers": P + 2, "levels": 10, "accumulate": 5 + 2 * Ab, "erode": 5 + Ab + 3 * P}


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default="grid10000_f32")
    ap.add_argument("--edge", type=int, default=0,
                    help="run the workload's recipe on an edge x edge grid instead\n"
                         "(smaller cases of the same kernel for profiling)")
    ap.add_argument("--flush-mib", type=int, default=512)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-phases", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the FP32, 10000^2, batch and adjoint measurements")
    ap.add_argument("--batch-steps", type=int, default=200,
                    help="steps of every realization of the 512-grid batch")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--sweep", action="store_true",
                    help="time the FP64 step at edge lengths 100 .. 16000 and fit the\n"
                         "wall-time exponent x of O(N^x) per edge-length region")
    ap.add_argument("--sweep-steps", type=int, default=10)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_params(w):
    import oracle
    return oracle.params(dx=w.dx, K=w.K, m=w.m, U=w.U, dt=w.dt)


def cpu_oracle_rate(w, target_s, h0=None):
    """Time the oracle (single thread, as written) on the workload's own
    initial surface; scale the step count so the sample takes ~target_s."""
    import oracle
    p = oracle_params(w)
    h0 = w.initial() if h0 is None else h0
    side = w.nx
    # one probe step on the full grid decides the sample size
    t0 = time.perf_counter()
    oracle.run(h0, p, 1)
    t1 = time.perf_counter() - t0
    if t1 * 2 > target_s:
        # full-grid steps are too slow: run a smaller square of the same recipe
        from paper_1803_02977_gb300 import synth
        frac = max(1e-3, target_s / (4 * t1))
        side = max(64, int(w.nx * frac ** 0.5))
        h0 = synth.noise_surface(side, side, w.seed, 0.0, w.noise_hi, w.south_tilt, w.dx)
        t0 = time.perf_counter()
        oracle.run(h0, p, 1)
        t1 = time.perf_counter() - t0
    nsteps = max(1, int(target_s / max(t1, 1e-6)))
    t0 = time.perf_counter()
    oracle.run(h0, p, nsteps)
    el = time.perf_counter() - t0
    cells = h0.size
    return {"value": cells * nsteps / el, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"{nsteps} oracle steps on a {h0.shape[1]}x{h0.shape[0]} grid of the "
                      f"same recipe, {el:.1f} s, single-threaded C (-O2, FP64); the metric "
                      f"is per cell-step, so the configuration's step count does not change it",
            "host": host_info()}


def host_info():
    """The host's logical CPU count and CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1803_02977_gb300 import synth
    import oracle
    w = workload_of(synth, args)
    p = oracle_params(w)
    h = w.initial()
    # size each step so that warmup + steps end within a few minutes
    t0 = time.perf_counter()
    oracle.run(h, p, 1)
    t1 = time.perf_counter() - t0
    budget = 150.0
    if t1 * (args.steps + args.warmup) > budget:
        frac = budget / (t1 * (args.steps + args.warmup))
        side = max(32, int(w.nx * frac ** 0.5))
        h = synth.noise_surface(side, side, w.seed, 0.0, w.noise_hi, w.south_tilt, w.dx)
        sample = f"each step: one oracle step on a {side}x{side} grid of the same recipe"
    else:
        sample = f"each step: one oracle step on the full {w.nx}x{w.ny} grid"
    h = oracle.run(h, p, args.warmup)
    t0 = time.perf_counter()
    oracle.run(h, p, args.steps)
    el = time.perf_counter() - t0
    cells = h.size
    value = cells * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(w, args),
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
                             "sample": sample, "host": host_info()},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_of(synth, args):
    """The named workload, on an edge x edge grid if --edge is given."""
    import dataclasses
    w = synth.workload(args.workload)
    if args.edge:
        w = dataclasses.replace(w, name=f"{w.name}_edge{args.edge}", nx=args.edge, ny=args.edge)
    return w


def config_of(w, args):
    return {"workload": w.name, "nx": w.nx, "ny": w.ny, "dtype": w.dtype,
            "count_bits": 64 if w.area_dtype == "i64" else 32, "dx": w.dx, "K": w.K, "m": w.m,
            "U": w.U, "dt": w.dt, "seed": w.seed, "noise": [0.0, w.noise_hi],
            "south_tilt": w.south_tilt, "area_scale": "dx*dx",
            "l2": f"flushed between timed steps ({args.flush_mib} MiB write)",
            "parallelism": f"replicas{args.gpus}"}


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1803_02977_gb300 import lem, synth

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload_of(synth, args)
    P = 8 if w.dtype == "f64" else 4
    Ab = 8 if w.area_dtype == "i64" else 4
    h0_np = w.initial().astype(np.float64 if P == 8 else np.float32)
    N = w.nx * w.ny
    par = dict(dx=w.dx, K=w.K, m=w.m, U=w.U, dt=w.dt, count_bits=8 * Ab)

    h = torch.tensor(h0_np, device=dev)
    mdl = lem.Model(h, **par)
    flush = torch.empty(args.flush_mib << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    # the step's work decomposition, picked by the autotuner on the initial
    # surface (outside the timed region; the surface is left as it was)
    from paper_1803_02977_gb300 import autotune
    tiling, tiling_ms = autotune.tune_step(mdl, steps=3, use_cache=False)

    def barrier():
        if ws > 1:
            dist.barrier()

    # the timed window ends at the configuration's last step: the steps
    # before the warm-up run untimed, in one launch
    K = args.steps
    ahead = max(0, w.steps - K - args.warmup)
    if ahead:
        mdl.step(ahead)
    for _ in range(args.warmup):
        mdl.step(1)
        flush.zero_()
    mdl.sync()
    tiers0 = lem.lem_tier_stats(mdl.ctx)

    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    t_wall = time.perf_counter()
    for i in range(K):
        ev0[i].record(stream)
        mdl.step(1)
        ev1[i].record(stream)
        flush.zero_()
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    barrier()
    clk = clocks.stop()
    mdl.sync()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    tot_ms = float(sum(step_ms))
    t = torch.tensor([tot_ms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tot_ms = float(t.item())
    value = N * K * ws / (tot_ms / 1e3)
    ms_per_step = tot_ms / K

    # which tier handled the cells of the timed steps (warp tiles, block
    # queues, device-wide levels)
    tiers = [b_ - a_ for a_, b_ in zip(tiers0, lem.lem_tier_stats(mdl.ctx))]
    tier_frac = [x / max(1, sum(tiers)) for x in tiers]

    # level count of the state the timed window ended on (outside the timed
    # region; the stage calls recompute the graph of the current surface)
    mdl.receivers()
    L = lem.lem_levels(mdl.ctx)

    # one traced launch after the timed region: in-kernel time per phase of
    # the production step, and the achieved bandwidth of each phase
    ab = algo_bytes(P, Ab)
    peak = measured_peaks().get("hbm_gbs")
    tc0 = lem.lem_tier_stats(mdl.ctx)
    timeline = traced_step(lem, mdl, flush)
    tcells = [b_ - a_ for a_, b_ in zip(tc0, lem.lem_tier_stats(mdl.ctx))]
    phases = step_phase_split(timeline, tcells, ab, N, peak)

    # per-stage split through the stage-by-stage calls (device-wide levels),
    # on the initial surface (outside the timed region)
    stage_calls = None
    if not args.no_phases:
        hp = torch.tensor(h0_np, device=dev)
        mp = lem.Model(hp, **par)
        reps = 5
        acc = {k: 0.0 for k in PHASES}
        for r in range(reps + 1):
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(PHASES) + 1)]
            flush.zero_()
            evs[0].record(stream)
            mp.receivers()
            evs[1].record(stream)
            lem.lem_levels(mp.ctx)
            evs[2].record(stream)
            lem.lem_accumulate(mp.ctx)
            evs[3].record(stream)
            mp.erode()
            evs[4].record(stream)
            torch.cuda.synchronize()
            if r > 0:
                for i, k in enumerate(PHASES):
                    acc[k] += evs[i].elapsed_time(evs[i + 1]) / reps
            hp.copy_(torch.tensor(h0_np, device=dev))
        stage_calls = {k: {"ms": acc[k], "algo_bytes_per_cell": ab[k],
                           "gbs": ab[k] * N / (acc[k] / 1e3) / 1e9,
                           "cell_steps_per_s": N / (acc[k] / 1e3)} for k in PHASES}
        if peak:
            for k in PHASES:
                stage_calls[k]["frac_of_measured_hbm"] = stage_calls[k]["gbs"] / peak
        mp.close()
        del hp

    e2e = measure_e2e(lem, h0_np, par, dev, max(3, min(K, 20)), ws)
    mdl.close()
    del h
    torch.cuda.empty_cache()

    forms = None
    if not args.no_forms and not args.edge:
        forms = measure_forms(lem, synth, args, w, ms_per_step, flush, dev, ws, rank)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(w, args.cpu_seconds)

    per_cell = sum(ab.values())
    achieved = per_cell * N / (ms_per_step / 1e3) / 1e9
    traffic, traffic_src = profiled_traffic(w.name)
    kname = {("f64", 4): "<double, int, false>", ("f64", 8): "<double, long long, false>",
             ("f32", 4): "<float, int, false>", ("f32", 8): "<float, long long, false>"}
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if peak else None, "traffic": traffic,
                "traffic_source": traffic_src,
                "kernel": "lem::lem_step_kernel" + kname[(w.dtype, Ab)]
                          + " (one cooperative launch per step)",
                "algo_bytes_per_cell_step": per_cell,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy), of measured"
                               if peak else None}
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": w.dtype, "data": "synthetic",
            "config": config_of(w, args),
            "window": {"first_timed_step": ahead + args.warmup + 1,
                       "last_timed_step": ahead + args.warmup + K, "config_steps": w.steps},
            "levels_after": int(L),
            "step_ms_min_median_max": [min(step_ms), float(np.median(step_ms)), max(step_ms)],
            "wall_s_timed_region": t_wall,
            "roofline": roofline, "phases": phases, "stage_calls": stage_calls,
            "timeline": timeline,
            "tier_cell_fraction": {"warp_tiles": tier_frac[0], "block_queues": tier_frac[1],
                                   "device_wide": tier_frac[2]},
            "tiling": {"strip_rows": tiling[0], "half_tiles": tiling[1],
                       "autotune_ms_per_step": {k: round(v, 4) for k, v in tiling_ms.items()}},
            "clocks": clk, "e2e": e2e,
            "gpu_launches": K, "cpu_baseline": cpu, "forms": forms}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def step_phase_split(timeline, tier_cells, ab, N, peak):
    """Achieved bandwidth of each phase of the production step from the
    device trace (block 0's view of the traced launch's steady-state step):
    the codes pass (Algs 1-2, P+2 bytes per cell) up to the grid barrier
    after it, the warp and block tiers (Algs 3-6, the levels + accumulation +
    erosion bytes of each cell they handled) up to the next barrier, and the
    device-wide tier (the same bytes per cell it handled)."""
    if not timeline:
        return None
    us = (timeline.get("steady_state_step") or timeline)["us"]
    tot = max(1, sum(tier_cells))
    nsteps = timeline.get("steps_in_launch", 1)
    per = {k: v / nsteps for k, v in zip(("warp", "block", "device"), tier_cells)}
    sweep = ab["levels"] + ab["accumulate"] + ab["erode"]
    out = {}
    parts = {"codes": (us["codes"] + us["codes_wait"], ab["receivers"] * N),
             "tiles": (us["tiles_warp"] + us["tiles_block"] + us["tiles_wait"],
                       sweep * (per["warp"] + per["block"])),
             "device": (us["device_tier"], sweep * per["device"])}
    for k, (t_us, nbytes) in parts.items():
        if t_us <= 0 or nbytes <= 0:
            out[k] = {"us": t_us, "algo_bytes": nbytes, "gbs": None, "frac_of_measured_hbm": None}
            continue
        gbs = nbytes / (t_us / 1e6) / 1e9
        out[k] = {"us": t_us, "algo_bytes": nbytes, "gbs": gbs,
                  "frac_of_measured_hbm": gbs / peak if peak else None}
    out["codes"]["algo_bytes_per_cell"] = ab["receivers"]
    out["tiles"]["algo_bytes_per_cell"] = sweep
    out["tier_cells_per_step"] = {k: v for k, v in per.items()}
    out["cells"] = N
    out["source"] = "in-kernel %globaltimer trace, block 0, steady-state step of a 3-step launch"
    del tot
    return out


def measure_e2e(lem, h0_np, par, dev, steps, ws, nbuf=3):
    """End to end through the public API with host buffers: every step the
    elevations are copied from pinned host memory to the device, advanced one
    step by lem_step, and copied back to pinned host memory.  Copies and the
    step run on three streams over nbuf device buffers, so the upload of
    step i+1 and the download of step i-1 overlap step i (the context is
    bound to step i's buffer before its launch); the timed region spans the
    first upload to the last download."""
    import torch
    import torch.distributed as dist
    hin = torch.from_numpy(np.ascontiguousarray(h0_np)).pin_memory()
    hout = [torch.empty_like(hin).pin_memory() for _ in range(nbuf)]
    d = [torch.empty(hin.shape, dtype=hin.dtype, device=dev) for _ in range(nbuf)]
    me = lem.Model(d[0], **par)
    comp = torch.cuda.current_stream()
    s_up, s_down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    up_done = [torch.cuda.Event() for _ in range(nbuf)]
    comp_done = [torch.cuda.Event() for _ in range(nbuf)]
    down_done = [torch.cuda.Event() for _ in range(nbuf)]

    def one(i):
        b = i % nbuf
        if i >= nbuf:
            s_up.wait_event(down_done[b])  # buffer b's previous result has left
        with torch.cuda.stream(s_up):
            d[b].copy_(hin, non_blocking=True)
            up_done[b].record(s_up)
        comp.wait_event(up_done[b])
        lem.lem_bind_elevation(me.ctx, d[b], me.dtype)
        me.step(1)
        comp_done[b].record(comp)
        s_down.wait_event(comp_done[b])
        with torch.cuda.stream(s_down):
            hout[b].copy_(d[b], non_blocking=True)
            down_done[b].record(s_down)

    for i in range(nbuf + 1):
        one(i)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(comp)
    s_up.wait_event(e0)
    for i in range(steps):
        one(i)
    for b in range(nbuf):
        comp.wait_event(down_done[b])
    e1.record(comp)
    torch.cuda.synchronize()
    me.sync()
    ms = e0.elapsed_time(e1)
    # the result of the last step, checked to have left the device intact
    last = (steps - 1) % nbuf
    ok = bool(torch.equal(hout[last], d[last].cpu()))
    me.close()
    te = torch.tensor([ms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    n = hin.numel()
    nb = n * hin.element_size()
    return {"value": n * steps * ws / (float(te.item()) / 1e3), "unit": METRIC,
            "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb, "steps": steps,
            "ms_per_step": float(te.item()) / steps, "result_copied_back": ok,
            "how": f"pinned host -> device, lem_step, device -> pinned host every step; three "
                   f"streams, {nbuf} device buffers (upload i+1 and download i-1 overlap step i)"}


def measure_forms(lem, synth, args, w, ms_per_step, flush, dev, ws, rank):
    """The other configurations and forms, each at its stated horizon."""
    import torch
    import torch.distributed as dist
    forms = {}
    N = w.nx * w.ny
    plain_here = N / (ms_per_step / 1e3)
    # the same grid in FP64 (the plain path the FP32 form must beat)
    if w.name == "grid10000_f32":
        w64 = synth.workload("grid10000_f64")
        r = time_grid(lem, w64, 10, 3, flush, dev, horizon=w64.steps)
        forms["grid10000_f64_same_grid"] = dict(r, workload=w64.name,
                                                vs_fp32=r["value"] / plain_here)
    # the 2048^2 workload, FP64 and FP32, timed on steps 481-500 of its 500
    w2 = synth.workload("grid2048_f64")
    r64 = time_grid(lem, w2, 20, 3, flush, dev, horizon=w2.steps)
    forms["grid2048_f64"] = dict(r64, workload=w2.name)
    w2f = synth.workload("grid2048_f32")
    r32 = time_grid(lem, w2f, 20, 3, flush, dev, horizon=w2f.steps)
    forms["grid2048_f32"] = dict(r32, workload=w2f.name, vs_plain_fp64=r32["value"] / r64["value"])
    plain = r64["value"]
    forms["fill"] = measure_fill(lem, w2, flush, dev, plain)
    forms["mfd_accumulation"] = measure_mfd(lem, w2, flush, dev)
    # Alg 6 with n-hat = 2 and 1.5 (Newton-Raphson in every tier)
    for nh in (2.0, 1.5):
        rn = time_grid(lem, w2, 20, 3, flush, dev, slope_exponent=nh)
        forms[f"slope_exponent_n{nh:g}"] = dict(rn, workload=w2.name, n_hat=nh, eps_m=1e-12,
                                                 max_iter=100, vs_plain_fp64=rn["value"] / plain)
    del flush
    torch.cuda.empty_cache()
    bt = measure_batch(lem, args.batch_steps, ws, rank, dev)
    t = torch.tensor([bt["ms"], bt["plain_fp64"]["ms"]], dtype=torch.float64, device=dev)
    cs = torch.tensor([bt["cell_steps"], bt["plain_fp64"]["cells"] * bt["steps"]],
                      dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(cs)
    bt["value"] = float(cs[0]) / (float(t[0]) / 1e3)
    bt["plain_fp64"]["value"] = float(cs[1]) / (float(t[1]) / 1e3)
    bt["vs_plain_fp64"] = bt["value"] / bt["plain_fp64"]["value"]
    peak = measured_peaks().get("hbm_gbs")
    per_cell = sum(algo_bytes(4, 4).values())
    bt["algo_bytes_per_cell_step"] = per_cell
    bt["achieved_gbs"] = per_cell * bt["value"] / 1e9
    bt["frac_of_measured_hbm"] = bt["achieved_gbs"] / peak if peak else None
    bt["ranks"] = ws
    forms["batch512_f32"] = bt
    if rank == 0:
        forms["adjoint_grid1024_f64"] = measure_adjoint(lem, dev)
    return forms


def time_grid(lem, w, steps, warmup, flush, dev, slope_exponent=None, mode=None, horizon=None):
    """`steps` single-step lem_step calls on workload w, each bracketed by
    CUDA events, L2 flushed between them; with `horizon`, the timed window
    ends at that step (the steps before it run untimed).  slope_exponent:
    Alg 6's Newton form with that n-hat (eps 1e-12 m, at most 100 updates);
    mode: the lem_set_step_mode form.  Returns the mean time per step, the
    rate, the window, the level count of the state reached and the tiers."""
    import torch
    P = 8 if w.dtype == "f64" else 4
    count_bits = 64 if w.area_dtype == "i64" else 32
    h = torch.tensor(w.initial().astype(np.float64 if P == 8 else np.float32), device=dev)
    mdl = lem.Model(h, dx=w.dx, K=w.K, m=w.m, U=w.U, dt=w.dt, count_bits=count_bits)
    if slope_exponent is not None:
        mdl.set_slope_exponent(slope_exponent, 1e-12, 100)
    if mode is not None:
        lem.lem_set_step_mode(mdl.ctx, mode)
    stream = torch.cuda.current_stream()
    ahead = max(0, (horizon or 0) - steps - warmup)
    if ahead:
        mdl.step(ahead)
    for _ in range(warmup):
        mdl.step(1)
        flush.zero_()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    mdl.sync()
    t0 = lem.lem_tier_stats(mdl.ctx)
    torch.cuda.synchronize()
    for e0, e1 in ev:
        e0.record(stream)
        mdl.step(1)
        e1.record(stream)
        flush.zero_()
    torch.cuda.synchronize()
    mdl.sync()
    ms = [a.elapsed_time(b) for a, b in ev]
    tiers = [b_ - a_ for a_, b_ in zip(t0, lem.lem_tier_stats(mdl.ctx))]
    mdl.receivers()
    L = lem.lem_levels(mdl.ctx)
    mdl.close()
    mean = float(np.mean(ms))
    return {"ms_per_step": mean, "value": w.cells / (mean / 1e3), "steps_timed": steps,
            "window": [ahead + warmup + 1, ahead + warmup + steps], "levels_after": int(L),
            "tier_cell_fraction": [x / max(1, sum(tiers)) for x in tiers]}


def measure_fill(lem, w, flush, dev, plain, reps=5):
    """Depression filling (lem_fill) of workload w's initial surface: device
    time per flood (a fresh copy of the surface each time, L2 flushed) and
    the work it took; then, on the evolving surface, a flood followed by a
    time step, the two timed separately."""
    import torch
    h0 = torch.tensor(w.initial(), device=dev)
    h = h0.clone()
    mdl = lem.Model(h, dx=w.dx, K=w.K, m=w.m, U=w.U, dt=w.dt)
    stream = torch.cuda.current_stream()
    ms = []
    for r in range(reps + 2):
        h.copy_(h0)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mdl.fill()
        e1.record(stream)
        torch.cuda.synchronize()
        if r >= 2:
            ms.append(e0.elapsed_time(e1))
    mdl.sync()
    rounds, visits, passes, unsettled = lem.lem_fill_stats(mdl.ctx)
    changed = int((h != h0).sum().item())
    mdl.close()
    # the evolving surface: a flood, then a step, three times untimed, then
    # both timed separately (with L, the level count of the filled surface)
    h.copy_(h0)
    mdl = lem.Model(h, dx=w.dx, K=w.K, m=w.m, U=w.U, dt=w.dt)
    fms, sms = [], []
    for r in range(3 + 4):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        flush.zero_()
        evs[0].record(stream)
        mdl.fill()
        evs[1].record(stream)
        mdl.step(1)
        evs[2].record(stream)
        torch.cuda.synchronize()
        if r >= 3:
            fms.append(evs[0].elapsed_time(evs[1]))
            sms.append(evs[1].elapsed_time(evs[2]))
    mdl.sync()
    tiers = lem.lem_tier_stats(mdl.ctx)
    ev_rounds = lem.lem_fill_stats(mdl.ctx)[0]
    mdl.fill()
    mdl.receivers()
    L = lem.lem_levels(mdl.ctx)
    mdl.close()
    N = w.cells
    f_ms = float(np.median(ms))
    # algorithmic bytes of a flood: read h, write the filled h
    gbs = 2 * (8 if w.dtype == "f64" else 4) * N / (f_ms / 1e3) / 1e9
    step_ms = float(np.mean(fms)) + float(np.mean(sms))
    return {"workload": w.name, "ms_per_fill": f_ms, "rounds": rounds,
            "tile_visits": visits, "passes": passes, "unsettled_visits": unsettled,
            "cells_changed": changed, "cells_per_s": N / (f_ms / 1e3),
            "algo_gbs_read_h_write_h": gbs,
            "evolving_surface": {
                "ms_per_fill": float(np.mean(fms)), "fill_rounds": ev_rounds,
                "ms_per_step_after_fill": float(np.mean(sms)),
                "levels_of_filled_surface": L,
                "tier_cells": {"warp_tiles": tiers[0], "block_queues": tiers[1],
                               "device_wide": tiers[2]},
                "ms_per_fill_and_step": step_ms, "value": N / (step_ms / 1e3),
                "vs_plain_fp64": N / (step_ms / 1e3) / plain}}


def measure_mfd(lem, w, flush, dev, reps=5, p=1.1):
    """Flow accumulation with multiple flow directions (lem_accumulate_mfd)
    on workload w's initial surface, with Freeman's exponent p and with
    p = 1 (no powers): device time per call with L2 flushed before it, and
    the number of levels."""
    import torch
    h = torch.tensor(w.initial(), device=dev)
    mdl = lem.Model(h, dx=w.dx, K=w.K, m=w.m, U=w.U, dt=w.dt)
    A = torch.empty_like(h)
    stream = torch.cuda.current_stream()
    out = {"workload": w.name}
    for key, pe in (("p", p), ("p1", 1.0)):
        ms, L = [], 0
        for r in range(reps + 2):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            L = lem.lem_accumulate_mfd(mdl.ctx, A, pe)
            e1.record(stream)
            torch.cuda.synchronize()
            if r >= 2:
                ms.append(e0.elapsed_time(e1))
        t = float(np.median(ms))
        out[key] = {"p": pe, "ms": t, "levels": L, "cells_per_s": w.cells / (t / 1e3)}
    mdl.close()
    return out


def measure_batch(lem, steps, ws, rank, dev, count=512):
    """The 512-realization FP32 batch in one launch (autotuned shape), this
    rank's LPT shard, `steps` steps of every realization; against the plain
    FP64 path run one grid at a time on every realization of the shard, for
    the same steps (the same total cell-steps)."""
    import torch
    from paper_1803_02977_gb300 import autotune, sharding, synth
    bw = synth.batch_workload(count=count)
    sizes = [s * s for s in bw.sides]
    mine = sharding.lpt_partition(sizes, ws)[rank]
    out = sharding.run_shard(lem, bw, mine, steps, tune=True)
    cells = sum(sizes[r] for r in mine)
    # plain FP64 path, one grid at a time, every realization of the shard
    stream = torch.cuda.current_stream()
    plain_ms = 0.0
    for r in mine:
        h = torch.tensor(bw.initial(r), device=dev)
        mdl = lem.Model(h, dx=bw.dx, K=bw.K[r], m=bw.m[r], U=bw.U, dt=bw.dt)
        mdl.step(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        mdl.step(steps)
        b.record(stream)
        torch.cuda.synchronize()
        plain_ms += a.elapsed_time(b)
        mdl.close()
    return {"ms": out["ms"], "cells": cells, "cell_steps": cells * steps,
            "realizations": len(mine), "steps": steps, "shape": list(out["shape"]),
            "autotune_ms_per_step": {k: round(v, 3) for k, v in out["tune_ms"].items()},
            "plain_fp64": {"realizations": len(mine), "cells": cells, "ms": plain_ms,
                           "value": cells * steps / (plain_ms / 1e3),
                           "how": "one lem_step launch of all steps per realization, "
                                  "one realization after another"}}


def measure_adjoint(lem, dev, nsteps=50, ckpt=10):
    """Gradient of sum((h_T - h_obs)^2) wrt the uplift field and K on the
    1024 x 1024 FP64 adjoint workload: forward + checkpointed adjoint."""
    import torch
    from paper_1803_02977_gb300 import autodiff, synth
    w = synth.workload("grid1024_adjoint")
    h0 = torch.tensor(w.initial(), device=dev)
    xi = torch.tensor(synth.signed_field(w.nx, w.ny, 6), device=dev)
    U = torch.full_like(h0, w.U)
    obs = h0.clone()
    m_obs = lem.Model(obs, dx=w.dx, K=1.2 * w.K, m=w.m, U=0.0, dt=w.dt)
    m_obs.set_uplift_field(U * (1.0 + 0.1 * xi))
    m_obs.step(nsteps)
    m_obs.sync()
    m_obs.close()
    def grad():
        Ut = U.clone().requires_grad_(True)
        Kt = torch.tensor(w.K, dtype=torch.float64, device=dev, requires_grad=True)
        hT = autodiff.run(h0, Ut, Kt, nsteps, ckpt_every=ckpt, dx=w.dx, m=w.m, dt=w.dt)
        loss = torch.sum((hT - obs) ** 2)
        loss.backward()
        return loss, Kt

    grad()  # warm-up: first use of autograd and its kernels in this process
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss, Kt = grad()
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    return {"grid": [w.nx, w.ny], "steps": nsteps, "ckpt_every": ckpt, "wall_ms": el * 1e3,
            "loss": loss.item(), "dL_dK": Kt.grad.item(),
            "gradient_cell_steps_per_s": w.nx * w.ny * nsteps / el}


def traced_step(lem, mdl, flush, nsteps=3):
    """Device-side trace of one launch of nsteps tiered steps, as seen by
    block 0: the microseconds between consecutive trace points, grouped by
    what ended them (block 0's own work, or the wait at a device-wide
    barrier).  The first step of a launch includes the launch itself (blocks
    starting on their SMs); later steps show the kernel in steady state."""
    lem.lem_trace_enable(mdl.ctx, 1 << 16)
    flush.zero_()
    mdl.step(nsteps)
    tr = lem.lem_trace_read(mdl.ctx, 1 << 16)
    lem.lem_trace_enable(mdl.ctx, 0)
    starts = [i for i, e in enumerate(tr) if e[1] == "start"] + [len(tr) - 1]
    steps = []
    for k in range(len(starts) - 1):
        seg = tr[starts[k]:starts[k + 1] + 1]
        if len(seg) < 2:
            continue
        out = {"codes": 0.0, "codes_wait": 0.0, "tiles_warp": 0.0, "tiles_block": 0.0,
               "tiles_wait": 0.0, "device_tier": 0.0}
        for (t0, _, _), (t1, ph, lvl) in zip(seg[:-1], seg[1:]):
            us = (t1 - t0) / 1e3
            if ph == "block0_done":
                key = {1: "codes", 4: "tiles_warp"}.get(lvl, "tiles_block")
            elif ph == "receivers":
                key = "codes_wait"
            elif ph == "tiles_end":
                key = "tiles_wait"
            elif ph == "block_end":
                key = "tiles_block"
            else:
                key = "device_tier"
            out[key] += us
        steps.append({"us": out, "total_us": (seg[-1][0] - seg[0][0]) / 1e3})
    if not steps:
        return None
    raw = [[ph, lvl, round((t1 - t0) / 1e3, 2)]
           for (t0, _, _), (t1, ph, lvl) in zip(tr[:-1], tr[1:])][:64]
    return {"us": steps[0]["us"], "total_us": steps[0]["total_us"],
            "steady_state_step": steps[-1] if len(steps) > 1 else None,
            "steps_in_launch": nsteps, "raw": raw}


STEP_KERNEL_SOURCES = ("lem_step_kernel.cuh", "lem_tiles.cuh", "lem_jump.cuh", "lem_device.cuh",
                       "lem_context.cuh", "lem_api.cu")


def kernel_source_hash():
    """sha256 over what the step kernel and its launch are built from (its
    device sources, the translation unit that launches it and the compiler
    flags; name + bytes in order); a committed ncu summary records the hash
    it was taken at, so its DRAM figures are only reported while the kernel
    matches."""
    from paper_1803_02977_gb300 import build as b
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1803_02977_gb300", "csrc")
    for p in [os.path.join(csrc, n) for n in STEP_KERNEL_SOURCES]:
        h.update(os.path.basename(p).encode())
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(b.ARCH + [f for f in b.NVCC_FLAGS if not f.startswith("/")]).encode())
    return h.hexdigest()


def profiled_traffic(workload):
    """DRAM bytes (read + write) per launch of the step kernel from the
    committed ncu summary of this workload, or None when there is none or
    the kernel sources changed since it was captured."""
    want = kernel_source_hash()
    for p in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(p) as f:
            kv = dict(re.findall(r"^(traffic_bytes_per_launch|workload|source_sha256): (\S+)$",
                                 f.read(), re.M))
        if kv.get("workload") == workload and kv.get("source_sha256") == want \
                and "traffic_bytes_per_launch" in kv:
            return int(kv["traffic_bytes_per_launch"]), os.path.relpath(p, ROOT)
    return None, None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}


# Edge-length regions of the paper's GPU scaling table (Table 2): upper edge
# bounds and the wall-time exponents x of O(N^x) it reports in each.
SWEEP_REGIONS = (("A", 400, 0.33), ("B", 1000, 0.16), ("C", 2500, 0.42), ("D", 16000, 0.92))
SWEEP_EDGES = (100, 141, 200, 283, 400, 566, 800, 1000, 1414, 2000, 2500, 2828, 4000, 5657,
               8000, 11314, 16000)


def fit_exponents(edges, ms, regions=SWEEP_REGIONS):
    """Least-squares slope of log(time) against log(cells) in each region;
    a region spans the edges from the previous region's bound to its own,
    both bounds included (a point on a bound belongs to both sides)."""
    edges = np.asarray(edges, dtype=np.float64)
    t = np.asarray(ms, dtype=np.float64)
    out, lo = {}, 0.0
    for name, hi, _ in regions:
        sel = (edges >= lo) & (edges <= hi)
        if sel.sum() >= 2:
            x = np.log(edges[sel] ** 2)
            y = np.log(t[sel])
            out[name] = float(np.polyfit(x, y, 1)[0])
        else:
            out[name] = None
        lo = hi
    return out


def run_sweep(args):
    """The paper's scaling experiment (Table 2) on the tiered FP64 step: per
    edge length, seeded [0,1) noise with the 256^2 workload's parameters,
    warm-up steps, then single-step launches timed with CUDA events, L2
    flushed between them; prints one JSON line."""
    import torch
    from paper_1803_02977_gb300 import lem, synth

    dev = torch.device("cuda", 0)
    w = synth.workload("grid256_f64")
    flush = torch.empty(args.flush_mib << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(0)
    clocks.start()
    points = []
    for e in SWEEP_EDGES:
        h = torch.tensor(synth.noise_surface(e, e, w.seed), device=dev)
        mdl = lem.Model(h, dx=w.dx, K=w.K, m=w.m, U=w.U, dt=w.dt)
        for _ in range(max(3, args.warmup)):
            mdl.step(1)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.sweep_steps)]
        torch.cuda.synchronize()
        for e0, e1 in ev:
            flush.zero_()
            e0.record(stream)
            mdl.step(1)
            e1.record(stream)
        torch.cuda.synchronize()
        mdl.sync()
        tiers = lem.lem_tier_stats(mdl.ctx)
        tl = traced_step(lem, mdl, flush)
        mdl.close()
        del h
        ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
        n = e * e
        ss = (tl or {}).get("steady_state_step") or {}
        points.append({"edge": e, "cells": n, "ms_per_step": ms,
                       "cell_steps_per_s": n / (ms / 1e3),
                       "warp_tier_fraction": tiers[0] / max(1, sum(tiers)),
                       "trace_first_step_us": round((tl or {}).get("total_us", 0.0), 1),
                       "trace_steady_step_us": {k: round(v, 1)
                                                for k, v in (ss.get("us") or {}).items()}})
    clk = clocks.stop()
    fit = fit_exponents([p["edge"] for p in points], [p["ms_per_step"] for p in points])
    print(json.dumps({"sweep": "tiered step, FP64, int32 counts", "metric": "ms/step",
                      "steps_timed": args.sweep_steps, "data": "synthetic",
                      "l2": f"flushed between timed steps ({args.flush_mib} MiB write)",
                      "points": points, "fit_x": fit,
                      "paper_x": {n: x for n, _, x in SWEEP_REGIONS},
                      "region_max_edge": {n: hi for n, hi, _ in SWEEP_REGIONS},
                      "clocks": clk}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return run_sweep(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
