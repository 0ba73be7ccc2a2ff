"""Benchmark of the operator-split tissue SSA on GB300.

One "step" is one Lie splitting step of the whole hot path (chi on every
cell, then S on every x-face and every y-face) over the benchmark tissue:
64x64 cells of 16x16 voxels, the Notch-Delta model, dt = 0.1 (the medium
tissue; synthetic, seeded).  The state is first advanced by an untimed
burn-in so that the timed steps see molecule counts near their working
level, then W warm-up steps and K timed steps run.

Metric: SSA events per second (all events of chi and both face phases), with
cell-steps per second beside it.  `value` times the steps with the state
resident in device memory (CUDA events on the tissue's stream, L2 flushed
between steps); `e2e` times the same steps through the C ABI with the state
copied host->device before and device->host after every step.

Multi-GPU (torchrun, N ranks): every rank advances its own replica tissue
(tissue_id = rank); there is no data exchange (weak scaling).

The serving leg (default: the first 4 requests of the serving workload,
about a minute) reports p50/p99 latency beside the served events/s.

`--impl reference` times the CPU oracle (test infrastructure, plain C with
OpenMP) on a bounded patch of the same workload.
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

import numpy as np  # noqa: E402

from paper_1806_10889_gb300 import workloads as W  # noqa: E402

METRIC = "SSA events/s (chi + face binding), medium tissue 64x64 cells x 16x16 voxels, dt 0.1"
UNIT = "events/s"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Issue-slot peak of the chip: 152 SMs x 4 schedulers x 1 warp-instruction per
# clock at the 2070 MHz maximum SM clock.
ISSUE_PEAK_GINST = 152 * 4 * 2.070
# Warp instructions the chi kernel executes per chi event on the medium
# tissue, per launch variant, from ncu (smsp__inst_executed.sum over the 10
# timed chi launches / their chi events; profiles/k_chi_medium_metrics.md).
CHI_INST_PER_EVENT = {("persistent", 16, 0): 298.0}
# DRAM bytes (read + write) per chi launch from the same capture, per variant.
CHI_TRAFFIC = {("persistent", 16, 0): 1.314e7}
# Algorithmic DRAM bytes of one chi launch per cell: the state read + write.
STATE_BYTES_PER_CELL_RW = lambda V: 2 * 3 * V * 4  # noqa: E731


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            # nvidia-smi's start-up (driver and NVML initialisation) must not
            # overlap the timed launches: wait for its first sample
            t0 = time.perf_counter()
            while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 5.0:
                time.sleep(0.01)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for name, val in zip(names, p[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def job_totals(dist, local_ms: float, local_events: float, device="cuda"):
    """Whole-job figures over ranks: the slowest rank's time and the sum of
    all ranks' events (every rank runs its own replica; weak scaling)."""
    if dist is None:
        return local_ms, local_events
    import torch
    t = torch.tensor([local_ms, local_events], dtype=torch.float64, device=device)
    mx, sm = t.clone(), t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


def _peaks():
    try:
        with open(PEAKS) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1806_10889_gb300.tissue import DEFAULT_CHI_WPB, Tissue

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    from dataclasses import replace
    spec = {"medium": lambda: W.medium(args.dt).tissue,
            "promoter": lambda: W.promoter().tissue,
            "mixed": lambda: W.mixed_fidelity().tissue}[args.workload]()
    if args.side or args.n:  # profiling cases: same model and seed, other sizes
        spec = replace(spec, width=args.side or spec.width, height=args.side or spec.height,
                       n=args.n or spec.n)
    if world > 1:  # independent replica per rank
        spec = replace(spec, tissue_id=rank)
    g = Tissue(spec)
    if args.kernel == "persistent":
        g.set_launch_config(1, args.lanes, args.chi_wpb or 4, 0, args.layout)
    elif args.kernel == "warp":
        g.set_launch(args.chi_wpb or DEFAULT_CHI_WPB)
    launch = g.launch_config()
    burn = int(round(args.burn_in / args.dt))
    if burn:
        g.step(args.dt, burn)
    for _ in range(args.warmup):
        g.step(args.dt, 1)
    g.sync()
    # the state the timed steps start from, for the CPU baseline (untimed)
    base_state, base_step = None, 0
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not (args.side or args.n) \
            and args.workload == "medium":
        base_state, base_step = g.read_counts(), g.get_step()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    ev0 = g.total_events()
    chi_ms = sig_ms = 0.0
    step_ms = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clocks:
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (outside the event pair)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            c_ms, s_ms = g.step_timed(args.dt, 1)
            b.record(stream)
            b.synchronize()
            step_ms.append(a.elapsed_time(b))
            chi_ms += c_ms
            sig_ms += s_ms
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_wall
    ev1 = g.total_events()
    events = int((ev1 - ev0).sum())
    chi_events = int(ev1[0] - ev0[0])
    total_ms = float(sum(step_ms))
    total_ms_job, events_job = job_totals(dist, total_ms, float(events))
    value = events_job / (total_ms_job / 1e3)
    cell_steps = spec.cells * args.steps * world

    # end to end through the C ABI: pinned host state in and out every step
    e2e = None
    if not args.no_e2e:
        host = torch.empty(spec.state_ints, dtype=torch.int32, pin_memory=True)
        g.read_counts_into(host)
        e0 = g.total_events()
        k0 = g.get_step()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(args.steps):
            g.write_counts_from(host, step_index=k0 + i)   # H2D of the step's input state
            g.step(args.dt, 1)
            g.read_counts_into(host)                       # D2H of the step's result
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e_ev = float((g.total_events() - e0).sum())
        e2e_s, e_ev = job_totals(dist, e2e_s, e_ev)
        nbytes = spec.state_ints * 4
        e2e = {"value": e_ev / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes}

    peaks, peak_kind = _peaks()
    chi_s = chi_ms / 1e3
    chi_rate = chi_events / chi_s if chi_s > 0 else 0.0
    hbm_achieved = STATE_BYTES_PER_CELL_RW(spec.V) * spec.cells * args.steps / chi_s / 1e9
    variant = (["warp", "persistent"][launch[0]], launch[1], launch[4])
    ipe = (CHI_INST_PER_EVENT.get(variant)
           if not (args.side or args.n) and args.workload == "medium" else None)
    if ipe:
        ach = chi_rate * ipe / 1e9
        roofline = {"bound": "alu", "achieved": ach, "peak": ISSUE_PEAK_GINST,
                    "unit": "Gwarp-inst/s", "frac": ach / ISSUE_PEAK_GINST,
                    "traffic": args.chi_traffic or CHI_TRAFFIC.get(variant),
                    "kernel": f"k_chi ({variant[0]}, {variant[1]} lanes per cell)",
                    "inst_per_event": ipe,
                    "hbm_gbs": hbm_achieved, "hbm_frac": hbm_achieved / peaks["hbm_gbs"],
                    "peak_source": "152 SMs x 4 issue/clk x 2.070 GHz"}
    else:
        roofline = {"bound": "hbm", "achieved": hbm_achieved, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": hbm_achieved / peaks["hbm_gbs"],
                    "traffic": args.chi_traffic, "kernel": "k_chi",
                    "peak_source": f"{peak_kind} hbm_gbs"}

    # our kernels per step: chi, both face phases, the step counter; cells of
    # more than 256 voxels (Notch-Delta, persistent prefix layout) add the
    # 32-bit redo pass of the 16-bit-count chi launch
    narrow = launch[0] == 1 and launch[4] == 0 and spec.V > 256 and "kind" not in spec.model
    launches_per_step = 4 + int(narrow) + int(spec.fidelity != "lattice")
    out = {
        "metric": METRIC if args.workload == "medium" else f"SSA events/s, {args.workload} tissue",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_job / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64+f64",
        "data": "synthetic", "impl": "ours",
        "config": {"workload": f"{args.workload if not (args.side or args.n) else 'custom'} "
                               f"tissue {spec.width}x{spec.height} cells of {spec.n}x{spec.n} "
                               f"voxels, {'promoter' if 'kind' in spec.model else 'Notch-Delta'}"
                               f" model, fidelity {spec.fidelity}",
                   "dt": args.dt, "burn_in_time": args.burn_in, "cells": spec.cells,
                   "voxels_per_cell": spec.V, "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"replicas x{world}",
                   "chi_launch": {"kernel": ["warp", "persistent"][launch[0]],
                                  "lanes_per_cell": launch[1], "warps_per_block": launch[2],
                                  "smem_layout": ["prefix", "recompute"][launch[4]]}},
        "cell_steps_per_s": cell_steps / (total_ms_job / 1e3),
        "events_per_step": events_job / args.steps,
        "chi_events_per_step": chi_events / args.steps,
        "chi_ms_per_step": chi_ms / args.steps, "sig_ms_per_step": sig_ms / args.steps,
        "step_ms_median": statistics.median(step_ms), "step_ms_max": max(step_ms),
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roofline,
        "clocks": clocks.summary(),
        "wall_s_timed": wall,
    }
    g.close()
    if rank == 0 and world == 1 and not args.no_promoter:
        out["promoter"] = promoter_leg(args)
        out["mixed_fidelity"] = promoter_leg(args, W.mixed_fidelity())
    if rank == 0 and world == 1 and not args.no_batch:
        out["batched"] = batch_leg(args)
    if rank == 0 and world == 1 and args.serving:
        out["serving"] = serving_leg(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, base_state, base_step)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return out if rank == 0 else None


def promoter_leg(args, run=None) -> dict:
    """The paper's promoter Notch model (Table I rates in lattice units) on a
    64x64 tissue of 16x16-voxel cells, dt = 0.1 s, after 2 s of burn-in:
    the same timing as the main line (device-resident state, L2 flushed
    between timed steps, CUDA events on the tissue's stream).  With `run`
    (the mixed-fidelity tissue) the same for that workload."""
    import torch

    from paper_1806_10889_gb300.tissue import Tissue
    from paper_1806_10889_gb300.workloads import fidelity_mask

    run = run or W.promoter()
    g = Tissue(run.tissue)
    g.step(run.dt, 20)
    g.step(run.dt, 3)
    g.sync()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    ev0 = g.total_events()
    total_ms = chi_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        c_ms, _ = g.step_timed(run.dt, 1)
        b.record(stream)
        b.synchronize()
        total_ms += a.elapsed_time(b)
        chi_ms += c_ms
    ev = g.total_events() - ev0
    launch = g.launch_config()
    g.close()
    spec = run.tissue
    mask = fidelity_mask(spec)
    wm = int(mask.sum()) if mask is not None else 0
    return {"workload": f"promoter model, {spec.width}x{spec.height} cells of {spec.n}x{spec.n} "
                        f"voxels, dt 0.1 s, burn-in 2 s, fidelity {spec.fidelity} "
                        f"({wm} well-mixed cells)",
            "rates": {k: v for k, v in spec.model.items() if k != "kind"},
            "events_per_s": float(ev.sum()) / (total_ms / 1e3),
            "chi_events_per_s": float(ev[0]) / (chi_ms / 1e3),
            "cell_steps_per_s": spec.cells * args.steps / (total_ms / 1e3),
            "events_per_step": float(ev.sum()) / args.steps,
            "face_events_per_step": float(ev[1] + ev[2]) / args.steps,
            "ms_per_step": total_ms / args.steps, "chi_ms_per_step": chi_ms / args.steps,
            "chi_launch": {"kernel": ["warp", "persistent"][launch[0]],
                           "lanes_per_cell": launch[1], "warps_per_block": launch[2]}}


def batch_leg(args) -> dict:
    """The uneven 256-tissue batch: one persistent launch per cell-size class
    and step (graph-captured, autotuned) against the plain per-tissue launch
    (every tissue stepped by its own tissue_step call).  Both legs start from
    the same state and must end bit-identical."""
    import torch

    from paper_1806_10889_gb300 import autotune
    from paper_1806_10889_gb300.batching import Batch
    from paper_1806_10889_gb300.tissue import Tissue

    runs = W.batch()
    dt, K = runs[0].dt, args.batch_steps
    cells = sum(r.tissue.cells for r in runs)
    plain = [Tissue(r.tissue) for r in runs]
    for t in plain:
        t.step(dt, 1)
    torch.cuda.synchronize()
    ev0 = sum(int(t.total_events().sum()) for t in plain)
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(K):
        for t in plain:
            t.step(dt, 1)
    b.record(stream)
    b.synchronize()
    plain_ms = a.elapsed_time(b)
    plain_events = sum(int(t.total_events().sum()) for t in plain) - ev0

    members = [Tissue(r.tissue) for r in runs]
    torch.cuda.synchronize()
    bt = Batch(members)
    bt.step(dt, 1)
    bt.sync()
    tuned = autotune.tune_batch(members, dt, steps=1, max_clones=24) if args.autotune else None
    if tuned:
        autotune.apply_batch(bt, tuned)
    ev1 = sum(int(m.total_events().sum()) for m in members)
    a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a2.record(bt.stream)
    bt.step(dt, K)
    b2.record(bt.stream)
    b2.synchronize()
    batch_ms = a2.elapsed_time(b2)
    bt.sync()
    batch_events = sum(int(m.total_events().sum()) for m in members) - ev1
    same = all(np.array_equal(x.read_counts(), y.read_counts()) for x, y in zip(plain, members))
    bt.close()
    for t in plain + members:
        t.close()
    return {"workload": "256 uneven tissues (side 2..64, n in {8,16,32}, kD U[5,20]), dt 0.1",
            "cells": cells, "steps": K,
            "batched_events_per_s": batch_events / (batch_ms / 1e3),
            "plain_events_per_s": plain_events / (plain_ms / 1e3),
            "speedup": (batch_events / batch_ms) / (plain_events / plain_ms),
            "batched_cell_steps_per_s": cells * K / (batch_ms / 1e3),
            "batched_ms_per_step": batch_ms / K, "plain_ms_per_step": plain_ms / K,
            "bit_identical": bool(same),
            "tuned": None if not tuned else {
                "classes": {str(k): list(v) for k, v in tuned["classes"].items()},
                "steps_per_graph": tuned["steps_per_graph"]}}


def serving_leg(args) -> dict:
    """The first --serving requests of the serving workload (Poisson arrivals
    at 50 req/s, 1..64 replicas, lognormal sides, 16x16 voxels, T = 20),
    admitted by a device-memory budget and served by continuous batching;
    against the plain alternative of serving them one tissue at a time."""
    import torch

    from paper_1806_10889_gb300.serving import Server, latency_summary
    from paper_1806_10889_gb300.tissue import Tissue

    reqs = W.serving()[: args.serving]
    free, _ = torch.cuda.mem_get_info()
    srv = Server(budget_bytes=int(free * 0.6), chunk_steps=10)
    t0 = time.perf_counter()
    res = srv.run(reqs)
    wall = time.perf_counter() - t0
    out = {"requests": len(reqs), "arrivals_per_s": 50.0, "budget_bytes": srv.budget,
           "policy": f"{srv.policy} (rounds of at least {srv.fill_cells} cells)",
           "served_events_per_s": srv.device_events / wall, "wall_s": wall,
           "latency": latency_summary(res)}
    if args.serving_plain:
        ev, t1 = 0, time.perf_counter()
        for q in reqs:
            for spec in q.replica_specs():
                t = Tissue(spec)
                t.step(q.dt, q.n_steps)
                ev += int(t.total_events().sum())
                t.close()
        torch.cuda.synchronize()
        out["plain_events_per_s"] = ev / (time.perf_counter() - t1)
        out["served_vs_plain"] = out["served_events_per_s"] / out["plain_events_per_s"]
    return out


def _oracle_patch(side: int):
    import oracle as O
    spec = W.medium(0.1).tissue
    d = O.Desc(side, side, spec.n, seed=spec.seed, tissue_id=spec.tissue_id,
               init_lambda=tuple(spec.init_lambda))
    return O, d, O.Model(**spec.model)


def cpu_baseline(args, state=None, step0: int = 0, side: int = 64, budget_s: float = 10.0,
                 max_steps: int = 30):
    """The oracle, as it stands, on the benchmark tissue: whole-tissue steps
    from the state the timed GPU steps start from (after the burn-in), until
    about budget_s seconds of CPU work are done."""
    O, d, m = _oracle_patch(side)
    counts = O.init_counts(d) if state is None else np.array(state, dtype=np.int32, copy=True)
    threads = O.max_threads()
    total, steps = 0, 0
    t0 = time.perf_counter()
    while steps < max_steps and (steps == 0 or time.perf_counter() - t0 < budget_s):
        ne, _ = O.step(d, m, counts, step0 + steps, 1, args.dt, n_threads=threads)
        total += int(ne.sum())
        steps += 1
    dt_s = time.perf_counter() - t0
    start = "the state after the GPU burn-in" if state is not None else "the initial state"
    # one core: chi of the first 256 cells of the same starting state
    one = O.init_counts(d) if state is None else np.array(state, dtype=np.int32, copy=True)
    ev1, t1 = 0, time.perf_counter()
    for c in range(256):
        ev1 += O.chi_cell(d, m, one, c, step0, args.dt)[0]
    t1 = time.perf_counter() - t1
    return {"value": total / dt_s, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{side}x{side} cells of the medium tissue (16x16 voxels), {steps} steps "
                      f"from {start} (steps {step0}-{step0 + steps - 1}), dt {args.dt}, "
                      f"{total} events in {dt_s:.2f} s",
            "single_core": {"value": ev1 / t1, "unit": UNIT, "cores": 1,
                            "sample": f"chi of cells 0-255 at step {step0}, {ev1} events in "
                                      f"{t1:.2f} s"}}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    O, d, m = _oracle_patch(args.ref_side)
    counts = O.init_counts(d)
    threads = O.max_threads()
    burn = int(round(args.burn_in / args.dt))  # the same untimed burn-in as the GPU arm
    for k in range(burn + args.warmup):
        O.step(d, m, counts, k, 1, args.dt, n_threads=threads)
    total, t0 = 0, time.perf_counter()
    for k in range(burn + args.warmup, burn + args.warmup + args.steps):
        ne, _ = O.step(d, m, counts, k, 1, args.dt, n_threads=threads)
        total += int(ne.sum())
    el = time.perf_counter() - t0
    value = total / el
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64+f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "medium tissue 64x64 cells of 16x16 voxels, Notch-Delta model",
                       "dt": args.dt, "burn_in_time": args.burn_in,
                       "sample_cells": args.ref_side ** 2},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{args.ref_side}x{args.ref_side}-cell patch of the medium "
                                       f"tissue per step, after {burn} burn-in steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _gpu_rate(spec, dt, steps, burn=0, config=None):
    """Device-timed rate of `steps` splitting steps after `burn` untimed ones:
    (events/s, cell-steps/s, events per step, device ms per step)."""
    import torch

    from paper_1806_10889_gb300.tissue import Tissue

    g = Tissue(spec)
    if config:
        g.set_launch_config(*config)
    if burn:
        g.step(dt, burn)
    g.step(dt, 1)
    g.sync()
    stream = torch.cuda.current_stream()
    ev0 = g.total_events()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    g.step(dt, steps)
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b)
    ev = float((g.total_events() - ev0).sum())
    g.close()
    return ev / (ms / 1e3), spec.cells * steps / (ms / 1e3), ev / steps, ms / steps


def _cpu_rate(spec, dt, steps, burn_state=None, step0=0, cells=None, threads=0):
    """The oracle's rate: whole-tissue steps (all cores) or, with `cells`,
    chi of those cells only (one core is enough for a subset)."""
    import oracle as O
    d = O.Desc(spec.width, spec.height, spec.n, seed=spec.seed, tissue_id=spec.tissue_id,
               init_lambda=tuple(spec.init_lambda))
    m = O.Model(**spec.model)
    if burn_state is not None:
        counts = np.array(burn_state, copy=True)
    elif cells is None:
        counts = O.init_counts(d)
    else:  # only the cells timed need initial counts
        counts = np.zeros(spec.cells * 3 * spec.V, dtype=np.int32)
        for c in cells:
            O.init_cell(d, counts, int(c))
    threads = threads or O.max_threads()
    t0, ev = time.perf_counter(), 0
    if cells is None:
        for k in range(steps):
            ne, _ = O.step(d, m, counts, step0 + k, 1, dt, n_threads=threads)
            ev += int(ne.sum())
        return ev / (time.perf_counter() - t0), threads
    for c in cells:
        ev += O.chi_cell(d, m, counts, int(c), step0, dt)[0]
    return ev / (time.perf_counter() - t0), 1


def run_suite(args) -> dict:
    """Every configuration of the benchmark suite on this GPU, with the
    oracle beside it (host cores, all and one), for the results table."""
    from paper_1806_10889_gb300.tissue import Tissue

    out = {}
    peaks, _ = _peaks()
    hbm = peaks["hbm_gbs"] * 1e9

    def row(name, spec, dt, steps, burn, cpu_steps=2, cpu_cells=256):
        ev_s, cs_s, ev_step, ms = _gpu_rate(spec, dt, steps, burn)
        state = None
        if burn:  # the oracle starts from the same burned-in state
            g = Tissue(spec)
            g.step(dt, burn)
            state, step0 = g.read_counts(), g.get_step()
            g.close()
        else:
            step0 = 0
        all_cores, thr = _cpu_rate(spec, dt, cpu_steps, state, step0) if cpu_steps else (None, 0)
        one_core, _ = _cpu_rate(spec, dt, 1, state, step0,
                                cells=range(min(cpu_cells, spec.cells)))
        out[name] = {"gpu_events_per_s": ev_s, "gpu_cell_steps_per_s": cs_s,
                     "events_per_step": ev_step, "gpu_ms_per_step": ms,
                     "hbm_frac": 24 * spec.V * cs_s / hbm,
                     "cpu_events_per_s": all_cores, "cpu_cores": thr,
                     "cpu_1core_events_per_s": one_core,
                     "cpu_sample": f"{cpu_steps} whole-tissue steps (all cores); chi of "
                                   f"{min(cpu_cells, spec.cells)} cells (one core)",
                     "dt": dt, "burn_in_steps": burn, "timed_steps": steps}

    tiny = W.tiny()
    row("tiny", tiny.tissue, tiny.dt, tiny.n_steps, 0, cpu_steps=tiny.n_steps)
    for dt, burn, steps in ((0.01, 2000, 50), (0.1, 200, 10), (1.0, 20, 3)):
        row(f"medium_dt{dt}", W.medium(dt).tissue, dt, steps, burn, cpu_steps=2 if dt < 1 else 1)
    lg = W.large()
    row("large", lg.tissue, lg.dt, 2, 0, cpu_steps=0, cpu_cells=128)
    out["large"]["cpu_sample"] = "chi of 128 cells at step 0 (one core); all cores not run"
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--dt", type=float, default=0.1, choices=[0.01, 0.1, 1.0])
    ap.add_argument("--burn-in", type=float, default=20.0, help="untimed simulated time first")
    ap.add_argument("--chi-wpb", type=int, default=0)
    ap.add_argument("--kernel", choices=["default", "warp", "persistent"], default="default")
    ap.add_argument("--lanes", type=int, choices=[8, 16, 32], default=16)
    ap.add_argument("--layout", type=int, choices=[0, 1], default=0,
                    help="persistent kernel: 0 prefix arrays, 1 recompute")
    ap.add_argument("--chi-traffic", type=float, default=None,
                    help="DRAM bytes per chi launch from an ncu capture, if known")
    ap.add_argument("--ref-side", type=int, default=16)
    ap.add_argument("--side", type=int, default=0, help="profiling only: tissue side in cells")
    ap.add_argument("--n", type=int, default=0, help="profiling only: voxels per cell side")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-vs-plain leg")
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--autotune", type=int, default=1)
    ap.add_argument("--workload", choices=["medium", "promoter", "mixed"], default="medium",
                    help="main line: the medium Notch-Delta tissue (the benchmark), or the "
                         "promoter or mixed-fidelity tissue (profiling)")
    ap.add_argument("--no-promoter", action="store_true",
                    help="skip the promoter-model and mixed-fidelity legs")
    ap.add_argument("--serving", type=int, default=4,
                    help="serve the first K requests of the serving workload (0: skip)")
    ap.add_argument("--serving-plain", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--suite", action="store_true",
                    help="measure every configuration of the suite (GPU and oracle) and print "
                         "one JSON object instead of the benchmark line (several minutes)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    rank, world, local_rank = _env_rank()
    if args.suite:
        print(json.dumps(run_suite(args)))
        return
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world, local_rank)
    if rank == 0 and out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
