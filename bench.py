"""Benchmark of the operator-split tissue SSA on GB300.

Headline (`value`): the uneven 256-tissue batch -- tissue sides drawn from
2..64 cells, cells of 8x8, 16x16 or 32x32 voxels, D production drawn from
[5, 20] per tissue, the Notch-Delta model, dt = 0.1 (synthetic, seeded) --
advanced by the batched path: one persistent chi launch per cell-size class
and one launch per face phase per step, captured in a CUDA graph, launch
shapes picked by the autotuner.  One "step" is one Lie splitting step of the
whole hot path (chi on every cell of every tissue, then S on every x-face and
every y-face) over all 256 tissues.  The batch is first advanced by an untimed
burn-in (default 5 time units of the configuration's 20), so the timed steps
see molecule counts well on their way to their working level; then W warm-up
and K timed steps run.  The state (about 2 GB) is larger than L2, so no flush
is needed between steps.

Metric: SSA events per second (all events of chi and both face phases), with
cell-steps per second beside it and the plain per-tissue launch (every tissue
its own tissue_step) from the same state.  `value` times the steps with the
state resident in device memory (CUDA events on the batch stream); `e2e`
times batch steps through the C ABI with every tissue's state copied
host->device before and device->host after every step.  `roofline` is the SM
issue fraction of the dominant chi launch, from its live CUDA-event time and
the warp instructions per event ncu measured for that kernel instantiation.
`cpu_baseline` is the oracle on a sample of member tissues from the same
state, which must also agree bit for bit with the GPU (`parity_checked`).

Extra keys: `medium` (64x64 cells of 16x16 voxels, the single-tissue line with
its own roofline, e2e and oracle check), `large` (256x256 cells of 32x32
voxels from a burned-in state), `promoter`, `mixed_fidelity` and `serving`
(p50/p99 latency at a sustainable arrival rate beside saturation throughput).

Multi-GPU (torchrun, N ranks): every rank advances its own copy of the batch
(tissue ids offset by rank); there is no data exchange (weak scaling).

`--impl reference` times the CPU oracle (test infrastructure, plain C with
OpenMP) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time
from dataclasses import replace

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1806_10889_gb300 import workloads as W  # noqa: E402

METRIC = "SSA events/s (chi + face binding), 256-tissue uneven batch, batched, dt 0.1"
MEDIUM_METRIC = "SSA events/s (chi + face binding), medium tissue 64x64 cells x 16x16 voxels, dt 0.1"
UNIT = "events/s"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Issue-slot peak of the chip: 152 SMs x 4 schedulers x 1 warp-instruction per
# clock at the 2070 MHz maximum SM clock.
ISSUE_PEAK_GINST = 152 * 4 * 2.070
CSRC = os.path.join(ROOT, "paper_1806_10889_gb300", "csrc")
# The files that fix the persistent chi kernel's instruction stream.
CHI_SOURCES = ["chi_seg.cuh", "tissue_dev.cuh", "tissue_internal.h", "k_chi_seg.cu",
               "k_chi_seg_narrow.cu", "k_chi_seg_gen.cu", "k_chi_seg_pm.cu"]
# Warp instructions and DRAM bytes per chi event of each
# instantiation of the persistent chi kernel (lanes per cell, layout, QB, model
# code, 16-bit counts), measured by ncu (smsp__inst_executed.sum and
# dram__bytes_{read,write}.sum over the chi launches of the command in
# profiles/k_chi_inst_per_event_by_cell_size.md, divided by their chi events).
# `sources` is chi_sources_sha() of the kernel they were measured on: when the
# kernel changes, the figures are stale and the roofline reports none.
CHI_IPE = {
    "sources": "60a170fec9320f83",
    "kernels": {
        "batch:V1024/H16/rec/qb1/nd/u16": (396.1, 0.6815),
        "batch:V256/H16/pre/qb0/nd/u32": (302.0, 0.4476),
        "batch:V64/H8/pre/qb0/nd/u32": (170.8, 0.5267),
        "medium:V256/H16/pre/qb0/nd/u32": (297.5, 0.3128),
        "large:V1024/H16/rec/qb1/nd/u16": (389.5, 1.3076),
        # launch shapes the autotuner may pick for the batch classes
        "batch:V1024/H32/pre/qb0/nd/u16": (543.6, 0.6815),
        "batch:V1024/H16/pre/qb1/nd/u16": (361.1, 0.6835),
        "batch:V1024/H32/rec/qb0/nd/u16": (628.6, 0.6813),
        "batch:V256/H8/pre/qb1/nd/u32": (206.9, 0.4517),
        "batch:V256/H8/rec/qb1/nd/u32": (226.9, 0.4469),
        "batch:V256/H32/pre/qb0/nd/u32": (551.6, 0.4475),
        "batch:V64/H16/pre/qb0/nd/u32": (305.6, 0.5301),
        "batch:V64/H32/pre/qb0/nd/u32": (551.9, 0.5321),
        "batch:V64/H8/rec/qb0/nd/u32": (239.3, 0.5607),
    },
}


def _code_of(name: str, text: str) -> str:
    """The part of a source file that fixes the kernel's instructions: the
    text without comments or blank lines; of tissue_internal.h only the device
    structures and constants before its host-side launcher declarations."""
    if name == "tissue_internal.h":
        text = text[:text.index("cudaError_t launch_")]
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*", "", ln).rstrip() for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln.strip())


def chi_sources_sha(read=None) -> str:
    """SHA-256 over the persistent chi kernel's code (comments stripped) and
    the nvcc flags.  read(name) returns a source's text (default: the files
    in csrc/)."""
    from paper_1806_10889_gb300.build import NVCC_FLAGS
    if read is None:
        def read(name):
            with open(os.path.join(CSRC, name)) as fh:
                return fh.read()
    h = hashlib.sha256()
    for f in CHI_SOURCES:
        h.update(f.encode() + b"\0" + _code_of(f, read(f)).encode())
    h.update(" ".join(x for x in NVCC_FLAGS if not x.startswith("-I")).encode())
    return h.hexdigest()[:16]


def chi_kernel_key(V: int, lanes: int, layout: int, model: str = "nd") -> str:
    """The cell size and the kernel instantiation the launcher picks for it
    (the instructions per event depend on both)."""
    qb = V > lanes * lanes
    narrow = model == "nd" and V > 256
    return (f"V{V}/H{lanes}/{'pre' if layout == 0 else 'rec'}/qb{int(qb)}/{model}/"
            f"{'u16' if narrow else 'u32'}")


def chi_ipe(workload: str, key: str):
    """(warp instructions per chi event, DRAM bytes per chi event) of a kernel
    instantiation on a workload, or None when unmeasured or measured on other
    kernel sources."""
    if CHI_IPE["sources"] != chi_sources_sha():
        return None
    return CHI_IPE["kernels"].get(f"{workload}:{key}")


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


def _events(tissues) -> np.ndarray:
    """Cumulative (chi, x-face, y-face) events of each tissue: [len, 3]."""
    return np.array([t.total_events() for t in tissues], dtype=np.int64).reshape(-1, 3)


def _digest(tissues) -> str:
    h = hashlib.sha256()
    for t in tissues:
        h.update(t.read_counts().tobytes())
    return h.hexdigest()


def issue_roofline(workload: str, chi_events: float, chi_ms: float, key: str, V: int,
                   cells: int, steps: int, launches: int) -> dict:
    """Issue-bound roofline of one chi launch class: achieved = warp
    instructions (events x measured instructions per event) per second of its
    live CUDA-event time.  HBM fraction of the algorithmic state traffic
    (24 V bytes per cell-step) beside it."""
    peaks, peak_kind = _peaks()
    chi_s = chi_ms / 1e3
    rate = chi_events / chi_s if chi_s > 0 else 0.0
    hbm = 24 * V * cells * steps / chi_s / 1e9 if chi_s > 0 else 0.0
    m = chi_ipe(workload, key)
    out = {"bound": "alu", "unit": "Gwarp-inst/s", "peak": ISSUE_PEAK_GINST,
           "peak_source": "152 SMs x 4 issue/clk x 2.070 GHz", "kernel": f"k_chi_seg {key}",
           "chi_events_per_s": rate, "launch_ms": chi_ms / max(launches, 1),
           "hbm_gbs": hbm, "hbm_frac": hbm / peaks["hbm_gbs"], "hbm_peak_source": peak_kind}
    if m is None:
        out.update({"achieved": None, "frac": None, "traffic": None, "inst_per_event": None,
                    "stale": "no instruction count measured on the current kernel sources"})
        return out
    ipe, traffic_per_event = m
    ach = rate * ipe / 1e9
    out.update({"achieved": ach, "frac": ach / ISSUE_PEAK_GINST, "inst_per_event": ipe,
                "traffic": (traffic_per_event * chi_events / max(launches, 1)
                            if traffic_per_event is not None else None)})
    return out


# ---------------------------------------------------------------------------
# Headline: the batch
# ---------------------------------------------------------------------------

def batch_runs(rank: int = 0):
    runs = W.batch()
    if rank:
        runs = [replace(r, tissue=replace(r.tissue, tissue_id=rank * len(runs) + i))
                for i, r in enumerate(runs)]
    return runs


def oracle_sample(runs, per_class: int = 1, target_cells: int = 256):
    """Indices of the member tissues the oracle reruns: per cell size, the
    tissue(s) whose cell count is nearest target_cells (enough cells to keep
    the host cores busy, few enough to run in seconds)."""
    pick = []
    for n in (8, 16, 32):
        idx = [i for i, r in enumerate(runs) if r.tissue.n == n]
        idx.sort(key=lambda i: (abs(runs[i].tissue.cells - target_cells), i))
        pick += idx[:per_class]
    return sorted(pick)


def _orc(spec):
    import oracle as O
    d = O.Desc(spec.width, spec.height, spec.n, seed=spec.seed, tissue_id=spec.tissue_id,
               init_lambda=tuple(spec.init_lambda))
    return O, d, O.Model(**spec.model)


def oracle_check(items, steps: int, dt: float) -> dict:
    """Rerun each sampled tissue with the oracle from its GPU start state for
    `steps` steps (all host cores, timed) and compare counts and the last
    step's statistics bit for bit with the GPU's.

    items: (spec, start counts, start step, gpu counts, gpu n_events, gpu t_last)."""
    total_ev, total_s, ok, cores, detail = 0, 0.0, True, 1, []
    for spec, start, step0, g_counts, g_ne, g_tl in items:
        O, d, m = _orc(spec)
        counts = np.array(start, dtype=np.int32, copy=True)
        cores = O.max_threads()
        t0 = time.perf_counter()
        ev = 0
        for k in range(steps):
            ne, tl = O.step(d, m, counts, step0 + k, 1, dt, n_threads=cores)
            ev += int(ne.sum())
        el = time.perf_counter() - t0
        same = (np.array_equal(counts, g_counts) and np.array_equal(ne, g_ne)
                and np.array_equal(tl.view(np.uint64), g_tl.view(np.uint64)))
        ok &= same
        total_ev += ev
        total_s += el
        detail.append({"tissue_id": spec.tissue_id, "cells": spec.cells, "n": spec.n,
                       "steps": f"{step0}-{step0 + steps - 1}", "events": ev, "bit_exact": same})
    return {"parity_checked": bool(ok), "events": total_ev, "seconds": total_s, "cores": cores,
            "tissues": detail}


def oracle_single_core(spec, start, step0, dt, cells: int = 32) -> dict:
    O, d, m = _orc(spec)
    counts = np.array(start, dtype=np.int32, copy=True)
    ev, t0 = 0, time.perf_counter()
    for c in range(min(cells, spec.cells)):
        ev += O.chi_cell(d, m, counts, c, step0, dt)[0]
    el = time.perf_counter() - t0
    return {"value": ev / el, "unit": UNIT, "cores": 1,
            "sample": f"chi of cells 0-{min(cells, spec.cells) - 1} of tissue {spec.tissue_id} "
                      f"({spec.n}x{spec.n} voxels) at step {step0}, {ev} events in {el:.2f} s"}


def batch_headline(args, rank: int, world: int, dist) -> dict:
    import torch

    from paper_1806_10889_gb300 import autotune
    from paper_1806_10889_gb300.batching import Batch
    from paper_1806_10889_gb300.tissue import Tissue

    runs = batch_runs(rank)
    dt = runs[0].dt
    members = [Tissue(r.tissue) for r in runs]
    torch.cuda.synchronize()
    bt = Batch(members)
    burn = int(round(args.batch_burn_in / dt))
    t_burn = time.perf_counter()
    if burn:
        bt.step(dt, burn)
        bt.sync()
    t_burn = time.perf_counter() - t_burn
    tuned = None
    if args.autotune:
        tuned = autotune.tune_batch(members, dt, steps=1, max_clones=args.tune_clones)
        autotune.apply_batch(bt, tuned)
    # the timed steps replay one step per graph so that each is timed
    bt.set_schedule(1)
    # overlapped or sequential classes: chosen from 4 steps of the batch
    # itself (before the warm-up steps), or forced
    overlap_tune = None
    if args.class_overlap == "auto":
        overlap_tune = autotune.tune_overlap(bt, dt)
    else:
        bt.set_overlap(args.class_overlap == "on")
    bt.set_timing(True)
    for _ in range(args.warmup):
        bt.step(dt, 1)
    bt.sync()
    classes = bt.classes()
    step0 = members[0].get_step()
    sample = oracle_sample(runs, per_class=args.oracle_per_class) if (
        rank == 0 and world == 1 and not args.no_cpu_baseline) else []
    starts = {i: members[i].read_counts() for i in sample}

    ev0 = _events(members)
    step_ms, class_ms, chi_ms = [], np.zeros(len(classes)), 0.0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clocks:
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(bt.stream)
            bt.step(dt, 1)
            b.record(bt.stream)
            b.synchronize()
            step_ms.append(a.elapsed_time(b))
            _, c, _, cls = bt.read_timing()
            chi_ms += c
            class_ms += np.array(cls)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_wall
    bt.sync()
    ev1 = _events(members)
    bt.set_timing(False)
    d_ev = ev1 - ev0
    events = int(d_ev.sum())
    total_ms = float(sum(step_ms))
    total_ms_job, events_job = job_totals(dist, total_ms, float(events))
    cells = sum(r.tissue.cells for r in runs)
    after = {i: (members[i].read_counts(), *members[i].read_stats()) for i in sample}

    # the chi phase's classes run overlapped (one launch per class, all
    # ready at the phase's start): the roofline covers the phase as a whole,
    # warp instructions of every class (its events x its measured
    # instructions per event) over the phase's live time; a class's span
    # runs from when its launch became ready (overlapped: the phase's start)
    # to its last block
    per_class, inst, traffic, stale = [], 0.0, 0.0, False
    for ci, c in enumerate(classes):
        idx = [i for i, r in enumerate(runs) if r.tissue.V == c["V"]]
        key = chi_kernel_key(c["V"], c["lanes_per_cell"], c["smem_layout"])
        ev_c = float(d_ev[idx, 0].sum())
        m = chi_ipe("batch", key)
        if m is None:
            stale = True
        else:
            inst += ev_c * m[0]
            traffic = None if traffic is None or m[1] is None else traffic + ev_c * m[1]
        per_class.append({"V": c["V"], "cells": c["cells"], "tissues": len(idx),
                          "launch": [c["lanes_per_cell"], c["warps_per_block"], c["smem_layout"]],
                          "kernel": f"k_chi_seg {key}",
                          "span_ms_per_step": class_ms[ci] / args.steps,
                          "chi_events_per_step": ev_c / args.steps,
                          "inst_per_event": None if m is None else m[0]})
    peaks, peak_kind = _peaks()
    chi_s = chi_ms / 1e3
    chi_events = float(d_ev[:, 0].sum())
    hbm = sum(24 * c["V"] * c["cells"] for c in classes) * args.steps / chi_s / 1e9
    roofline = {"bound": "alu", "unit": "Gwarp-inst/s", "peak": ISSUE_PEAK_GINST,
                "peak_source": "152 SMs x 4 issue/clk x 2.070 GHz",
                "kernel": "k_chi_seg, one launch per cell-size class, " +
                          ("overlapped" if bt.overlap else "one after another"),
                "chi_events_per_s": chi_events / chi_s, "launch_ms": chi_ms / args.steps,
                "hbm_gbs": hbm, "hbm_frac": hbm / peaks["hbm_gbs"], "hbm_peak_source": peak_kind}
    if stale:
        roofline.update({"achieved": None, "frac": None, "traffic": None, "inst_per_event": None,
                         "stale": "no instruction count measured on the current kernel sources"})
    else:
        ach = inst / chi_s / 1e9
        roofline.update({"achieved": ach, "frac": ach / ISSUE_PEAK_GINST,
                         "inst_per_event": inst / chi_events,
                         "traffic": None if traffic is None else traffic / args.steps})

    # end to end through the C ABI: every tissue's state from pinned host
    # memory before each step, back to pinned host memory after it (the
    # batch's state I/O: all copies queued on the batch stream, one wait)
    e2e = None
    hosts = [torch.empty(m.spec.state_ints, dtype=torch.int32, pin_memory=True) for m in members]
    for m, h in zip(members, hosts):
        m.read_counts_into(h)
    if args.e2e_steps:
        k0 = members[0].get_step()
        e0 = _events(members)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        phases = np.zeros((args.e2e_steps, 3))  # host wall s: write, step (to its end), read
        t0 = time.perf_counter()
        for i in range(args.e2e_steps):
            ta = time.perf_counter()
            bt.write_counts(hosts, step_index=k0 + i)  # H2D of every member's input state
            tb = time.perf_counter()
            bt.step(dt, 1)
            bt.sync()
            tc = time.perf_counter()
            bt.read_counts(hosts)                      # D2H of every member's result
            phases[i] = (tb - ta, tc - tb, time.perf_counter() - tc)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e_ev = float((_events(members) - e0).sum())
        e2e_s, e_ev = job_totals(dist, e2e_s, e_ev)
        nbytes = sum(r.tissue.state_ints * 4 for r in runs)
        e2e = {"value": e_ev / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": args.e2e_steps,
               "ms_per_step": {"write": [round(1e3 * x, 2) for x in phases[:, 0]],
                               "step": [round(1e3 * x, 2) for x in phases[:, 1]],
                               "read": [round(1e3 * x, 2) for x in phases[:, 2]]}}

    # plain per-tissue launches against the batch, from the same state
    plain = None
    if args.plain_steps and rank == 0 and world == 1:
        k_now = members[0].get_step()
        clones = [Tissue(r.tissue) for r in runs]
        for c, h in zip(clones, hosts):
            c.write_counts_from(h, step_index=k_now)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        p0 = _events(clones)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.plain_steps):
            for c in clones:
                c.step(dt, 1)
        b.record(stream)
        b.synchronize()
        plain_ms = a.elapsed_time(b)
        plain_ev = float((_events(clones) - p0).sum())
        q0 = _events(members)
        a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a2.record(bt.stream)
        bt.step(dt, args.plain_steps)
        b2.record(bt.stream)
        b2.synchronize()
        bt.sync()
        same_ms = a2.elapsed_time(b2)
        same_ev = float((_events(members) - q0).sum())
        same = _digest(clones) == _digest(members)
        plain = {"plain_events_per_s": plain_ev / (plain_ms / 1e3),
                 "batched_events_per_s": same_ev / (same_ms / 1e3),
                 "batched_vs_plain": (same_ev / same_ms) / (plain_ev / plain_ms),
                 "steps": args.plain_steps, "from_step": k_now, "bit_identical": bool(same)}
        for c in clones:
            c.close()

    bt.close()
    for m in members:
        m.close()
    del hosts

    cpu = None
    if sample:
        items = [(runs[i].tissue, starts[i], step0, *after[i]) for i in sample]
        chk = oracle_check(items, args.steps, dt)
        i_big = max(sample, key=lambda i: runs[i].tissue.V)
        cpu = {"value": chk["events"] / chk["seconds"], "unit": UNIT, "cores": chk["cores"],
               "kind": "oracle",
               "sample": f"{len(sample)} member tissues of the batch (one per cell size, "
                         f"{sum(runs[i].tissue.cells for i in sample)} cells), the {args.steps} "
                         f"timed steps {step0}-{step0 + args.steps - 1} from the GPU's state, "
                         f"{chk['events']} events in {chk['seconds']:.2f} s",
               "parity_checked": chk["parity_checked"], "tissues": chk["tissues"],
               "single_core": oracle_single_core(runs[i_big].tissue, starts[i_big], step0, dt)}

    out = {
        "metric": METRIC, "value": events_job / (total_ms_job / 1e3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms_job / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64+f64", "data": "synthetic", "impl": "ours",
        "config": {"workload": "256 uneven tissues (side U{2..64} cells, cells of 8x8, 16x16 "
                               "or 32x32 voxels, kD U[5,20]), Notch-Delta model, batched",
                   "dt": dt, "burn_in_time": args.batch_burn_in, "timed_steps_from": step0,
                   "config_steps": runs[0].n_steps, "cells": cells, "tissues": len(runs),
                   "state_bytes": sum(r.tissue.state_ints * 4 for r in runs),
                   "l2": "state (~2 GB) larger than L2; no flush",
                   "parallelism": f"replicas x{world}", "graph": "one step per captured graph",
                   "classes_overlapped": bt.overlap, "overlap_tuning": overlap_tune,
                   "tuned": None if not tuned else {
                       "classes": {str(k): list(v) for k, v in tuned["classes"].items()},
                       "steps_per_graph": tuned["steps_per_graph"]}},
        "cell_steps_per_s": cells * world * args.steps / (total_ms_job / 1e3),
        "events_per_step": events_job / args.steps,
        "chi_events_per_step": float(d_ev[:, 0].sum()) / args.steps,
        "step_ms_median": statistics.median(step_ms), "step_ms_max": max(step_ms),
        "chi_ms_per_step": chi_ms / args.steps,
        "sig_ms_per_step": (total_ms - chi_ms) / args.steps,
        "classes": per_class,
        "e2e": e2e,
        "gpu_launches": None,
        "roofline": roofline,
        "clocks": clocks.summary(),
        "wall_s_timed": wall,
        "burn_in_wall_s": t_burn,
        "plain": plain,
        "cpu_baseline": cpu,
        "parity_checked": None if cpu is None else cpu["parity_checked"],
    }
    # our kernels per step: per class the chi launch (and, for cells of more
    # than 256 voxels with 16-bit counts, its 32-bit redo pass), both face
    # phases and the step-counter update
    per_step = sum(1 + int(chi_kernel_key(c["V"], c["lanes_per_cell"], c["smem_layout"])
                           .endswith("u16")) for c in classes) + 3
    out["gpu_launches"] = per_step * args.steps
    return out


# ---------------------------------------------------------------------------
# Single tissues
# ---------------------------------------------------------------------------

def medium_leg(args) -> dict:
    """The medium tissue (64x64 cells of 16x16 voxels, dt 0.1) after 20 time
    units of burn-in: K steps device-timed with the L2 flushed between steps,
    e2e through the C ABI, its chi roofline, and the oracle rerunning the same
    K steps from the same state, compared bit for bit."""
    import torch

    from paper_1806_10889_gb300.tissue import Tissue

    spec = W.medium(args.dt).tissue
    if args.side or args.n:  # profiling cases: same model and seed, other sizes
        spec = replace(spec, width=args.side or spec.width, height=args.side or spec.height,
                       n=args.n or spec.n)
    g = Tissue(spec)
    if args.kernel == "persistent":
        g.set_launch_config(1, args.lanes, args.chi_wpb or 4, 0, args.layout)
    launch = g.launch_config()
    burn = int(round(args.burn_in / args.dt))
    if burn:
        g.step(args.dt, burn)
    for _ in range(args.warmup):
        g.step(args.dt, 1)
    g.sync()
    check = not args.no_cpu_baseline and not (args.side or args.n)
    base_state, base_step = (g.read_counts(), g.get_step()) if check else (None, g.get_step())
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    ev0 = g.total_events()
    chi_ms = sig_ms = 0.0
    step_ms = []
    torch.cuda.synchronize()
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
    ev1 = g.total_events()
    after = (g.read_counts(), *g.read_stats()) if check else None
    events = int((ev1 - ev0).sum())
    chi_events = int(ev1[0] - ev0[0])
    total_ms = float(sum(step_ms))

    host = torch.empty(spec.state_ints, dtype=torch.int32, pin_memory=True)
    g.read_counts_into(host)
    e0 = g.total_events()
    k0 = g.get_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        g.write_counts_from(host, step_index=k0 + i)   # H2D of the step's input state
        g.step(args.dt, 1)
        g.read_counts_into(host)                       # D2H of the step's result
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e_ev = float((g.total_events() - e0).sum())
    nbytes = spec.state_ints * 4
    g.close()

    key = chi_kernel_key(spec.V, launch[1], launch[4]) if launch[0] == 1 else "warp"
    out = {"metric": MEDIUM_METRIC, "value": events / (total_ms / 1e3), "unit": UNIT,
           "workload": f"tissue {spec.width}x{spec.height} cells of {spec.n}x{spec.n} voxels, "
                       f"Notch-Delta model, dt {args.dt}, burn-in {args.burn_in} time units, "
                       "L2 flushed between timed steps (256 MB write)",
           "steps": args.steps, "timed_steps_from": base_step,
           "ms_per_step": total_ms / args.steps,
           "cell_steps_per_s": spec.cells * args.steps / (total_ms / 1e3),
           "events_per_step": events / args.steps, "chi_events_per_step": chi_events / args.steps,
           "chi_ms_per_step": chi_ms / args.steps, "sig_ms_per_step": sig_ms / args.steps,
           "step_ms_median": statistics.median(step_ms), "step_ms_max": max(step_ms),
           "chi_launch": {"kernel": ["warp", "persistent"][launch[0]],
                          "lanes_per_cell": launch[1], "warps_per_block": launch[2],
                          "smem_layout": ["prefix", "recompute"][launch[4]]},
           "e2e": {"value": e_ev / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                   "d2h_bytes_per_step": nbytes},
           "roofline": issue_roofline("medium", chi_events, chi_ms, key, spec.V, spec.cells,
                                      args.steps, args.steps)}
    if check:
        chk = oracle_check([(spec, base_state, base_step, *after)], args.steps, args.dt)
        out["parity_checked"] = chk["parity_checked"]
        out["cpu_baseline"] = {"value": chk["events"] / chk["seconds"], "unit": UNIT,
                               "cores": chk["cores"], "kind": "oracle",
                               "sample": f"the whole tissue, the {args.steps} timed steps "
                                         f"{base_step}-{base_step + args.steps - 1} from the GPU's "
                                         f"state, {chk['events']} events in "
                                         f"{chk['seconds']:.2f} s",
                               "single_core": oracle_single_core(spec, base_state, base_step,
                                                                 args.dt, cells=256)}
    return out


def _timed_tissue(spec, dt: float, burn: int, steps: int, flush: bool = True) -> dict:
    """Device-timed steps of one tissue after `burn` untimed ones."""
    import torch

    from paper_1806_10889_gb300.tissue import Tissue

    g = Tissue(spec)
    if burn:
        g.step(dt, burn)
    g.step(dt, 3)
    g.sync()
    buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda") if flush else None
    stream = torch.cuda.current_stream()
    ev0 = g.total_events()
    k0 = g.get_step()
    total_ms = chi_ms = 0.0
    for _ in range(steps):
        if buf is not None:
            buf.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        c_ms, _ = g.step_timed(dt, 1)
        b.record(stream)
        b.synchronize()
        total_ms += a.elapsed_time(b)
        chi_ms += c_ms
    ev = g.total_events() - ev0
    launch = g.launch_config()
    g.close()
    return {"events_per_s": float(ev.sum()) / (total_ms / 1e3),
            "chi_events_per_s": float(ev[0]) / (chi_ms / 1e3),
            "cell_steps_per_s": spec.cells * steps / (total_ms / 1e3),
            "events_per_step": float(ev.sum()) / steps,
            "face_events_per_step": float(ev[1] + ev[2]) / steps,
            "ms_per_step": total_ms / steps, "chi_ms_per_step": chi_ms / steps,
            "steps": steps, "timed_steps_from": k0, "chi_ev": float(ev[0]), "chi_ms": chi_ms,
            "chi_launch": {"kernel": ["warp", "persistent"][launch[0]],
                           "lanes_per_cell": launch[1], "warps_per_block": launch[2],
                           "smem_layout": launch[4]}}


def promoter_leg(args, run=None) -> dict:
    """The paper's promoter Notch model (Table I rates in lattice units) on a
    64x64 tissue of 16x16-voxel cells, dt = 0.1 s, after 2 s of burn-in.  With
    `run` (the mixed-fidelity tissue) the same for that workload."""
    from paper_1806_10889_gb300.workloads import fidelity_mask

    run = run or W.promoter()
    spec = run.tissue
    r = _timed_tissue(spec, run.dt, 20, args.steps)
    mask = fidelity_mask(spec)
    wm = int(mask.sum()) if mask is not None else 0
    r.pop("chi_ev")
    r.pop("chi_ms")
    r.update({"workload": f"promoter model, {spec.width}x{spec.height} cells of {spec.n}x{spec.n} "
                          f"voxels, dt 0.1 s, burn-in 2 s, fidelity {spec.fidelity} "
                          f"({wm} well-mixed cells)",
              "rates": {k: v for k, v in spec.model.items() if k != "kind"}})
    return r


def large_leg(args) -> dict:
    """The large tissue (256x256 cells of 32x32 voxels, 0.8 GB of state, larger
    than L2) from a burned-in state, with its chi roofline."""
    lg = W.large()
    burn = int(round(args.large_burn_in / lg.dt))
    r = _timed_tissue(lg.tissue, lg.dt, burn, args.large_steps, flush=False)
    cl = r["chi_launch"]
    key = chi_kernel_key(lg.tissue.V, cl["lanes_per_cell"], cl["smem_layout"])
    r["roofline"] = issue_roofline("large", r.pop("chi_ev"), r.pop("chi_ms"), key, lg.tissue.V,
                                   lg.tissue.cells, args.large_steps, args.large_steps)
    r["workload"] = (f"tissue 256x256 cells of 32x32 voxels, Notch-Delta model, dt 0.1, "
                     f"burn-in {args.large_burn_in} time units; state larger than L2, no flush")
    return r


# ---------------------------------------------------------------------------
# Serving
# ---------------------------------------------------------------------------

def serving_requests(count: int, max_replicas: int):
    """The first `count` requests of the serving workload with at most
    `max_replicas` replicas each (the request mix, sides and seeds unchanged)."""
    return [replace(q, replicas=min(q.replicas, max_replicas)) for q in W.serving()[:count]]


def serving_leg(args) -> dict:
    """Continuous-batching server on `--serving` requests of the serving
    workload (replicas capped at --serving-replicas so that one GB300 can keep
    up): saturation throughput with every request arriving at the workload's
    50 req/s, then p50/p99 latency with the arrival gaps stretched to a
    sustainable rate (a fraction of the measured saturation rate), and the
    plain one-tissue-at-a-time rate on the first few requests."""
    import torch

    from paper_1806_10889_gb300.serving import Server, latency_summary
    from paper_1806_10889_gb300.tissue import Tissue

    reqs = serving_requests(args.serving, args.serving_replicas)
    free, _ = torch.cuda.mem_get_info()
    budget = int(free * 0.6)
    srv = Server(budget_bytes=budget, chunk_steps=10)
    t0 = time.perf_counter()
    res = srv.run(reqs)
    wall = time.perf_counter() - t0
    sat = {"arrivals_per_s": 50.0, "wall_s": wall, "served_events_per_s": srv.device_events / wall,
           "requests_per_s": len(reqs) / wall, "latency": latency_summary(res),
           "rebuilds": srv.rebuilds, "rebuild_s": srv.rebuild_s}
    out = {"requests": len(reqs), "max_replicas": args.serving_replicas, "budget_bytes": budget,
           "policy": f"{srv.policy} (rounds of at least {srv.fill_cells} cells)",
           "saturation": sat}
    # a sustainable rate: arrivals at args.serving_load x the saturation rate
    rate = args.serving_load * sat["requests_per_s"]
    scale = 50.0 / rate
    srv2 = Server(budget_bytes=budget, chunk_steps=10)
    t0 = time.perf_counter()
    res2 = srv2.run(reqs, time_scale=scale)
    wall2 = time.perf_counter() - t0
    out["sustained"] = {"arrivals_per_s": rate, "time_scale": scale, "wall_s": wall2,
                        "served_events_per_s": srv2.device_events / wall2,
                        "latency": latency_summary(res2), "rebuilds": srv2.rebuilds,
                        "rebuild_s": srv2.rebuild_s}
    out["same_results"] = all(a.digest == b.digest for a, b in zip(res, res2))
    if args.serving_plain:
        sub = reqs[: args.serving_plain]
        ev, t1 = 0, time.perf_counter()
        for q in sub:
            for spec in q.replica_specs():
                t = Tissue(spec)
                t.step(q.dt, q.n_steps)
                ev += int(t.total_events().sum())
                t.close()
        torch.cuda.synchronize()
        el = time.perf_counter() - t1
        sub_ev = sum(r.events for r in res[: args.serving_plain])
        out["plain"] = {"requests": len(sub), "plain_events_per_s": ev / el,
                        "note": "the first requests served one tissue at a time, in arrival "
                                "order, with no batching",
                        "events_match": ev == sub_ev}
        out["served_vs_plain"] = sat["served_events_per_s"] / (ev / el)
    return out


# ---------------------------------------------------------------------------
# Suite: every configuration, GPU and oracle, for the results table
# ---------------------------------------------------------------------------

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
    burn = int(round(args.large_burn_in / lg.dt))
    row("large", lg.tissue, lg.dt, max(args.large_steps, 1), burn, cpu_steps=0, cpu_cells=128)
    out["large"]["cpu_sample"] = (f"chi of 128 cells at step {burn} (one core); all cores "
                                  "not run")
    return out



# ---------------------------------------------------------------------------
# Profiling case for the instructions-per-event table
# ---------------------------------------------------------------------------

def profile_subset(runs, per_class: int = 16, target_cells: int = 1024):
    """A smaller batch with every cell-size class of the full one: per cell
    size the `per_class` member tissues nearest target_cells cells (about
    260 MB of state, more than L2, so DRAM figures stay meaningful)."""
    return oracle_sample(runs, per_class=per_class, target_cells=target_cells)


def run_profile(args) -> dict:
    """Steps one workload as the benchmark does (burn-in, warm-up, then
    --steps steps) and reports each class's chi launch key and chi events
    per step, so that ncu's per-launch counters of the same run give
    instructions and DRAM bytes per event.  Workloads: "batch" (a subset of
    the batch with every cell-size class), "medium" and "large".  Under ncu,
    skip the chi launches of the burn-in and warm-up (launches_before in the
    output) and capture launches_per_step x steps of them."""
    import torch

    from paper_1806_10889_gb300.batching import Batch
    from paper_1806_10889_gb300.tissue import Tissue

    if args.profile_chi == "batch":
        runs = batch_runs()
        idx = profile_subset(runs)
        sub = [runs[i] for i in idx]
        burn_time = args.batch_burn_in
    else:
        run = W.medium(args.dt) if args.profile_chi == "medium" else W.large()
        idx, sub = [0], [run]
        burn_time = args.burn_in if args.profile_chi == "medium" else args.large_burn_in
    dt = sub[0].dt
    members = [Tissue(r.tissue) for r in sub]
    torch.cuda.synchronize()
    if args.profile_chi == "batch":
        bt = Batch(members)
        # classes one after another, so that the profiler's launch order is
        # the class order (instructions per event do not depend on overlap)
        bt.set_overlap(False)
        for part in args.profile_class:  # V:lanes:warps:layout, e.g. an autotuner pick
            V, lanes, wpb, layout = (int(x) for x in part.split(":"))
            bt.set_class_launch(V, lanes, wpb, layout)
        classes = bt.classes()
        step = bt.step

        def sync():
            bt.sync()
    else:
        g = members[0]
        la = g.launch_config()
        classes = [{"V": g.spec.V, "lanes_per_cell": la[1], "warps_per_block": la[2],
                    "smem_layout": la[4], "cells": g.spec.cells}]
        step, sync = g.step, g.sync
    keys = [chi_kernel_key(c["V"], c["lanes_per_cell"], c["smem_layout"]) for c in classes]
    per_step = sum(1 + int(k.endswith("u16")) for k in keys)
    burn = int(round(burn_time / dt))
    step(dt, burn + args.warmup)
    sync()
    steps = []
    for _ in range(args.steps):
        e0 = _events(members)
        step(dt, 1)
        sync()
        d = _events(members) - e0
        steps.append([int(sum(d[j, 0] for j, r in enumerate(sub) if r.tissue.V == c["V"]))
                      for c in classes])
    if args.profile_chi == "batch":
        bt.close()
    for m in members:
        m.close()
    return {"workload": args.profile_chi, "tissues": idx,
            "cells": sum(r.tissue.cells for r in sub),
            "state_bytes": sum(r.tissue.state_ints * 4 for r in sub),
            "classes": [dict(c, key=k) for c, k in zip(classes, keys)],
            "chi_launches_per_step": per_step,
            "launches_before": per_step * (burn + args.warmup),
            "chi_events_per_step_by_class": steps, "sources": chi_sources_sha()}


# ---------------------------------------------------------------------------
# Bound on a wavefront across steps
# ---------------------------------------------------------------------------

def wavefront_bound(events: np.ndarray, width: int, height: int) -> dict:
    """How much a barrier-free wavefront across steps could shorten K steps of
    one tissue, in events along the longest chain (a cell's chi events are one
    dependent chain, so its time is proportional to them).

    events[k, c]: chi events of cell c in step k.  With a barrier per step,
    K steps take sum_k max_c e[k, c].  Without one, cell c may start step k
    once the faces it touches are done for step k-1; the two face phases make
    that the 3x3 neighbourhood of c, so the finish of (c, k) is
    F[c, k] = max over that neighbourhood of F[., k-1] + e[k, c], and the
    wavefront takes max_c F[c, K-1].  Both ignore the (short) face phases."""
    e = np.asarray(events, dtype=np.float64).reshape(-1, height, width)
    barrier = float(e.max(axis=(1, 2)).sum())
    chain = float(e.sum(axis=0).max())
    F = np.zeros((height, width))
    for k in range(e.shape[0]):
        p = np.pad(F, 1)
        nb = np.max(np.stack([p[1 + dy:1 + dy + height, 1 + dx:1 + dx + width]
                              for dy in (-1, 0, 1) for dx in (-1, 0, 1)]), axis=0)
        F = nb + e[k]
    wave = float(F.max())
    return {"steps": int(e.shape[0]), "barrier_events": barrier, "wavefront_events": wave,
            "slowest_cell_events": chain, "gain_bound": 1.0 - wave / barrier,
            "mean_over_max_per_step": float((e.mean(axis=(1, 2)) / e.max(axis=(1, 2))).mean())}


def run_wavefront(args) -> dict:
    """The medium tissue after its burn-in, --steps steps with every cell's
    chi events read back after each step, and the bound above."""
    from paper_1806_10889_gb300.tissue import Tissue

    spec = W.medium(args.dt).tissue
    g = Tissue(spec)
    g.step(args.dt, int(round(args.burn_in / args.dt)))
    ev = []
    for _ in range(args.steps):
        g.step(args.dt, 1)
        ev.append(g.read_stats()[0][0].astype(np.int64))
    g.close()
    out = wavefront_bound(np.array(ev), spec.width, spec.height)
    out["workload"] = (f"medium tissue {spec.width}x{spec.height} cells of {spec.n}x{spec.n} "
                       f"voxels, dt {args.dt}, after {args.burn_in} time units")
    return out


# ---------------------------------------------------------------------------
# Driver
# ---------------------------------------------------------------------------

def run_ours(args, rank, world, local_rank):
    import torch

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    out = batch_headline(args, rank, world, dist)
    if rank == 0 and world == 1:
        if not args.no_medium:
            out["medium"] = medium_leg(args)
        if not args.no_promoter:
            out["promoter"] = promoter_leg(args)
            out["mixed_fidelity"] = promoter_leg(args, W.mixed_fidelity())
        if args.large_steps:
            out["large"] = large_leg(args)
        if args.serving:
            out["serving"] = serving_leg(args)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return out if rank == 0 else None


def run_reference(args, rank, world):
    """The oracle, as it stands, on the host cores: each step is the same
    splitting step of the sampled member tissues of the batch (one per cell
    size), after the same simulated burn-in as the GPU arm."""
    if rank != 0:
        return None
    import oracle as O
    runs = W.batch()
    dt = runs[0].dt
    sample = oracle_sample(runs, per_class=args.oracle_per_class)
    tissues = []
    for i in sample:
        _, d, m = _orc(runs[i].tissue)
        tissues.append((d, m, O.init_counts(d)))
    threads = O.max_threads()
    burn = int(round(args.batch_burn_in / dt))
    for k in range(burn + args.warmup):
        for d, m, c in tissues:
            O.step(d, m, c, k, 1, dt, n_threads=threads)
    total, t0 = 0, time.perf_counter()
    for k in range(burn + args.warmup, burn + args.warmup + args.steps):
        for d, m, c in tissues:
            ne, _ = O.step(d, m, c, k, 1, dt, n_threads=threads)
            total += int(ne.sum())
    el = time.perf_counter() - t0
    value = total / el
    cells = sum(runs[i].tissue.cells for i in sample)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64+f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "256 uneven tissues (side U{2..64} cells, cells of 8x8, 16x16 "
                                   "or 32x32 voxels, kD U[5,20]), Notch-Delta model; the oracle "
                                   "steps a sample of them",
                       "dt": dt, "burn_in_time": args.batch_burn_in, "sample_tissues": sample,
                       "sample_cells": cells},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"member tissues {sample} of the batch ({cells} cells), "
                                       f"whole splitting steps after {burn} burn-in steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--batch-burn-in", type=float, default=5.0,
                    help="untimed simulated time of the batch before its timed steps")
    ap.add_argument("--autotune", type=int, default=1)
    ap.add_argument("--class-overlap", choices=["auto", "on", "off"], default="auto",
                    help="the batch's cell-size classes overlapped or one after another "
                         "(off: their live times separate); auto picks the faster from "
                         "4 steps of the batch before the warm-up")
    ap.add_argument("--tune-clones", type=int, default=8,
                    help="member tissues per cell-size class the autotuner clones")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--plain-steps", type=int, default=2,
                    help="steps of the plain per-tissue comparison (0: skip)")
    ap.add_argument("--oracle-per-class", type=int, default=1)
    ap.add_argument("--dt", type=float, default=0.1, choices=[0.01, 0.1, 1.0],
                    help="medium tissue: splitting step")
    ap.add_argument("--burn-in", type=float, default=20.0,
                    help="medium tissue: untimed simulated time first")
    ap.add_argument("--chi-wpb", type=int, default=0)
    ap.add_argument("--kernel", choices=["default", "persistent"], default="default")
    ap.add_argument("--lanes", type=int, choices=[8, 16, 32], default=16)
    ap.add_argument("--layout", type=int, choices=[0, 1], default=0,
                    help="persistent kernel: 0 prefix arrays, 1 recompute")
    ap.add_argument("--side", type=int, default=0, help="profiling only: medium tissue side")
    ap.add_argument("--n", type=int, default=0, help="profiling only: voxels per cell side")
    ap.add_argument("--no-medium", action="store_true")
    ap.add_argument("--no-promoter", action="store_true",
                    help="skip the promoter-model and mixed-fidelity legs")
    ap.add_argument("--large-steps", type=int, default=3, help="large tissue timed steps (0: skip)")
    ap.add_argument("--large-burn-in", type=float, default=2.0)
    ap.add_argument("--serving", type=int, default=50,
                    help="serve the first K requests of the serving workload (0: skip)")
    ap.add_argument("--serving-replicas", type=int, default=2,
                    help="cap on the replicas of each served request")
    ap.add_argument("--serving-load", type=float, default=0.7,
                    help="sustained arrival rate as a fraction of the saturation rate")
    ap.add_argument("--serving-plain", type=int, default=4,
                    help="requests served one tissue at a time for the plain rate (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-chi", choices=["batch", "medium", "large"], default=None,
                    help="profiling case: step this workload, printing each chi launch class's "
                         "events per step for ncu's per-launch counters")
    ap.add_argument("--profile-class", action="append", default=[],
                    help="with --profile-chi batch: V:lanes:warps:layout launch of one class")
    ap.add_argument("--wavefront", action="store_true",
                    help="bound the gain of a barrier-free wavefront across --steps steps of "
                         "the medium tissue (per-cell events read back every step)")
    ap.add_argument("--suite", action="store_true",
                    help="measure every single-tissue configuration (GPU and oracle) and print "
                         "one JSON object instead of the benchmark line (several minutes)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    rank, world, local_rank = _env_rank()
    if args.suite:
        print(json.dumps(run_suite(args)))
        return
    if args.profile_chi:
        print(json.dumps(run_profile(args)))
        return
    if args.wavefront:
        print(json.dumps(run_wavefront(args)))
        return
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world, local_rank)
    if rank == 0 and out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
