"""Autotuner of the chi launch shape, the cells-per-warp split and the
split-step schedule.

Every candidate runs the same steps from the same state on a clone of the
work and must end with the same counts and statistics bit for bit (the
arithmetic is exact, so a variant that differs is a bug, not noise); the
fastest is kept.  Results are cached per GPU, cell size, tissue size class
and dt in ``_build/autotune.json`` beside the compiled library.
"""
from __future__ import annotations

import json
import math
import os
import threading

import numpy as np

from .tissue import (KERNEL_PERSISTENT, KERNEL_WARP, LAYOUT_PREFIX, LAYOUT_RECOMPUTE, Tissue,
                     TissueError)
from .workloads import TissueSpec

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
_lock = threading.Lock()


class VariantMismatch(RuntimeError):
    """Two launch variants produced different trajectories."""


def _recompute_fits(V: int, lanes: int) -> bool:
    """The counts-only layout takes cells of V voxels with this many lanes:
    a block fits the lanes (V <= lanes^2), or the lanes cover up to four
    voxels each (16 lanes and V <= 1024, 8 lanes and V <= 256; Notch-Delta
    launches, others run the prefix layout)."""
    return V <= lanes * lanes or (lanes == 16 and V <= 1024) or (lanes == 8 and V <= 256)


def tissue_candidates(V: int) -> list[tuple]:
    """(kernel, lanes per cell, warps per block, blocks, shared-memory layout)
    candidates for cells of V voxels."""
    c = [(KERNEL_WARP, 32, w, 0, LAYOUT_PREFIX) for w in (2, 4, 8)]
    for lanes in (8, 16, 32):
        c += [(KERNEL_PERSISTENT, lanes, w, 0, LAYOUT_PREFIX) for w in (1, 2, 4)]
        if _recompute_fits(V, lanes):
            c += [(KERNEL_PERSISTENT, lanes, w, 0, LAYOUT_RECOMPUTE) for w in (1, 2, 4)]
    return c


def batch_class_candidates(V: int) -> list[tuple]:
    """(lanes per cell, warps per block, layout) candidates for one cell-size class."""
    c = []
    for lanes in (8, 16, 32):
        c += [(lanes, w, LAYOUT_PREFIX) for w in (1, 2, 4)]
        if _recompute_fits(V, lanes):
            c += [(lanes, w, LAYOUT_RECOMPUTE) for w in (1, 2, 4)]
    return c


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def _load() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, value) -> None:
    with _lock:
        data = _load()
        data[key] = value
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, CACHE)


def _size_class(cells: int) -> int:
    return int(2 ** round(math.log2(max(cells, 1))))


def _time_steps(run, n_steps: int, stream=None) -> float:
    """Device milliseconds of run(n_steps), timed on the stream it uses."""
    import torch
    stream = stream if stream is not None else torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    run(n_steps)
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b)


def tune_tissue(spec: TissueSpec, dt: float, state: np.ndarray | None = None,
                step_index: int = 0, steps: int = 2, candidates: list[tuple] | None = None,
                use_cache: bool = True, on_candidate=None) -> dict:
    """Pick the fastest chi launch for this tissue; returns
    {"config": (kernel, lanes, warps, blocks, layout), "ms": {str(config): ms}}.

    on_candidate(config, tissue), if given, runs after each candidate's clone
    is set up and before it steps (a hook for tests of the bit-identity
    check)."""
    key = f"tissue|{_gpu_name()}|V={spec.V}|cells~{_size_class(spec.cells)}|dt={dt}"
    if use_cache and candidates is None:
        hit = _load().get(key)
        if hit:
            return {"config": tuple(hit["config"]), "ms": hit["ms"], "cached": True}
    cands = candidates or tissue_candidates(spec.V)
    times, ref, tried = {}, None, []
    for cfg in cands:
        t = Tissue(spec)
        if state is not None:
            t.write_counts(state, step_index)
        try:
            t.set_launch_config(*cfg)
        except TissueError:  # the shape does not fit these cells (shared memory)
            t.close()
            continue
        tried.append(cfg)
        if on_candidate is not None:
            on_candidate(cfg, t)
        t.step(dt, 1)  # warm (first launch of a variant configures it)
        t.sync()
        times[str(cfg)] = _time_steps(lambda n: t.step(dt, n), steps)
        out = (t.read_counts(), *t.read_stats())
        if ref is None:
            ref = out
        elif not (np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])
                  and np.array_equal(out[2].view(np.uint64), ref[2].view(np.uint64))):
            t.close()
            raise VariantMismatch(f"launch {cfg} changed the trajectory of {spec}")
        t.close()
    best = min(tried, key=lambda c: times[str(c)])
    result = {"config": list(best), "ms": times}
    _store(key, result)
    return {"config": tuple(best), "ms": times, "cached": False}


def tune_batch(members: list[Tissue], dt: float, steps: int = 1, max_clones: int = 48,
               schedules=(1, 4), use_cache: bool = True, on_candidate=None) -> dict:
    """Pick (lanes per cell, warps per block, layout) per cell-size class and the
    steps-per-graph schedule for a batch of these tissues.

    Each class is tuned on clones of up to ``max_clones`` of its members
    (their current state and step index), so the members themselves do not
    move.  Returns {"classes": {V: (lanes, warps, layout)}, "steps_per_graph": k}.
    on_candidate((V, lanes, warps, layout), clones), if given, runs after each
    class candidate's clones are set up and before they step (a hook for
    tests of the bit-identity check).
    """
    from .batching import Batch

    by_v: dict[int, list[Tissue]] = {}
    for m in members:
        by_v.setdefault(m.spec.V, []).append(m)
    key = (f"batch|{_gpu_name()}|dt={dt}|" +
           ",".join(f"{V}:{_size_class(sum(m.spec.cells for m in ms))}"
                    for V, ms in sorted(by_v.items())))
    if use_cache:
        hit = _load().get(key)
        if hit:
            return {"classes": {int(k): tuple(v) for k, v in hit["classes"].items()},
                    "steps_per_graph": hit["steps_per_graph"], "cached": True}

    def clones_of(ms):
        out = []
        for m in ms[:max_clones]:
            c = Tissue(m.spec)
            c.write_counts(m.read_counts(), m.get_step())
            out.append(c)
        return out

    chosen, timings = {}, {}
    for V, ms in sorted(by_v.items()):
        ref, tried = None, []
        for lanes, wpb, layout in batch_class_candidates(V):
            clones = clones_of(ms)
            b = Batch(clones)
            try:
                b.set_class_launch(V, lanes, wpb, layout)
            except TissueError:  # does not fit shared memory for this V
                b.close()
                for c in clones:
                    c.close()
                continue
            tried.append((lanes, wpb, layout))
            if on_candidate is not None:
                on_candidate((V, lanes, wpb, layout), clones)
            b.step(dt, 1)
            b.sync()
            ms_ = _time_steps(lambda n: b.step(dt, n), steps, b.stream)
            b.sync()
            timings[f"{V}:{lanes}x{wpb}/{layout}"] = ms_
            out = [c.read_counts() for c in clones]
            if ref is None:
                ref = out
            elif not all(np.array_equal(x, y) for x, y in zip(out, ref)):
                raise VariantMismatch(f"batch launch {lanes}x{wpb}/{layout} changed results (V={V})")
            b.close()
            for c in clones:
                c.close()
        chosen[V] = min(tried, key=lambda c: timings[f"{V}:{c[0]}x{c[1]}/{c[2]}"])
    # schedule: tune on a clone of the whole (bounded) batch with the chosen classes
    best_k, best_ms = 1, None
    for k in schedules:
        clones = clones_of([m for ms in by_v.values() for m in ms][:max_clones])
        b = Batch(clones)
        for V, (lanes, wpb, layout) in chosen.items():
            if any(c.spec.V == V for c in clones):
                b.set_class_launch(V, lanes, wpb, layout)
        b.set_schedule(k)
        b.step(dt, k)
        b.sync()
        ms_ = _time_steps(lambda n: b.step(dt, n), k * max(1, steps), b.stream)
        timings[f"steps_per_graph={k}"] = ms_
        if best_ms is None or ms_ < best_ms:
            best_k, best_ms = k, ms_
        b.close()
        for c in clones:
            c.close()
    _store(key, {"classes": {str(V): list(c) for V, c in chosen.items()},
                 "steps_per_graph": best_k, "ms": timings})
    return {"classes": chosen, "steps_per_graph": best_k, "ms": timings, "cached": False}


def tune_overlap(batch, dt: float, rounds: int = 1) -> dict:
    """Overlapped or one-after-another cell-size classes for this batch, chosen
    from its own steps: whether overlapping pays depends on how the classes'
    launch shapes share an SM (measured on the 256-tissue batch: -1.9% per
    step with the default shapes, +0.9% with the shapes tune_batch picks).

    Advances the batch by 4 x rounds steps, in the order overlapped,
    sequential, sequential, overlapped (so that the drift of the step time as
    the state evolves cancels), each timed inside its captured graph; leaves
    the faster mode set (overlapped on a tie).  Results never depend on the
    mode.  Returns {"overlap": bool, "ms": {"overlapped": ms, "sequential": ms}}.
    """
    if len(batch.classes()) < 2:
        return {"overlap": batch.overlap, "ms": {}}
    timing = batch.timing
    batch.set_timing(True)
    total = {True: 0.0, False: 0.0}
    for on in (True, False, False, True) * max(1, rounds):
        batch.set_overlap(on)
        batch.step(dt, 1)
        total[on] += batch.read_timing()[0]
    best = total[True] <= total[False]
    batch.set_overlap(best)
    batch.set_timing(timing)
    n = 2 * max(1, rounds)
    return {"overlap": best, "ms": {"overlapped": total[True] / n, "sequential": total[False] / n}}


def apply_batch(batch, tuned: dict) -> None:
    from .tissue import TissueError
    for V, cfg in tuned["classes"].items():
        try:
            batch.set_class_launch(V, *cfg)
        except TissueError:
            pass  # the class is not present in this batch
    batch.set_schedule(tuned["steps_per_graph"])
