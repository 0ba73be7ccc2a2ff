"""Serving: ensemble simulation requests admitted by device-memory budget and
advanced together by continuous batching.

A request asks for ``replicas`` tissues of ``side x side`` cells (n x n
voxels each) run for ``n_steps`` splitting steps of length dt.  Replica r of
request q is the tissue (seed = q, tissue_id = r), so its trajectory is
fixed by the request alone: the same whether it runs alone or among others,
in whichever slot and batch it lands.

The server loop:
  1. admit arrived requests in arrival order while the bytes they need
     (state + library scratch of every replica) fit the budget;
  2. choose the round's requests (the scheduling policy, below) and rebuild
     the batch when its membership changed;
  3. advance the chosen requests' tissues by one chunk of steps with one
     batch step (one persistent launch per cell-size class and step);
  4. retire requests whose tissues reached their step count: read the
     result back, free the memory, record the latency.
Requests that arrive while others run join at the next chunk boundary, so
their work overlaps on the device with the work already in flight.

Policies: "srpt" (default) takes the active requests in order of least
remaining work (cells x steps left) until the round holds at least
`fill_cells` cells, enough to keep the device busy, and leaves the rest
waiting; small requests then finish early instead of paying every step of
the large ones.  "lockstep" advances every active request every round.
The policy decides only when a tissue steps, never what a step computes.
"""
from __future__ import annotations

import hashlib
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from .batching import Batch
from .tissue import Tissue, scratch_bytes, state_bytes
from .workloads import Request


@dataclass
class Result:
    index: int
    arrival_s: float
    admitted_s: float = float("nan")
    done_s: float = float("nan")
    events: int = 0
    cells: int = 0
    digest: str = ""
    counts: list = field(default_factory=list)
    rejected: bool = False
    cancelled: bool = False

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


@dataclass
class _Active:
    req: Request
    result: Result
    tissues: list
    steps_done: int = 0
    nbytes: int = 0


def request_bytes(req: Request) -> int:
    """Device bytes one request holds while active (all replicas)."""
    spec = req.replica_specs()[0]
    return req.replicas * (state_bytes(spec) + scratch_bytes(spec))


class Server:
    """Continuous-batching server over one device.

    budget_bytes: device memory the server may hold for tissue state and
    scratch; chunk_steps: steps per batch call between admission points;
    tuned: optional autotuner result (``autotune.tune_batch``) applied to
    every batch; keep_counts: return each replica's final counts.
    """

    def __init__(self, budget_bytes: int, chunk_steps: int = 10, tuned: dict | None = None,
                 keep_counts: bool = False, clock=time.perf_counter, policy: str = "srpt",
                 fill_cells: int = 16384):
        if policy not in ("srpt", "lockstep"):
            raise ValueError(f"unknown policy {policy!r}")
        self.policy = policy
        self.fill_cells = int(fill_cells)
        self.budget = int(budget_bytes)
        self.chunk = int(chunk_steps)
        self.tuned = tuned
        self.keep_counts = keep_counts
        self.clock = clock
        self.used = 0
        self.peak_used = 0
        self.device_events = 0
        # batch rebuilds on membership changes and the host time they took
        # (the batch's tables; its graph is captured on its first step)
        self.rebuilds = 0
        self.rebuild_s = 0.0
        self._cancel: set = set()
        self._cancel_lock = threading.Lock()

    def cancel(self, index: int) -> None:
        """Cancel request `index` (safe from any thread): a pending request
        is dropped; an active one is stopped at the next chunk boundary and
        its memory freed.  Its result is marked cancelled and has no digest."""
        with self._cancel_lock:
            self._cancel.add(int(index))

    def _take_cancelled(self) -> set:
        with self._cancel_lock:
            return set(self._cancel)

    def run(self, requests: list[Request], time_scale: float = 1.0,
            on_round=None) -> list[Result]:
        """Serve `requests`; on_round(server, indices), if given, is called
        after every round with the indices of the requests it advanced."""
        import torch
        if len({r.dt for r in requests}) > 1:
            raise ValueError("one server run serves requests of a single dt")
        pending = sorted(requests, key=lambda r: r.arrival_s)
        results = {r.index: Result(r.index, r.arrival_s * time_scale) for r in pending}
        active: list[_Active] = []
        batch = None
        members_key = None
        t0 = self.clock()
        while pending or active:
            now = self.clock() - t0
            # 0. cancellations: drop pending requests, stop active ones
            cancelled = self._take_cancelled()
            if cancelled:
                for r in [r for r in pending if r.index in cancelled]:
                    pending.remove(r)
                    results[r.index].cancelled = True
                keep = []
                for a in active:
                    if a.req.index not in cancelled:
                        keep.append(a)
                        continue
                    if batch is not None:
                        batch.close()
                        batch, members_key = None, None
                    for t in a.tissues:
                        t.close()
                    self.used -= a.nbytes
                    a.result.cancelled = True
                    a.result.done_s = now
                active = keep
            # 1. admission, arrival order
            while pending and pending[0].arrival_s * time_scale <= now:
                req = pending[0]
                need = request_bytes(req)
                if need > self.budget:
                    results[req.index].rejected = True
                    pending.pop(0)
                    continue
                if self.used + need > self.budget:
                    break
                pending.pop(0)
                tissues = [Tissue(s) for s in req.replica_specs()]
                res = results[req.index]
                res.admitted_s = now
                res.cells = sum(s.cells for s in req.replica_specs())
                active.append(_Active(req, res, tissues, 0, need))
                self.used += need
            if not active:
                if pending:
                    wait = pending[0].arrival_s * time_scale - (self.clock() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.05))
                continue
            # 2. the round's requests; the batch follows them
            chosen = self._choose(active)
            key = tuple(id(t) for a in chosen for t in a.tissues)
            rebuilt = key != members_key
            if rebuilt:
                tb = self.clock()
                if batch is not None:
                    batch.close()
                batch = Batch([t for a in chosen for t in a.tissues])
                if self.tuned:
                    from .autotune import apply_batch
                    apply_batch(batch, self.tuned)
                members_key = key
                self.rebuilds += 1
                self.rebuild_s += self.clock() - tb
            # 3. one chunk, bounded by the chosen request that finishes first
            dt = chosen[0].req.dt
            k = min(self.chunk, min(a.req.n_steps - a.steps_done for a in chosen))
            if rebuilt:
                # the first step of a new batch captures its graph: count the
                # host time of that capture as rebuild time too
                tb = self.clock()
                batch.step(dt, 1)
                self.rebuild_s += self.clock() - tb
                if k > 1:
                    batch.step(dt, k - 1)
            else:
                batch.step(dt, k)
            batch.sync()
            for a in chosen:
                a.steps_done += k
            self.peak_used = max(self.peak_used, self.used)
            if on_round is not None:
                on_round(self, [a.req.index for a in chosen])
            # 4. retire finished requests
            now = self.clock() - t0
            still = []
            for a in active:
                if a.steps_done < a.req.n_steps:
                    still.append(a)
                    continue
                h = hashlib.sha256()
                ev = 0
                for t in a.tissues:
                    c = t.read_counts()
                    h.update(c.tobytes())
                    ev += int(t.total_events().sum())
                    if self.keep_counts:
                        a.result.counts.append(c)
                a.result.digest = h.hexdigest()
                a.result.events = ev
                a.result.done_s = now
                self.device_events += ev
                if batch is not None:
                    batch.close()
                    batch, members_key = None, None
                for t in a.tissues:
                    t.close()
                self.used -= a.nbytes
            active = still
        if batch is not None:
            batch.close()
        torch.cuda.synchronize()
        return [results[r.index] for r in sorted(requests, key=lambda r: r.index)]

    def _choose(self, active: list) -> list:
        if self.policy == "lockstep":
            return active
        order = sorted(active, key=lambda a: (a.result.cells * (a.req.n_steps - a.steps_done),
                                              a.req.index))
        chosen, cells = [], 0
        for a in order:
            chosen.append(a)
            cells += a.result.cells
            if cells >= self.fill_cells:
                break
        return chosen


def latency_summary(results: list[Result]) -> dict:
    lat = np.array([r.latency_s for r in results if not (r.rejected or r.cancelled)])
    if lat.size == 0:
        return {"p50_s": None, "p99_s": None, "served": 0}
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "served": int(lat.size),
            "rejected": int(sum(r.rejected for r in results)),
            "cancelled": int(sum(r.cancelled for r in results))}
