"""Batched stepping of many tissues (binding of the tissue_batch_* C ABI).

A Batch groups existing Tissue objects; one batch step advances all of them
with one persistent chi launch per cell-size class (cells pulled from a work
list, largest cells first) and one launch per face phase, captured in a CUDA
graph.  Trajectories are bit-identical to stepping each tissue alone.
"""
from __future__ import annotations

import ctypes as C

from .tissue import Tissue, TissueError, _check, lib


class Batch:
    def __init__(self, members: list[Tissue], stream=None):
        import torch
        if not members:
            raise ValueError("a batch needs at least one tissue")
        self.members = list(members)
        # a dedicated stream: the legacy default stream cannot be graph-captured
        self.stream = stream if stream is not None else torch.cuda.Stream()
        arr = (C.c_void_p * len(members))(*[m.handle.value for m in members])
        self._h = C.c_void_p()
        self.timing = False  # tissue_batch_set_timing's state
        self.overlap = True  # tissue_batch_set_overlap's state
        _check(lib().tissue_batch_create(arr, len(members), C.c_void_p(self.stream.cuda_stream),
                                         C.byref(self._h)), "tissue_batch_create")

    def set_class_launch(self, V: int, lanes_per_cell: int, warps_per_block: int,
                         smem_layout: int = 0):
        _check(lib().tissue_batch_set_class_launch(self._h, V, lanes_per_cell, warps_per_block,
                                                   smem_layout),
               "tissue_batch_set_class_launch")

    def set_splitting(self, scheme: int):
        _check(lib().tissue_batch_set_splitting(self._h, int(scheme)),
               "tissue_batch_set_splitting")

    def set_schedule(self, steps_per_graph: int):
        _check(lib().tissue_batch_set_schedule(self._h, int(steps_per_graph)),
               "tissue_batch_set_schedule")

    def step(self, dt: float, n_steps: int = 1):
        _check(lib().tissue_batch_step(self._h, float(dt), int(n_steps)), "tissue_batch_step")

    def sync(self):
        """Wait for the batch's work; required before reading members."""
        _check(lib().tissue_batch_sync(self._h), "tissue_batch_sync")

    def info(self):
        a, b, c = C.c_uint32(), C.c_uint32(), C.c_uint64()
        _check(lib().tissue_batch_info(self._h, C.byref(a), C.byref(b), C.byref(c)),
               "tissue_batch_info")
        return int(a.value), int(b.value), int(c.value)

    def write_counts(self, host_tensors, step_index=None) -> None:
        """Every member's state from host memory (torch int32 CPU tensors,
        pinned for asynchronous copies), in member order; step_index: one int
        for all members, a list, or None to keep each member's index."""
        n = len(self.members)
        if len(host_tensors) != n:
            raise ValueError("one host array per member")
        for t, m in zip(host_tensors, self.members):
            if t.numel() != m.spec.state_ints or t.dtype != __import__("torch").int32:
                raise ValueError("each host array must be the member's int32 state")
        ptrs = (C.c_void_p * n)(*[t.data_ptr() for t in host_tensors])
        steps = None
        if step_index is not None:
            vals = [int(step_index)] * n if isinstance(step_index, int) else list(step_index)
            steps = (C.c_uint32 * n)(*vals)
        _check(lib().tissue_batch_write_counts(self._h, ptrs, steps), "tissue_batch_write_counts")

    def read_counts(self, host_tensors) -> None:
        """Every member's state into host memory (torch int32 CPU tensors)."""
        n = len(self.members)
        if len(host_tensors) != n:
            raise ValueError("one host array per member")
        for t, m in zip(host_tensors, self.members):
            if t.numel() != m.spec.state_ints or t.dtype != __import__("torch").int32:
                raise ValueError("each host array must be the member's int32 state")
        ptrs = (C.c_void_p * n)(*[t.data_ptr() for t in host_tensors])
        _check(lib().tissue_batch_read_counts(self._h, ptrs), "tissue_batch_read_counts")

    def classes(self) -> list[dict]:
        """Cell-size classes, largest cells first: V, launch shape, cells."""
        n = self.info()[1]
        out = []
        for i in range(n):
            v = [C.c_uint32() for _ in range(5)]
            _check(lib().tissue_batch_class_info(self._h, i, *[C.byref(x) for x in v]),
                   "tissue_batch_class_info")
            V, lanes, wpb, layout, cells = (int(x.value) for x in v)
            out.append({"V": V, "lanes_per_cell": lanes, "warps_per_block": wpb,
                        "smem_layout": layout, "cells": cells})
        return out

    def set_timing(self, on: bool) -> None:
        """Record device times of each following step (a measurement aid)."""
        _check(lib().tissue_batch_set_timing(self._h, 1 if on else 0), "tissue_batch_set_timing")
        self.timing = bool(on)

    def read_timing(self):
        """(step ms, chi phase ms, well-mixed chi ms, [chi ms per class]) of
        the last timed step (a class's time runs from when its launches became
        ready; overlapped classes are all ready at the chi phase's start)."""
        n = self.info()[1]
        st, chi, wm = C.c_double(), C.c_double(), C.c_double()
        cls = (C.c_double * max(n, 1))()
        _check(lib().tissue_batch_read_timing(self._h, C.byref(st), C.byref(chi), C.byref(wm),
                                              cls, n), "tissue_batch_read_timing")
        return st.value, chi.value, wm.value, [cls[i] for i in range(n)]

    def set_overlap(self, on: bool) -> None:
        """Overlapped cell-size classes (the default) or one after another."""
        _check(lib().tissue_batch_set_overlap(self._h, 1 if on else 0), "tissue_batch_set_overlap")
        self.overlap = bool(on)

    def total_events(self) -> int:
        return int(sum(int(m.total_events().sum()) for m in self.members))

    def close(self):
        if self._h:
            lib().tissue_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["Batch", "TissueError"]
