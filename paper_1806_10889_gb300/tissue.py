"""Thin ctypes binding of libtissue (include/tissue.h).

Argument marshalling only: every step of the method runs in the CUDA
kernels behind the C ABI.  PyTorch provides the device memory (the state
buffer is a torch tensor the caller owns) and the stream (the current torch
stream at creation).  There is no CPU fallback: without the compiled library
or a CUDA device every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from .workloads import TissueSpec

_lock = threading.Lock()
_lib = None

# Launch shape of the chi kernel used by the benchmark and its parity test.
DEFAULT_CHI_WPB = 4

OK, E_ARG, E_NOMEM, E_NOMODEL, E_OVERFLOW, E_CUDA, E_TIMEOUT, E_BUDGET = 0, -1, -2, -3, -4, -5, -6, -7
E_STATE = -9
E_BOUNDS = -10


class TissueError(RuntimeError):
    def __init__(self, code: int, what: str):
        msg = lib().tissue_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})")
        self.code = code


class Desc(C.Structure):
    _fields_ = [("width", C.c_uint32), ("height", C.c_uint32), ("n", C.c_uint32),
                ("tissue_id", C.c_uint32), ("seed", C.c_uint64),
                ("init_lambda", C.c_double * 3)]


MODEL_FIELDS = ["kD", "K", "kN", "gD", "gN", "gR", "hopD", "hopN", "hopR", "k_in", "k_off",
                "k_bind"]


class Model(C.Structure):
    _fields_ = [(f, C.c_double) for f in MODEL_FIELDS]


PROMOTER_FIELDS = ["tD", "ka", "kd", "kN", "d", "hop"]


class PromoterModel(C.Structure):
    _fields_ = [(f, C.c_double) for f in PROMOTER_FIELDS]


# tissue_event of the C ABI (the oracle's trace record has the same layout)
EVENT_DTYPE = np.dtype([("step", "<u4"), ("kind", "<u4"), ("unit", "<u4"), ("e", "<u4"),
                        ("t", "<f8"), ("site", "<u4"), ("channel", "<u4")])

KERNEL_WARP, KERNEL_PERSISTENT = 0, 1
LAYOUT_PREFIX, LAYOUT_RECOMPUTE = 0, 1
SPLIT_LIE, SPLIT_STRANG = 0, 1


class Launch(C.Structure):
    _fields_ = [("kernel", C.c_uint32), ("lanes_per_cell", C.c_uint32),
                ("warps_per_block", C.c_uint32), ("blocks", C.c_uint32),
                ("smem_layout", C.c_uint32)]


# Every exported symbol of include/tissue.h with (restype, argtypes).
_P = C.POINTER
SIGNATURES = {
    "tissue_state_bytes": (C.c_size_t, [_P(Desc)]),
    "tissue_scratch_bytes": (C.c_size_t, [_P(Desc)]),
    "tissue_create": (C.c_int, [_P(Desc), C.c_void_p, C.c_size_t, C.c_void_p, _P(C.c_void_p)]),
    "tissue_set_model": (C.c_int, [C.c_void_p, _P(Model)]),
    "tissue_set_promoter_model": (C.c_int, [C.c_void_p, _P(PromoterModel)]),
    "tissue_set_cell_fidelity": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "tissue_trace_begin": (C.c_int, [C.c_void_p, C.c_size_t]),
    "tissue_trace_read": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, _P(C.c_size_t)]),
    "tissue_trace_end": (C.c_int, [C.c_void_p]),
    "tissue_debug_fail_allocs": (C.c_int, [C.c_uint32]),
    "tissue_write_counts": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_uint32]),
    "tissue_step": (C.c_int, [C.c_void_p, C.c_double, C.c_uint32]),
    "tissue_step_timed": (C.c_int, [C.c_void_p, C.c_double, C.c_uint32, _P(C.c_double),
                                    _P(C.c_double)]),
    "tissue_read_counts": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "tissue_read_stats": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t]),
    "tissue_total_events": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tissue_get_step": (C.c_int, [C.c_void_p, _P(C.c_uint32)]),
    "tissue_sync": (C.c_int, [C.c_void_p]),
    "tissue_set_launch": (C.c_int, [C.c_void_p, C.c_uint32]),
    "tissue_set_splitting": (C.c_int, [C.c_void_p, C.c_uint32]),
    "tissue_batch_set_splitting": (C.c_int, [C.c_void_p, C.c_uint32]),
    "tissue_set_launch_config": (C.c_int, [C.c_void_p, _P(Launch)]),
    "tissue_get_launch_config": (C.c_int, [C.c_void_p, _P(Launch)]),
    "tissue_step_noalloc": (C.c_int, [_P(Desc), _P(Model), C.c_void_p, C.c_uint32, C.c_double,
                                      C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tissue_selftest_time": (C.c_int, [C.c_uint64, C.c_uint64, _P(C.c_uint64)]),
    "tissue_batch_create": (C.c_int, [C.c_void_p, C.c_uint32, C.c_void_p, _P(C.c_void_p)]),
    "tissue_batch_set_class_launch": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint32,
                                                 C.c_uint32]),
    "tissue_batch_step": (C.c_int, [C.c_void_p, C.c_double, C.c_uint32]),
    "tissue_batch_set_schedule": (C.c_int, [C.c_void_p, C.c_uint32]),
    "tissue_batch_sync": (C.c_int, [C.c_void_p]),
    "tissue_batch_info": (C.c_int, [C.c_void_p, _P(C.c_uint32), _P(C.c_uint32), _P(C.c_uint64)]),
    "tissue_batch_write_counts": (C.c_int, [C.c_void_p, _P(C.c_void_p), _P(C.c_uint32)]),
    "tissue_batch_read_counts": (C.c_int, [C.c_void_p, _P(C.c_void_p)]),
    "tissue_batch_class_info": (C.c_int, [C.c_void_p, C.c_uint32, _P(C.c_uint32),
                                          _P(C.c_uint32), _P(C.c_uint32), _P(C.c_uint32),
                                          _P(C.c_uint32)]),
    "tissue_batch_set_timing": (C.c_int, [C.c_void_p, C.c_uint32]),
    "tissue_batch_read_timing": (C.c_int, [C.c_void_p, _P(C.c_double), _P(C.c_double),
                                           _P(C.c_double), _P(C.c_double), C.c_uint32]),
    "tissue_batch_set_overlap": (C.c_int, [C.c_void_p, C.c_uint32]),
    "tissue_batch_destroy": (None, [C.c_void_p]),
    "tissue_destroy": (None, [C.c_void_p]),
    "tissue_strerror": (C.c_char_p, [C.c_int]),
}


def checked() -> bool:
    """True when TISSUE_CHECKED=1 selects the range-checked build."""
    return os.environ.get("TISSUE_CHECKED", "0") == "1"


def library_path() -> str:
    name = "libtissue_checked.so" if checked() else "libtissue.so"
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", name)


def lib(build_if_missing: bool = True) -> C.CDLL:
    """Load libtissue.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if build_if_missing:
                from .build import build, is_stale
                if is_stale(checked()):
                    build(checked=checked())
            if not os.path.exists(path):
                raise RuntimeError(f"libtissue.so is missing ({path}); run the build first")
            L = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def desc_of(spec: TissueSpec) -> Desc:
    d = Desc()
    d.width, d.height, d.n = spec.width, spec.height, spec.n
    d.tissue_id, d.seed = spec.tissue_id, spec.seed
    d.init_lambda = (C.c_double * 3)(*spec.init_lambda)
    return d


def model_of(model: dict):
    """The C struct of a model dict: PromoterModel if model["kind"] is
    "promoter", else the Notch-Delta Model."""
    if model.get("kind") == "promoter":
        p = PromoterModel()
        for f in PROMOTER_FIELDS:
            setattr(p, f, float(model[f]))
        return p
    m = Model()
    for f in MODEL_FIELDS:
        setattr(m, f, float(model[f]))
    return m


def state_bytes(spec: TissueSpec) -> int:
    d = desc_of(spec)
    return int(lib().tissue_state_bytes(C.byref(d)))


def scratch_bytes(spec: TissueSpec) -> int:
    d = desc_of(spec)
    return int(lib().tissue_scratch_bytes(C.byref(d)))


def _check(rc: int, what: str):
    if rc != OK:
        raise TissueError(rc, what)


def debug_fail_allocs(n: int) -> None:
    """Make the library's next n device allocations fail as out-of-memory
    (host-side fault injection for tests; 0 disarms)."""
    _check(lib().tissue_debug_fail_allocs(int(n)), "tissue_debug_fail_allocs")


def selftest_time(n_samples: int, seed: int = 1) -> int:
    """Mismatches of the integer binary64 time path against the FP64 unit."""
    out = C.c_uint64()
    _check(lib().tissue_selftest_time(int(n_samples), int(seed), C.byref(out)),
           "tissue_selftest_time")
    return int(out.value)


class Tissue:
    """One tissue on the current CUDA device and torch stream.

    ``buffer`` may be a caller-owned CUDA tensor of at least state_bytes(spec)
    bytes (16-byte aligned); otherwise one is allocated with torch.
    """

    def __init__(self, spec: TissueSpec, buffer=None, stream=None, model: dict | None = None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the tissue SSA runs on a CUDA device; none is available")
        L = lib()
        self.spec = spec
        self._desc = desc_of(spec)
        nbytes = int(L.tissue_state_bytes(C.byref(self._desc)))
        if nbytes == 0:
            raise TissueError(E_ARG, "tissue_state_bytes")
        if buffer is None:
            buffer = torch.empty(nbytes // 4, dtype=torch.int32, device="cuda")
        self.buffer = buffer
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._h = C.c_void_p()
        rc = L.tissue_create(C.byref(self._desc), C.c_void_p(buffer.data_ptr()),
                             buffer.numel() * buffer.element_size(),
                             C.c_void_p(self.stream.cuda_stream), C.byref(self._h))
        _check(rc, "tissue_create")
        self.set_model(model if model is not None else spec.model)
        from .workloads import fidelity_mask
        mask = fidelity_mask(spec)
        if mask is not None:
            self.set_cell_fidelity(mask)

    @property
    def handle(self):
        return self._h

    @property
    def n_ints(self) -> int:
        return self.spec.state_ints

    def set_model(self, model: dict):
        self._model = model_of(model)
        if isinstance(self._model, PromoterModel):
            _check(lib().tissue_set_promoter_model(self._h, C.byref(self._model)),
                   "tissue_set_promoter_model")
        else:
            _check(lib().tissue_set_model(self._h, C.byref(self._model)), "tissue_set_model")

    def set_cell_fidelity(self, well_mixed) -> None:
        """Per cell: 1 (or True) = well-mixed chi, 0 = lattice RDME."""
        a = np.ascontiguousarray(np.asarray(well_mixed).ravel(), dtype=np.uint8)
        _check(lib().tissue_set_cell_fidelity(self._h, a.ctypes.data_as(C.c_void_p), a.size),
               "tissue_set_cell_fidelity")

    def trace_begin(self, capacity: int) -> None:
        """Record every event of the following steps (up to `capacity`)."""
        _check(lib().tissue_trace_begin(self._h, int(capacity)), "tissue_trace_begin")
        self._trace_cap = int(capacity)

    def trace_read(self) -> np.ndarray:
        """The recorded events, sorted by (step, kind, unit, e).  Raises if
        more events happened than the capacity holds."""
        n = C.c_size_t()
        _check(lib().tissue_trace_read(self._h, None, 0, C.byref(n)), "tissue_trace_read")
        if n.value > self._trace_cap:
            raise RuntimeError(f"{n.value} events exceed the trace capacity {self._trace_cap}")
        out = np.zeros(n.value, dtype=EVENT_DTYPE)
        got = C.c_size_t()
        _check(lib().tissue_trace_read(self._h, out.ctypes.data_as(C.c_void_p), out.size,
                                       C.byref(got)), "tissue_trace_read")
        if got.value != n.value:
            raise RuntimeError("events were recorded while reading the trace")
        return np.sort(out, order=["step", "kind", "unit", "e"])

    def trace_end(self) -> None:
        _check(lib().tissue_trace_end(self._h), "tissue_trace_end")

    def set_launch(self, chi_warps_per_block: int):
        _check(lib().tissue_set_launch(self._h, int(chi_warps_per_block)), "tissue_set_launch")

    def set_launch_config(self, kernel: int, lanes_per_cell: int = 32, warps_per_block: int = 4,
                          blocks: int = 0, smem_layout: int = LAYOUT_PREFIX):
        c = Launch(kernel, lanes_per_cell, warps_per_block, blocks, smem_layout)
        _check(lib().tissue_set_launch_config(self._h, C.byref(c)), "tissue_set_launch_config")

    def launch_config(self) -> tuple:
        c = Launch()
        _check(lib().tissue_get_launch_config(self._h, C.byref(c)), "tissue_get_launch_config")
        return (c.kernel, c.lanes_per_cell, c.warps_per_block, c.blocks, c.smem_layout)

    def set_splitting(self, scheme: int):
        _check(lib().tissue_set_splitting(self._h, int(scheme)), "tissue_set_splitting")

    def step(self, dt: float, n_steps: int = 1):
        _check(lib().tissue_step(self._h, float(dt), int(n_steps)), "tissue_step")

    def step_timed(self, dt: float, n_steps: int = 1):
        """Run n_steps and return the device milliseconds of (chi, faces)."""
        a, b = C.c_double(), C.c_double()
        _check(lib().tissue_step_timed(self._h, float(dt), int(n_steps), C.byref(a), C.byref(b)),
               "tissue_step_timed")
        return a.value, b.value

    def read_counts(self, out: np.ndarray | None = None) -> np.ndarray:
        if out is None:
            out = np.empty(self.n_ints, dtype=np.int32)
        _check(lib().tissue_read_counts(self._h, out.ctypes.data_as(C.c_void_p), out.size),
               "tissue_read_counts")
        return out

    def read_counts_into(self, host_tensor) -> None:
        """D2H into a (pinned) torch int32 CPU tensor."""
        _check(lib().tissue_read_counts(self._h, C.c_void_p(host_tensor.data_ptr()),
                                        host_tensor.numel()), "tissue_read_counts")

    def write_counts(self, counts: np.ndarray, step_index: int = 0):
        counts = np.ascontiguousarray(counts, dtype=np.int32)
        _check(lib().tissue_write_counts(self._h, counts.ctypes.data_as(C.c_void_p), counts.size,
                                         int(step_index)), "tissue_write_counts")

    def write_counts_from(self, host_tensor, step_index: int = 0) -> None:
        _check(lib().tissue_write_counts(self._h, C.c_void_p(host_tensor.data_ptr()),
                                         host_tensor.numel(), int(step_index)),
               "tissue_write_counts")

    def read_stats(self):
        cells = self.spec.cells
        ne = np.zeros((3, cells), dtype=np.uint64)
        tl = np.zeros((3, cells), dtype=np.float64)
        _check(lib().tissue_read_stats(self._h, ne.ctypes.data_as(C.c_void_p),
                                       tl.ctypes.data_as(C.c_void_p), 3 * cells),
               "tissue_read_stats")
        return ne, tl

    def total_events(self) -> np.ndarray:
        out = np.zeros(3, dtype=np.uint64)
        _check(lib().tissue_total_events(self._h, out.ctypes.data_as(C.c_void_p)),
               "tissue_total_events")
        return out

    def get_step(self) -> int:
        s = C.c_uint32()
        _check(lib().tissue_get_step(self._h, C.byref(s)), "tissue_get_step")
        return int(s.value)

    def sync(self):
        _check(lib().tissue_sync(self._h), "tissue_sync")

    def close(self):
        if self._h:
            lib().tissue_destroy(self._h)
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
