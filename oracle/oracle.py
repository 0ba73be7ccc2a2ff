"""ctypes wrapper of the CPU oracle (test infrastructure only).

Each function restates nothing: it marshals numpy arrays into the C oracle in
``tissue_oracle.c`` and returns its results.  State arrays are int32 laid out
``[cell][species D,N,R][voxel]`` with voxel ``v = vy*n + vx`` and cell
``c = cy*width + cx``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tissue_oracle.c")
_HDR = os.path.join(_HERE, "tissue_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

E_ARG = -1
E_OVERFLOW = -4
E_STATE = -9

ND = 0        # Hill-repressed Delta-Notch lattice model
PROMOTER = 1  # the paper's Notch model with one DNA promoter per cell (Sec. III-A1)


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with code {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, no FMA contraction, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Desc(C.Structure):
    _fields_ = [("width", C.c_uint32), ("height", C.c_uint32), ("n", C.c_uint32),
                ("tissue_id", C.c_uint32), ("seed", C.c_uint64),
                ("init_lambda", C.c_double * 3), ("wm", C.c_void_p)]


_MODEL_FIELDS = ["kD", "K", "kN", "gD", "gN", "gR", "hopD", "hopN", "hopR",
                 "k_in", "k_off", "k_bind"]


_PROMOTER_FIELDS = ["tD", "ka", "kd", "kN", "d", "hop"]


class _Promoter(C.Structure):
    _fields_ = [(f, C.c_double) for f in _PROMOTER_FIELDS]


class _Model(C.Structure):
    _fields_ = ([(f, C.c_double) for f in _MODEL_FIELDS] +
                [("kind", C.c_int32), ("reserved", C.c_int32), ("pm", _Promoter)])


EVENT_DTYPE = np.dtype([("step", "<u4"), ("kind", "<u4"), ("unit", "<u4"), ("e", "<u4"),
                        ("t", "<f8"), ("site", "<u4"), ("channel", "<u4")])


class _Event(C.Structure):
    _fields_ = [("step", C.c_uint32), ("kind", C.c_uint32), ("unit", C.c_uint32),
                ("e", C.c_uint32), ("t", C.c_double), ("site", C.c_uint32),
                ("channel", C.c_uint32)]


assert C.sizeof(_Event) == EVENT_DTYPE.itemsize


@dataclass
class Desc:
    width: int
    height: int
    n: int
    seed: int
    tissue_id: int = 0
    init_lambda: tuple = (5.0, 5.0, 5.0)
    wm: np.ndarray | None = None  # per cell: 1 = well-mixed chi, 0 = lattice RDME

    def __post_init__(self):
        if self.wm is not None:
            self.wm = np.ascontiguousarray(self.wm, dtype=np.uint8)
            if self.wm.size != self.width * self.height:
                raise ValueError("wm needs one entry per cell")

    @property
    def cells(self) -> int:
        return self.width * self.height

    @property
    def V(self) -> int:
        return self.n * self.n

    def to_c(self) -> _Desc:
        d = _Desc()
        d.width, d.height, d.n = self.width, self.height, self.n
        d.tissue_id, d.seed = self.tissue_id, self.seed
        d.init_lambda = (C.c_double * 3)(*self.init_lambda)
        d.wm = self.wm.ctypes.data if self.wm is not None else None
        return d


@dataclass
class Model:
    kD: float = 10.0
    K: float = 20.0
    kN: float = 5.0
    gD: float = 0.1
    gN: float = 0.1
    gR: float = 0.2
    hopD: float = 1.0
    hopN: float = 1.0
    hopR: float = 1.0
    k_in: float = 0.0
    k_off: float = 0.0
    k_bind: float = 0.01

    def to_c(self) -> _Model:
        m = _Model()
        for f in _MODEL_FIELDS:
            setattr(m, f, float(getattr(self, f)))
        m.kind = ND
        return m


@dataclass
class Promoter:
    """The promoter model's rates in lattice units (per unit time):
    transcription tD, NICD binding ka (per NICD in the promoter's voxel),
    unbinding kd, Delta -> NICD across a face kN, decay d, hop per direction."""
    tD: float = 100.0
    ka: float = 256.0
    kd: float = 25.0
    kN: float = 1.0
    d: float = 1.0
    hop: float = 256.0

    def to_c(self) -> _Model:
        m = _Model()
        m.K = 1.0  # unused by this model
        m.kind = PROMOTER
        for f in _PROMOTER_FIELDS:
            setattr(m.pm, f, float(getattr(self, f)))
        return m


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            P = C.POINTER
            L.orc_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
            L.orc_philox4x32_10.restype = None
            L.orc_neg_ln_q58.argtypes = [C.c_uint64]
            L.orc_neg_ln_q58.restype = C.c_uint64
            L.orc_exp_variate.argtypes = [C.c_uint32, C.c_uint32]
            L.orc_exp_variate.restype = C.c_double
            L.orc_quantize.argtypes = [C.c_double, P(C.c_uint64)]
            L.orc_quantize.restype = C.c_int
            L.orc_hill_q.argtypes = [P(_Model), C.c_int64, P(C.c_uint64)]
            L.orc_hill_q.restype = C.c_int
            L.orc_validate.argtypes = [P(_Desc), P(_Model)]
            L.orc_validate.restype = C.c_int
            L.orc_init_counts.argtypes = [P(_Desc), C.c_void_p]
            L.orc_init_counts.restype = C.c_int
            L.orc_init_cell.argtypes = [P(_Desc), C.c_void_p, C.c_uint32]
            L.orc_init_cell.restype = C.c_int
            L.orc_chi_cell.argtypes = [P(_Desc), P(_Model), C.c_void_p, C.c_uint32, C.c_uint32,
                                       C.c_double, P(C.c_uint64), P(C.c_double), C.c_void_p,
                                       C.c_size_t, P(C.c_size_t)]
            L.orc_chi_cell.restype = C.c_int
            L.orc_sig_face.argtypes = [P(_Desc), P(_Model), C.c_void_p, C.c_uint32, C.c_int,
                                       C.c_uint32, C.c_double, P(C.c_uint64), P(C.c_double),
                                       C.c_void_p, C.c_size_t, P(C.c_size_t)]
            L.orc_sig_face.restype = C.c_int
            L.orc_step.argtypes = [P(_Desc), P(_Model), C.c_void_p, C.c_uint32, C.c_uint32,
                                   C.c_double, C.c_void_p, C.c_void_p, C.c_int]
            L.orc_step.restype = C.c_int
            L.orc_step_scheme.argtypes = [P(_Desc), P(_Model), C.c_void_p, C.c_uint32,
                                          C.c_uint32, C.c_double, C.c_int, C.c_void_p,
                                          C.c_void_p, C.c_int]
            L.orc_step_scheme.restype = C.c_int
            L.orc_step_traced.argtypes = [P(_Desc), P(_Model), C.c_void_p, C.c_uint32,
                                          C.c_uint32, C.c_double, C.c_void_p, C.c_size_t,
                                          P(C.c_size_t)]
            L.orc_step_traced.restype = C.c_int
            L.orc_step_traced_scheme.argtypes = [P(_Desc), P(_Model), C.c_void_p, C.c_uint32,
                                                 C.c_uint32, C.c_double, C.c_int, C.c_void_p,
                                                 C.c_size_t, P(C.c_size_t)]
            L.orc_step_traced_scheme.restype = C.c_int
            L.orc_set_mutation.argtypes = [C.c_int]
            L.orc_set_mutation.restype = None
            L.orc_set_paranoid.argtypes = [C.c_int]
            L.orc_set_paranoid.restype = None
            L.orc_get_max_threads.argtypes = []
            L.orc_get_max_threads.restype = C.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _check_state(d: Desc, counts: np.ndarray):
    if counts.dtype != np.int32 or not counts.flags.c_contiguous:
        raise TypeError("counts must be a C-contiguous int32 array")
    if counts.size != d.cells * 3 * d.V:
        raise ValueError("counts has the wrong size for this tissue")


def philox(ctr, key) -> np.ndarray:
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def neg_ln_q58(k: int) -> int:
    return int(lib().orc_neg_ln_q58(int(k)))


def exp_variate(w0: int, w1: int) -> float:
    return float(lib().orc_exp_variate(int(w0), int(w1)))


def quantize(x: float) -> int:
    q = C.c_uint64()
    rc = lib().orc_quantize(float(x), C.byref(q))
    if rc:
        raise OracleError(rc, "quantize")
    return int(q.value)


def hill_q(m: Model, R: int) -> int:
    q = C.c_uint64()
    mc = m.to_c()
    rc = lib().orc_hill_q(C.byref(mc), int(R), C.byref(q))
    if rc:
        raise OracleError(rc, "hill_q")
    return int(q.value)


def init_counts(d: Desc) -> np.ndarray:
    counts = np.zeros(d.cells * 3 * d.V, dtype=np.int32)
    dc = d.to_c()
    rc = lib().orc_init_counts(C.byref(dc), _ptr(counts))
    if rc:
        raise OracleError(rc, "init_counts")
    return counts


def init_cell(d: Desc, counts: np.ndarray, c: int) -> None:
    """Write the initial counts of cell c only into a full-tissue array."""
    _check_state(d, counts)
    dc = d.to_c()
    rc = lib().orc_init_cell(C.byref(dc), _ptr(counts), int(c))
    if rc:
        raise OracleError(rc, "init_cell")


def chi_cell(d: Desc, m: Model, counts: np.ndarray, c: int, step: int, dt: float,
             trace_cap: int = 0):
    """Advance one cell's chi in place; returns (n_events, t_last[, trace])."""
    _check_state(d, counts)
    dc, mc = d.to_c(), m.to_c()
    ne, tl, tlen = C.c_uint64(), C.c_double(), C.c_size_t()
    tr = np.zeros(trace_cap, dtype=EVENT_DTYPE) if trace_cap else None
    rc = lib().orc_chi_cell(C.byref(dc), C.byref(mc), _ptr(counts), c, step, dt,
                            C.byref(ne), C.byref(tl), _ptr(tr) if tr is not None else None,
                            trace_cap, C.byref(tlen))
    if rc:
        raise OracleError(rc, "chi_cell")
    if tr is not None:
        return int(ne.value), float(tl.value), tr[:min(tlen.value, trace_cap)]
    return int(ne.value), float(tl.value)


def sig_face(d: Desc, m: Model, counts: np.ndarray, c: int, axis: int, step: int, dt: float):
    """Advance the x-face (axis 0) or y-face (axis 1) owned by cell c in place."""
    _check_state(d, counts)
    dc, mc = d.to_c(), m.to_c()
    ne, tl, tlen = C.c_uint64(), C.c_double(), C.c_size_t()
    rc = lib().orc_sig_face(C.byref(dc), C.byref(mc), _ptr(counts), c, axis, step, dt,
                            C.byref(ne), C.byref(tl), None, 0, C.byref(tlen))
    if rc:
        raise OracleError(rc, "sig_face")
    return int(ne.value), float(tl.value)


LIE, STRANG = 0, 1


def step(d: Desc, m: Model, counts: np.ndarray, step0: int, n_steps: int, dt: float,
         n_threads: int = 0, scheme: int = LIE):
    """Run n_steps Lie splitting steps in place.

    Returns (n_events[3, cells] uint64, t_last[3, cells] float64) of the last
    step: row 0 chi per cell, rows 1 and 2 the x- and y-face owned by the cell.
    """
    _check_state(d, counts)
    dc, mc = d.to_c(), m.to_c()
    ne = np.zeros((3, d.cells), dtype=np.uint64)
    tl = np.zeros((3, d.cells), dtype=np.float64)
    rc = lib().orc_step_scheme(C.byref(dc), C.byref(mc), _ptr(counts), step0, n_steps, dt,
                               scheme, _ptr(ne), _ptr(tl), n_threads)
    if rc:
        raise OracleError(rc, "step")
    return ne, tl


def step_traced(d: Desc, m: Model, counts: np.ndarray, step0: int, n_steps: int, dt: float,
                trace_cap: int = 1 << 22, scheme: int = 0):
    """Like step() but single-threaded, returning every fired event in order."""
    _check_state(d, counts)
    dc, mc = d.to_c(), m.to_c()
    tr = np.zeros(trace_cap, dtype=EVENT_DTYPE)
    tlen = C.c_size_t()
    rc = lib().orc_step_traced_scheme(C.byref(dc), C.byref(mc), _ptr(counts), step0, n_steps,
                                      dt, int(scheme), _ptr(tr), trace_cap, C.byref(tlen))
    if rc:
        raise OracleError(rc, "step_traced")
    if tlen.value > trace_cap:
        raise ValueError(f"trace overflow: {tlen.value} events > capacity {trace_cap}")
    return tr[:tlen.value]


def set_mutation(which: int) -> None:
    lib().orc_set_mutation(int(which))


def set_paranoid(on: bool) -> None:
    lib().orc_set_paranoid(1 if on else 0)


def max_threads() -> int:
    return int(lib().orc_get_max_threads())
