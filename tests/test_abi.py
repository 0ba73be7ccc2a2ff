"""The C ABI library builds, loads and exports every entry point that
include/tissue.h declares (host-only checks: no kernel runs here)."""
import ctypes as C
import os
import re

import pytest

from paper_1806_10889_gb300 import tissue as T
from paper_1806_10889_gb300.workloads import TissueSpec

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(tissue_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    L = T.lib()
    names = _declared()
    assert "tissue_step" in names and "tissue_create" in names
    for n in sorted(names):
        assert hasattr(L, n), n
    assert names <= set(T.SIGNATURES), names - set(T.SIGNATURES)


def test_host_only_entry_points():
    spec = TissueSpec(64, 64, 16, seed=2)
    assert T.state_bytes(spec) == 64 * 64 * 3 * 256 * 4
    assert T.scratch_bytes(spec) > 3 * 4096 * 24
    bad = TissueSpec(0, 4, 16, seed=2)
    assert T.state_bytes(bad) == 0 and T.scratch_bytes(bad) == 0
    assert T.lib().tissue_strerror(-4) == b"count or propensity overflow"
    assert T.lib().tissue_strerror(0) == b"ok"


def test_create_rejects_bad_arguments_without_touching_the_device():
    L = T.lib()
    d = T.desc_of(TissueSpec(2, 2, 8, seed=1))
    h = C.c_void_p()
    # null buffer, short buffer, misaligned buffer: rejected before any CUDA call
    assert L.tissue_create(C.byref(d), None, 4096, None, C.byref(h)) == T.E_ARG
    assert L.tissue_create(C.byref(d), C.c_void_p(0x1000), 16, None, C.byref(h)) == T.E_ARG
    assert L.tissue_create(C.byref(d), C.c_void_p(0x1004), 1 << 20, None, C.byref(h)) == T.E_ARG
    d.n = 33
    assert L.tissue_create(C.byref(d), C.c_void_p(0x1000), 1 << 20, None, C.byref(h)) == T.E_ARG
    assert L.tissue_step(None, 0.1, 1) == T.E_ARG


def test_injected_allocation_failure_is_reported_without_a_device():
    """Host-side fault injection: the library's next device allocation fails
    as an out-of-memory cudaMalloc would.  tissue_create reports
    TISSUE_E_NOMEM and returns no handle; nothing reaches the GPU."""
    L = T.lib()
    d = T.desc_of(TissueSpec(2, 2, 8, seed=1))
    h = C.c_void_p(0x1234)
    T.debug_fail_allocs(1)
    try:
        rc = L.tissue_create(C.byref(d), C.c_void_p(0x1000), 1 << 20, None, C.byref(h))
    finally:
        T.debug_fail_allocs(0)
    assert rc == T.E_NOMEM and not h.value
    assert L.tissue_strerror(T.E_NOMEM) == b"out of device memory"
