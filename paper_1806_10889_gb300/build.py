"""Build libtissue.so (the C ABI of include/tissue.h) for sm_103a with nvcc.

The translation units compile in parallel into ``_build/`` next to this
file; the result is an in-tree shared library that the binding loads with
ctypes.  No torch types cross the ABI, so no torch headers are needed.
"""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libtissue.so")
# The checked build (-DTISSUE_CHECKED): every kernel array index is range
# checked and an out-of-range one is reported (TISSUE_E_BOUNDS) instead of
# accessed.  The binding loads it when TISSUE_CHECKED=1.
LIB_CHECKED = os.path.join(OUT, "libtissue_checked.so")
SOURCES = ["k_chi.cu", "k_chi_seg.cu", "k_chi_seg_gen.cu", "k_chi_seg_pm.cu", "k_chi_seg_narrow.cu", "k_chi_wm.cu", "k_sig.cu", "tissue_lib.cu", "tissue_batch.cu", "tissue_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "--expt-relaxed-constexpr",
                     "-Xcompiler", "-fPIC,-ffp-contract=off", f"-I{INCLUDE}", f"-I{CSRC}"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _inputs() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "tissue.h"))
    return [f for f in files if f.endswith((".cu", ".cuh", ".h"))]


def is_stale(checked: bool = False) -> bool:
    lib = LIB_CHECKED if checked else LIB
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None,
          checked: bool = False) -> str:
    """Compile (if stale) and return the path of libtissue.so (or, with
    checked=True, of libtissue_checked.so)."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not is_stale(checked):
        return lib
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    flags = NVCC_FLAGS + list(extra_flags or []) + (["-DTISSUE_CHECKED"] if checked else [])
    suffix = "_checked.o" if checked else ".o"

    def compile_one(src: str) -> str:
        obj = os.path.join(OUT, src.replace(".cu", suffix))
        cmd = [nvcc, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
