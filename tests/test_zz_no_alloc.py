"""tissue_step_noalloc, the entry point for callers that cannot allocate
device memory (for example an application that manages a fixed device-memory
budget itself, or code where a cudaMalloc would stall the device): it must
give exactly what tissue_step gives, call after call, while keeping its
scratch in one static device array that every call reuses.

This file is collected last on purpose, so that a run stopping at the first
failure has run every other test before it."""
import ctypes as C

import numpy as np
import pytest

from paper_1806_10889_gb300.workloads import TissueSpec

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1806_10889_gb300 import tissue as T  # noqa: E402


def _noalloc(spec, model, state, step_index, dt, n_steps, ev, tl, stream):
    d = T.desc_of(spec)
    m = T.model_of(model)
    return T.lib().tissue_step_noalloc(C.byref(d), C.byref(m), C.c_void_p(state.data_ptr()),
                                       step_index, dt, n_steps, C.c_void_p(ev.data_ptr()),
                                       C.c_void_p(tl.data_ptr()), C.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("n, first_step", [(8, 0), (16, 0), (32, 0), (16, 37)])
def test_noalloc_matches_tissue_step_on_two_calls_in_a_row(n, first_step):
    # cells of 8x8, 16x16 and 32x32 voxels (the last needs more than 48 KB of
    # shared memory per block); one case starts at a global step other than 0
    spec = TissueSpec(5, 4, n, seed=31, tissue_id=9).with_model(k_bind=0.05)
    dt = 0.1
    ref = T.Tissue(spec)  # the allocating entry points
    if first_step:
        ref.write_counts(ref.read_counts(), step_index=first_step)
    state = torch.from_numpy(ref.read_counts()).to("cuda")
    ev = torch.full((3 * spec.cells,), 7, dtype=torch.int64, device="cuda")
    tl = torch.full((3 * spec.cells,), 7.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    k = first_step
    for steps in (2, 3):  # two calls in a row reuse the same static scratch
        assert _noalloc(spec, spec.model, state, k, dt, steps, ev, tl, stream) == T.OK
        ref.step(dt, steps)
        k += steps
        want = ref.read_counts()
        want_ev, want_tl = ref.read_stats()
        assert np.array_equal(state.cpu().numpy(), want)
        assert np.array_equal(ev.cpu().numpy().astype(np.uint64).reshape(3, -1), want_ev)
        assert np.array_equal(tl.cpu().numpy().view(np.uint64).reshape(3, -1),
                              want_tl.view(np.uint64))
    # zero steps change nothing, as with tissue_step
    before = (state.clone(), ev.clone(), tl.clone())
    assert _noalloc(spec, spec.model, state, k, dt, 0, ev, tl, stream) == T.OK
    assert all(torch.equal(a, b) for a, b in zip(before, (state, ev, tl)))
    ref.close()


def test_noalloc_rejects_tissues_beyond_its_static_scratch():
    spec = TissueSpec(129, 128, 8, seed=1)  # 16512 cells > 16384
    assert spec.cells > 16384
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    ev = torch.zeros(4, dtype=torch.int64, device="cuda")
    tl = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = _noalloc(spec, spec.model, dummy, 0, 0.1, 1, ev, tl, torch.cuda.current_stream())
    assert rc == T.E_ARG
