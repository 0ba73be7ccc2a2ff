"""Full event logs: every event the GPU fires -- step, module call, unit,
event index, binary64 time, site and channel -- equals the oracle's, for
lattice chi, well-mixed chi and both face phases.  The traced launches run
the model-generic instantiation of the persistent chi kernel (the same
template as the Notch-Delta fast path, whose counts and statistics the
parity tests check every step)."""
import numpy as np
import pytest
from dataclasses import replace

import oracle as O
from paper_1806_10889_gb300 import workloads as W
from paper_1806_10889_gb300.workloads import TissueSpec
from tests._util import orc_desc, orc_model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1806_10889_gb300 import tissue as T  # noqa: E402
from paper_1806_10889_gb300.tissue import Tissue  # noqa: E402

P, PRE, REC = T.KERNEL_PERSISTENT, T.LAYOUT_PREFIX, T.LAYOUT_RECOMPUTE


def _oracle_trace(spec, dt, n_steps, scheme=O.LIE):
    d, m = orc_desc(spec), orc_model(spec)
    counts = O.init_counts(d)
    tr = O.step_traced(d, m, counts, 0, n_steps, dt, trace_cap=1 << 23, scheme=scheme)
    tr = np.sort(tr, order=["step", "kind", "unit", "e"])
    return counts, tr


def _gpu_trace(spec, dt, n_steps, config=None, cap=1 << 23, scheme=O.LIE):
    g = Tissue(spec)
    if config:
        g.set_launch_config(*config)
    if scheme == O.STRANG:
        g.set_splitting(T.SPLIT_STRANG)
    g.trace_begin(cap)
    g.step(dt, n_steps)
    counts = g.read_counts()
    tr = g.trace_read()
    g.trace_end()
    g.close()
    return counts, tr


def _same(a, b):
    assert a.size == b.size, (a.size, b.size)
    for f in ("step", "kind", "unit", "e", "site", "channel"):
        bad = np.flatnonzero(a[f] != b[f])
        assert bad.size == 0, (f, a[bad[:3]], b[bad[:3]])
    assert np.array_equal(a["t"].view(np.uint64), b["t"].view(np.uint64))


def test_tiny_config_full_event_log():
    """The tiny configuration, all 100 steps: ~1.6 M events."""
    run = W.tiny()
    c_ref, t_ref = _oracle_trace(run.tissue, run.dt, run.n_steps)
    c_gpu, t_gpu = _gpu_trace(run.tissue, run.dt, run.n_steps)
    assert np.array_equal(c_gpu, c_ref)
    assert set(np.unique(t_ref["kind"])) == {1, 2, 3}
    _same(t_gpu, t_ref)


@pytest.mark.parametrize("config", [(P, 8, 4, 0, PRE), (P, 16, 4, 0, PRE), (P, 32, 2, 0, PRE),
                                    (P, 16, 4, 0, REC)])
def test_event_log_every_launch_shape(config):
    spec = TissueSpec(3, 3, 16, seed=31, tissue_id=2).with_model(k_bind=0.05)
    c_ref, t_ref = _oracle_trace(spec, 0.1, 3)
    c_gpu, t_gpu = _gpu_trace(spec, 0.1, 3, config)
    assert np.array_equal(c_gpu, c_ref)
    _same(t_gpu, t_ref)


@pytest.mark.parametrize("fidelity", ["lattice", "edge:1", "well_mixed"])
def test_event_log_promoter_and_mixed_fidelity(fidelity):
    model = W.promoter_model(8)
    model["kd"] = 3.0
    spec = TissueSpec(4, 3, 8, seed=33, tissue_id=1, init_lambda=(0.6, 0.4, 0.0), model=model,
                      fidelity=fidelity)
    c_ref, t_ref = _oracle_trace(spec, 0.1, 4)
    c_gpu, t_gpu = _gpu_trace(spec, 0.1, 4)
    assert np.array_equal(c_gpu, c_ref)
    _same(t_gpu, t_ref)


def test_event_log_notch_delta_well_mixed_cells():
    spec = replace(TissueSpec(4, 4, 8, seed=35).with_model(k_in=0.02, k_off=0.4),
                   fidelity="edge:1")
    c_ref, t_ref = _oracle_trace(spec, 0.1, 3)
    c_gpu, t_gpu = _gpu_trace(spec, 0.1, 3)
    assert np.array_equal(c_gpu, c_ref)
    _same(t_gpu, t_ref)


def test_trace_overflow_and_warp_kernel_are_reported():
    spec = TissueSpec(2, 2, 8, seed=37)
    g = Tissue(spec)
    g.trace_begin(100)
    g.step(0.1, 1)
    with pytest.raises(RuntimeError):
        g.trace_read()  # far more than 100 events happened
    g.set_launch_config(T.KERNEL_WARP, 32, 4, 0, PRE)
    with pytest.raises(T.TissueError) as e:
        g.step(0.1, 1)
    assert e.value.code == T.E_ARG
    g.trace_end()
    g.step(0.1, 1)  # the warp kernel runs again without a trace
    g.sync()
    g.close()


def test_event_log_strang_splitting():
    """Strang's five module calls per step, the second face halves on their
    own Philox tags (5 and 6)."""
    spec = TissueSpec(3, 3, 8, seed=39).with_model(k_bind=0.05)
    c_ref, t_ref = _oracle_trace(spec, 0.1, 4, O.STRANG)
    c_gpu, t_gpu = _gpu_trace(spec, 0.1, 4, scheme=O.STRANG)
    assert np.array_equal(c_gpu, c_ref)
    assert set(np.unique(t_ref["kind"])) == {1, 2, 3, 5, 6}
    _same(t_gpu, t_ref)
