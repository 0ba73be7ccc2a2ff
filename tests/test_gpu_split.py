"""A tissue that fits one wave of the default 16-lane chi launch runs its
heaviest cells (more than 33/32 of the mean chi events in the previous
step) one per warp on a second stream while the others run two per warp.
Which segment runs a cell changes nothing in its trajectory: these tests
check every step against the oracle, bit for bit, with heavy cells present,
for both models and both splitting schemes, and with the stream captured
into a CUDA graph."""
import numpy as np
import pytest

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


def _bits(x):
    return np.asarray(x, dtype=np.float64).view(np.uint64)


def _run(spec, dt, n_steps, scheme=O.LIE):
    d, m = orc_desc(spec), orc_model(spec)
    ref = O.init_counts(d)
    g = Tissue(spec)
    assert g.launch_config()[:4] == (T.KERNEL_PERSISTENT, 16, 4, 0)
    if scheme == O.STRANG:
        g.set_splitting(T.SPLIT_STRANG)
    heavy_steps = 0
    for k in range(n_steps):
        ne, tl = O.step(d, m, ref, k, 1, dt, scheme=scheme)
        g.step(dt, 1)
        assert np.array_equal(g.read_counts(), ref), f"step {k}"
        gne, gtl = g.read_stats()
        assert np.array_equal(gne, ne) and np.array_equal(_bits(gtl), _bits(tl)), f"step {k}"
        chi = ne[0].astype(np.float64)
        heavy_steps += int((32 * chi.size * chi > 33 * chi.sum()).any())
    g.close()
    return heavy_steps


@pytest.mark.parametrize("scheme", [O.LIE, O.STRANG])
def test_split_notch_delta_matches_oracle(scheme):
    spec = TissueSpec(40, 30, 10, seed=81, tissue_id=2).with_model(k_bind=0.05)
    assert _run(spec, 0.1, 4, scheme) >= 3  # every step after the first had heavy cells


def test_split_promoter_matches_oracle():
    model = W.promoter_model(12)
    model["kd"] = 3.0
    spec = TissueSpec(36, 32, 12, seed=83, tissue_id=1, init_lambda=(0.6, 0.4, 0.0), model=model)
    assert _run(spec, 0.1, 3) >= 2


def test_split_inside_a_captured_graph():
    """The fork to the second stream and the join back are recorded into a
    CUDA graph captured on the tissue's stream; replays give the oracle's
    bits."""
    spec = TissueSpec(33, 33, 16, seed=85, tissue_id=4)
    d, m = orc_desc(spec), orc_model(spec)
    ref = O.init_counts(d)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = Tissue(spec)
        g.step(0.05, 1)  # the first step has no event counts yet: all cells light
        O.step(d, m, ref, 0, 1, 0.05)
        g.sync()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream, capture_error_mode="thread_local"):
            g.step(0.05, 1)
        # capture recorded the step without running it; the host step index
        # advanced, so replay twice and compare with steps 1 and 2
        for k in (1, 2):
            graph.replay()
            stream.synchronize()
            O.step(d, m, ref, k, 1, 0.05)
            assert np.array_equal(g.read_counts(), ref), f"replay {k}"
    g.close()
