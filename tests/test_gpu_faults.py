"""Failure handling on the device path, with the failures made on the host:
an injected allocation failure in each allocating call is reported as
TISSUE_E_NOMEM, leaves no half-built object, and the next call succeeds."""
import numpy as np
import pytest

from paper_1806_10889_gb300.workloads import TissueSpec

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1806_10889_gb300 import tissue as T  # noqa: E402
from paper_1806_10889_gb300.batching import Batch  # noqa: E402
from paper_1806_10889_gb300.tissue import Tissue  # noqa: E402


def _fails_once(fn):
    T.debug_fail_allocs(1)
    try:
        with pytest.raises(T.TissueError) as e:
            fn()
    finally:
        T.debug_fail_allocs(0)
    assert e.value.code == T.E_NOMEM


def test_injected_allocation_failures():
    spec = TissueSpec(3, 2, 8, seed=4)
    _fails_once(lambda: Tissue(spec))
    a, b = Tissue(spec), Tissue(TissueSpec(2, 2, 16, seed=5))
    _fails_once(lambda: Batch([a, b]))
    _fails_once(lambda: a.trace_begin(1000))
    # everything works afterwards, and results are unaffected
    ref = Tissue(spec)
    ref.step(0.1, 2)
    bt = Batch([a, b])
    bt.step(0.1, 2)
    bt.sync()
    assert np.array_equal(a.read_counts(), ref.read_counts())
    bt.close()
    for t in (a, b, ref):
        t.close()
