"""The autotuner: every candidate launch must reproduce the same trajectory
(it raises otherwise), the choice is one of the candidates that fit, and it
is cached."""
import pytest

from paper_1806_10889_gb300.workloads import TissueSpec

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1806_10889_gb300 import autotune  # noqa: E402
from paper_1806_10889_gb300 import tissue as T  # noqa: E402


@pytest.mark.parametrize("n", [8, 16, 32])
def test_tune_tissue_picks_a_fitting_candidate(n):
    spec = TissueSpec(6, 6, n, seed=12)
    res = autotune.tune_tissue(spec, 0.1, steps=1, use_cache=False)
    assert tuple(res["config"]) in autotune.tissue_candidates(spec.V)
    assert str(tuple(res["config"])) in res["ms"]
    again = autotune.tune_tissue(spec, 0.1)
    assert again.get("cached") and tuple(again["config"]) == tuple(res["config"])


def test_tune_batch_classes_and_schedule():
    members = [T.Tissue(TissueSpec(4, 3, n, seed=5, tissue_id=i)) for i, n in enumerate((8, 16, 32, 8))]
    res = autotune.tune_batch(members, 0.1, steps=1, max_clones=4, use_cache=False)
    assert set(res["classes"]) == {64, 256, 1024}
    for V, cfg in res["classes"].items():
        assert tuple(cfg) in autotune.batch_class_candidates(V)
    assert res["steps_per_graph"] in (1, 4)
    for m in members:
        m.close()
