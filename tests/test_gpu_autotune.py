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


def _diverge_second(tissues):
    """Make the second candidate seen differ: one more Delta in voxel 0."""
    seen = []

    def hook(cfg, t):
        seen.append(cfg)
        if len(seen) == 2:
            for x in (t if isinstance(t, list) else [t]):
                c = x.read_counts()
                c[0] += 1
                x.write_counts(c, step_index=x.get_step())
    return hook, seen


def test_tune_tissue_raises_when_a_candidate_diverges():
    spec = TissueSpec(4, 4, 16, seed=21)
    hook, seen = _diverge_second(None)
    cands = [(T.KERNEL_PERSISTENT, 16, 4, 0, T.LAYOUT_PREFIX),
             (T.KERNEL_PERSISTENT, 32, 2, 0, T.LAYOUT_PREFIX)]
    with pytest.raises(autotune.VariantMismatch):
        autotune.tune_tissue(spec, 0.1, steps=1, candidates=cands, use_cache=False,
                             on_candidate=hook)
    assert len(seen) == 2
    # without the planted difference the same candidates agree
    res = autotune.tune_tissue(spec, 0.1, steps=1, candidates=cands, use_cache=False)
    assert tuple(res["config"]) in cands


def test_tune_batch_raises_when_a_candidate_diverges():
    members = [T.Tissue(TissueSpec(3, 3, 16, seed=5, tissue_id=i)) for i in range(3)]
    hook, seen = _diverge_second(None)
    with pytest.raises(autotune.VariantMismatch):
        autotune.tune_batch(members, 0.1, steps=1, max_clones=3, use_cache=False,
                            on_candidate=hook)
    assert len(seen) == 2
    for m in members:
        m.close()
