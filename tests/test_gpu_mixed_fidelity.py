"""Mixed-fidelity tissues on the GPU (well-mixed and lattice cells side by
side, Sec. IV), through the C ABI, against the CPU oracle bit for bit: both
single-cell models, every persistent launch shape, Lie and Strang, batches,
the medium workload, and the error paths."""
from dataclasses import replace

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
from paper_1806_10889_gb300.batching import Batch  # noqa: E402
from paper_1806_10889_gb300.tissue import Tissue  # noqa: E402

P, PRE, REC = T.KERNEL_PERSISTENT, T.LAYOUT_PREFIX, T.LAYOUT_RECOMPUTE


def _bits(x):
    return np.asarray(x, dtype=np.float64).view(np.uint64)


def _promoter(w, h, n, fidelity, seed=71, **rates):
    model = W.promoter_model(n)
    model.update(rates)
    return TissueSpec(w, h, n, seed=seed, tissue_id=3, init_lambda=(0.6, 0.4, 0.0), model=model,
                      fidelity=fidelity)


def _nd(w, h, n, fidelity, seed=72, **rates):
    return replace(TissueSpec(w, h, n, seed=seed, tissue_id=4).with_model(**rates),
                   fidelity=fidelity)


def _run_both(spec, dt, n_steps, config=None, scheme=O.LIE):
    d, m = orc_desc(spec), orc_model(spec)
    counts = O.init_counts(d)
    g = Tissue(spec)
    if config:
        g.set_launch_config(*config)
    if scheme == O.STRANG:
        g.set_splitting(T.SPLIT_STRANG)
    for k in range(n_steps):
        ne, tl = O.step(d, m, counts, k, 1, dt, scheme=scheme)
        g.step(dt, 1)
        got = g.read_counts()
        gne, gtl = g.read_stats()
        assert np.array_equal(got, counts), f"{spec.fidelity} step {k}"
        assert np.array_equal(gne, ne) and np.array_equal(_bits(gtl), _bits(tl)), k
    g.close()
    return counts


SPECS = [_promoter(6, 5, 8, "edge:1", kd=3.0),   # 12 well-mixed inside 18 lattice
         _promoter(4, 4, 16, "well_mixed"),
         _promoter(5, 4, 10, "edge:1"),           # V = 100: not a power of two
         _nd(6, 5, 8, "edge:1"),
         _nd(5, 5, 16, "edge:2", k_in=0.02, k_off=0.5),
         _nd(3, 3, 32, "edge:1")]


@pytest.mark.parametrize("spec", SPECS, ids=lambda s: f"{s.model.get('kind', 'nd')}-"
                         f"{s.width}x{s.height}x{s.n}-{s.fidelity}")
def test_mixed_fidelity_matches_oracle(spec):
    ref = _run_both(spec, 0.1, 3)
    # the launch shape of the lattice cells never changes a trajectory
    for cfg in ((P, 8, 4, 0, PRE), (P, 32, 2, 0, PRE), (P, 16, 4, 0, REC)):
        if cfg[4] == REC and spec.V > cfg[1] ** 2:
            continue
        try:
            out = _run_both(spec, 0.1, 3, cfg)
        except T.TissueError as e:  # shared memory of this shape does not fit
            assert e.code == T.E_ARG
            continue
        assert np.array_equal(out, ref)


def test_mixed_fidelity_strang():
    _run_both(_promoter(5, 4, 8, "edge:1"), 0.1, 3, scheme=O.STRANG)


def test_mixed_fidelity_medium_workload():
    run = W.mixed_fidelity()
    _run_both(run.tissue, run.dt, 2)


def test_batch_with_well_mixed_members():
    specs = [_promoter(4, 3, 8, "edge:1", seed=81),
             _nd(3, 3, 16, "well_mixed", seed=82),          # its lattice class is empty
             _nd(4, 4, 16, "lattice", seed=83),
             _promoter(2, 2, 32, "lattice", seed=84),
             _promoter(3, 4, 16, "edge:1", seed=85)]
    members = [Tissue(s) for s in specs]
    b = Batch(members)
    assert b.info()[2] == sum(s.cells for s in specs)
    ref = [O.init_counts(orc_desc(s)) for s in specs]
    dt = 0.05
    for k in range(3):
        b.step(dt, 1)
        b.sync()
        for i, s in enumerate(specs):
            ne, tl = O.step(orc_desc(s), orc_model(s), ref[i], k, 1, dt)
            assert np.array_equal(members[i].read_counts(), ref[i]), (k, i)
            gne, gtl = members[i].read_stats()
            assert np.array_equal(gne, ne) and np.array_equal(_bits(gtl), _bits(tl)), (k, i)
    b.close()
    for m in members:
        m.close()


def test_fidelity_argument_checks_and_warp_kernel():
    spec = _nd(3, 2, 8, "lattice")
    g = Tissue(spec)
    with pytest.raises(T.TissueError) as e:
        g.set_cell_fidelity(np.zeros(5, dtype=np.uint8))  # wrong size
    assert e.value.code == T.E_ARG
    with pytest.raises(T.TissueError) as e:
        g.set_cell_fidelity(np.full(6, 2, dtype=np.uint8))  # not 0/1
    assert e.value.code == T.E_ARG
    g.set_cell_fidelity(np.array([1, 0, 0, 1, 0, 0], dtype=np.uint8))
    g.set_launch_config(T.KERNEL_WARP, 32, 4, 0, PRE)
    with pytest.raises(T.TissueError) as e:
        g.step(0.1, 1)
    assert e.value.code == T.E_ARG
    g.set_cell_fidelity(np.zeros(6, dtype=np.uint8))  # all lattice again: the warp kernel runs
    g.step(0.1, 1)
    g.sync()
    g.close()


def test_well_mixed_invalid_promoter_state_is_reported():
    spec = _promoter(3, 2, 8, "well_mixed")
    g = Tissue(spec)
    x = g.read_counts().reshape(spec.cells, 3, spec.V)
    before = x.copy()
    x[2, 2, 0] = 1  # a bound site away from the promoter voxel
    g.write_counts(x.ravel(), 0)
    g.step(0.1, 1)
    with pytest.raises(T.TissueError) as e:
        g.read_counts()
    assert e.value.code == T.E_STATE
    g.close()
    d = orc_desc(spec)
    with pytest.raises(O.OracleError) as eo:
        O.step(d, orc_model(spec), x.ravel().copy(), 0, 1, 0.1)
    assert eo.value.code == O.E_STATE
    assert before.shape == x.shape
