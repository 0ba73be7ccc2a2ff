"""The paper's promoter Notch model (Sec. III-A1, Table I) on the GPU, through
the C ABI, against the CPU oracle bit for bit: every launch shape of the
persistent chi kernel, Lie and Strang splitting, batches that mix both models
in one launch, and the error paths that belong to this model."""
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


def _spec(w, h, n, seed=61, lam=(0.6, 0.4, 0.0), **rates):
    """A promoter tissue with Table I rates (overridable) and enough NICD that
    the promoters bind and unbind within a few steps."""
    model = W.promoter_model(n)
    model.update(rates)
    return TissueSpec(w, h, n, seed=seed, tissue_id=5, init_lambda=lam, model=model)


def _run_both(spec, dt, n_steps, config=None, scheme=O.LIE):
    d, m = orc_desc(spec), orc_model(spec)
    counts = O.init_counts(d)
    g = Tissue(spec)
    if config:
        g.set_launch_config(*config)
    if scheme == O.STRANG:
        g.set_splitting(T.SPLIT_STRANG)
    assert np.array_equal(g.read_counts(), counts)
    bound_seen = 0
    for k in range(n_steps):
        ne, tl = O.step(d, m, counts, k, 1, dt, scheme=scheme)
        g.step(dt, 1)
        got = g.read_counts()
        gne, gtl = g.read_stats()
        assert np.array_equal(got, counts), f"{spec.width}x{spec.height}x{spec.n} step {k}"
        assert np.array_equal(gne, ne) and np.array_equal(_bits(gtl), _bits(tl)), k
        bound_seen += int(counts.reshape(d.cells, 3, d.V)[:, 2].sum())
    g.close()
    return counts, bound_seen


def _configs(V):
    c = [None]
    for lanes, wpb in ((8, 4), (16, 4), (32, 2), (16, 1)):
        c.append((P, lanes, wpb, 0, PRE))
        if V <= lanes * lanes:
            c.append((P, lanes, min(wpb, 4), 0, REC))
    # counts-only launches with several voxels per lane serve the Notch-Delta
    # model only: a promoter tissue given one runs its prefix launch instead
    if 256 < V <= 1024:
        c.append((P, 16, 2, 0, REC))
    if 64 < V <= 256:
        c.append((P, 8, 2, 0, REC))
    return c


SHAPES = [(5, 3, 16, 0.1),   # several blocks, V = 256 (8 lanes: four voxels a lane per block)
          (3, 2, 10, 0.1),   # V = 100: ragged lane blocks, scalar loads
          (4, 4, 8, 0.1),    # V = 64
          (2, 2, 32, 0.02),  # V = 1024 (16 lanes: two voxels a lane per block)
          (3, 1, 2, 0.2)]    # n = 2: every voxel on a face, the promoter at voxel 3


@pytest.mark.parametrize("w,h,n,dt", SHAPES)
def test_promoter_matches_oracle_every_launch_shape(w, h, n, dt):
    spec = _spec(w, h, n, kd=3.0)
    ref = None
    for cfg in _configs(n * n):
        try:
            out, bound = _run_both(spec, dt, 4, cfg)
        except T.TissueError as e:  # shared memory of this shape does not fit
            assert e.code == T.E_ARG and cfg is not None, (cfg, e)
            continue
        if ref is None:
            ref = out
            assert bound > 0, "the promoters never bound: the test would not cover it"
        assert np.array_equal(out, ref)


def test_promoter_table1_rates_medium_tissue():
    """64x64 cells of 16x16 voxels with the paper's rates, in the launch the
    benchmark times, two full steps against the oracle."""
    run = W.promoter()
    _run_both(run.tissue, run.dt, 2)


@pytest.mark.parametrize("config", [None, (P, 8, 4, 0, PRE), (P, 32, 2, 0, PRE)])
def test_promoter_strang_matches_oracle(config):
    _run_both(_spec(4, 3, 8, kd=3.0), 0.1, 3, config, scheme=O.STRANG)


MIX = [TissueSpec(3, 2, 16, seed=3, tissue_id=0),             # Notch-Delta, V = 256
       _spec(4, 3, 16, seed=8, kd=3.0),                      # promoter, V = 256
       _spec(2, 2, 8, seed=9),                               # promoter, V = 64
       TissueSpec(2, 3, 8, seed=3, tissue_id=4).with_model(kD=19.0),
       _spec(1, 1, 32, seed=10)]                             # promoter alone in its class


@pytest.mark.parametrize("scheme", [T.SPLIT_LIE, T.SPLIT_STRANG])
def test_batch_mixing_both_models_matches_oracle(scheme):
    members = [Tissue(s) for s in MIX]
    b = Batch(members)
    b.set_splitting(scheme)
    ref = [O.init_counts(orc_desc(s)) for s in MIX]
    dt = 0.05
    oscheme = O.LIE if scheme == T.SPLIT_LIE else O.STRANG
    for k in range(3):
        if k == 2:  # every class asked for counts-only launches with several
            # voxels per lane: classes holding promoter tissues fall back to
            # the prefix launch, the others take them
            for V in sorted({x.V for x in MIX}):
                if 256 < V <= 1024:
                    b.set_class_launch(V, 16, 2, REC)
                elif 64 < V <= 256:
                    b.set_class_launch(V, 8, 2, REC)
        b.step(dt, 1)
        b.sync()
        for i, s in enumerate(MIX):
            ne, tl = O.step(orc_desc(s), orc_model(s), ref[i], k, 1, dt, scheme=oscheme)
            assert np.array_equal(members[i].read_counts(), ref[i]), (k, i)
            gne, gtl = members[i].read_stats()
            assert np.array_equal(gne, ne) and np.array_equal(_bits(gtl), _bits(tl)), (k, i)
    b.close()
    for m in members:
        m.close()


def test_promoter_rejects_the_warp_kernel():
    g = Tissue(_spec(2, 2, 8))
    g.set_launch_config(T.KERNEL_WARP, 32, 4, 0, PRE)
    with pytest.raises(T.TissueError) as e:
        g.step(0.1, 1)
    assert e.value.code == T.E_ARG
    g.set_launch_config(P, 8, 4, 0, PRE)
    g.step(0.1, 1)
    g.sync()
    g.close()


@pytest.mark.parametrize("config", [None, (P, 32, 2, 0, PRE), (P, 16, 4, 0, REC)])
def test_promoter_invalid_state_is_reported(config):
    spec = _spec(3, 2, 16)
    g = Tissue(spec)
    if config:
        g.set_launch_config(*config)
    x = g.read_counts().reshape(spec.cells, 3, spec.V)
    x[4, 2, 0] = 1  # a bound site away from the promoter voxel
    g.write_counts(x.ravel(), 0)
    g.step(0.1, 1)
    with pytest.raises(T.TissueError) as e:
        g.read_counts()
    assert e.value.code == T.E_STATE
    # the oracle rejects the same state
    with pytest.raises(O.OracleError) as eo:
        O.step(orc_desc(spec), orc_model(spec), x.ravel().copy(), 0, 1, 0.1)
    assert eo.value.code == O.E_STATE
    g.close()


def test_switching_models_between_steps():
    """A Notch-Delta tissue with no R switched to the promoter model continues
    exactly as the oracle does with the same switch."""
    spec = TissueSpec(3, 3, 8, seed=12, init_lambda=(1.0, 1.0, 0.0)).with_model(gR=0.0, hopR=0.0,
                                                                              k_bind=0.0)
    pm = _spec(3, 3, 8)
    d = orc_desc(spec)
    counts = O.init_counts(d)
    g = Tissue(spec)
    dt = 0.1
    O.step(d, orc_model(spec), counts, 0, 1, dt)
    g.step(dt, 1)
    assert counts.reshape(9, 3, 64)[:, 2].sum() == 0
    g.set_model(pm.model)
    O.step(d, orc_model(pm), counts, 1, 2, dt)
    g.step(dt, 2)
    assert np.array_equal(g.read_counts(), counts)
    g.close()
