"""Cells of more than 256 voxels run the chi kernel with 16-bit counts in
shared memory; a cell that holds a count above 65535 when its step starts, or
reaches one during it, is handed back unchanged and redone with 32-bit counts
from the same state and random streams.  Either way the result is the
oracle's, bit for bit: counts, event counts and event times.  These tests
put such counts in some cells of 32x32-, 21x21- and 20x20-voxel tissues (alone, in
a batch, in every launch shape) and check the count limit is still
reported."""
import numpy as np
import pytest

import oracle as O
from paper_1806_10889_gb300.batching import Batch
from paper_1806_10889_gb300.workloads import TissueSpec
from tests._util import orc_desc, orc_model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1806_10889_gb300 import tissue as T  # noqa: E402
from paper_1806_10889_gb300.tissue import Tissue  # noqa: E402

P, PRE, REC = T.KERNEL_PERSISTENT, T.LAYOUT_PREFIX, T.LAYOUT_RECOMPUTE
LIMIT = 0xFFFF  # the largest count the 16-bit layout holds

# D does not hop, and R -> D + N (k_off) releases D faster than it decays:
# a voxel with D just under the limit and many R crosses it within a step.
RELEASE = dict(hopD=0.0, k_off=1.0, k_in=0.0)


def _bits(x):
    return np.asarray(x, dtype=np.float64).view(np.uint64)


def _big_state(spec):
    """Poisson(5) counts from the oracle, then: cell 1 starts above the limit
    (D = 70,000 at voxel 0); cell 4 starts just below it (D = 65,000 next to
    R = 65,535 at voxel 5) and crosses it during the first step."""
    x = O.init_counts(orc_desc(spec)).reshape(spec.cells, 3, spec.V)
    x[1, 0, 0] = 70000
    x[4, 0, 5] = 65000
    x[4, 2, 5] = LIMIT
    return x.ravel().copy()


def _compare(g, d, ref, ne, tl, ctx):
    got = g.read_counts()
    assert np.array_equal(got, ref), f"{ctx}: counts differ at {np.flatnonzero(got != ref)[:5]}"
    gne, gtl = g.read_stats()
    assert np.array_equal(gne, ne), f"{ctx}: event counts differ"
    assert np.array_equal(_bits(gtl), _bits(tl)), f"{ctx}: event times differ"


def _run(spec, x0, dt, n_steps, config=None):
    d, m = orc_desc(spec), orc_model(spec)
    ref = x0.copy()
    g = Tissue(spec)
    if config:
        g.set_launch_config(*config)
    g.write_counts(x0, 0)
    crossed = False
    for k in range(n_steps):
        ne, tl = O.step(d, m, ref, k, 1, dt)
        g.step(dt, 1)
        _compare(g, d, ref, ne, tl, f"{spec.width}x{spec.height}x{spec.n} {config} step {k}")
        crossed |= bool(ref.reshape(spec.cells, 3, spec.V)[4, 0, 5] > LIMIT)
    g.close()
    return ref, crossed


@pytest.mark.parametrize("n", [32, 20, 21])  # 21: V = 441, not a multiple of 4 (scalar copies)
@pytest.mark.parametrize("config", [None, (P, 16, 2, 0, REC)])  # 16 lanes, counts only: 2-4 voxels per lane
def test_counts_above_16_bits_are_redone_bit_exact(n, config):
    spec = TissueSpec(3, 2, n, seed=71, tissue_id=3).with_model(**RELEASE)
    ref, crossed = _run(spec, _big_state(spec), 0.05, 3, config)
    assert crossed, "cell 4 never passed 65535: the mid-step hand-back was not covered"
    x = ref.reshape(spec.cells, 3, spec.V)
    assert x[1, 0, 0] > LIMIT


@pytest.mark.parametrize("config", [(P, 32, 2, 0, PRE), (P, 32, 1, 3, PRE), (P, 16, 4, 0, PRE),
                                    (P, 16, 1, 1, PRE), (P, 8, 2, 0, PRE), (P, 8, 1, 0, PRE),
                                    (P, 32, 2, 0, REC), (P, 32, 4, 0, REC), (P, 32, 1, 3, REC),
                                    (P, 16, 2, 0, REC), (P, 16, 1, 0, REC), (P, 16, 4, 5, REC)])
def test_every_launch_shape_with_16_bit_counts(config):
    spec = TissueSpec(3, 2, 32, seed=73, tissue_id=1).with_model(**RELEASE)
    _, crossed = _run(spec, _big_state(spec), 0.05, 2, config)
    assert crossed


def test_batch_shares_the_redo_list_across_classes():
    """Two large-cell classes (1,024 and 400 voxels) with counts above the
    limit, a large-cell member without, and a small-cell member, stepped as
    one batch."""
    specs = [TissueSpec(3, 2, 32, seed=75, tissue_id=0).with_model(**RELEASE),
             TissueSpec(2, 2, 32, seed=75, tissue_id=1),
             TissueSpec(3, 2, 20, seed=75, tissue_id=2).with_model(**RELEASE),
             TissueSpec(3, 3, 16, seed=75, tissue_id=3)]
    states = [_big_state(s) if i in (0, 2) else O.init_counts(orc_desc(s))
              for i, s in enumerate(specs)]
    members = [Tissue(s) for s in specs]
    for t, x in zip(members, states):
        t.write_counts(x, 0)
    b = Batch(members)
    dt = 0.05
    for k in range(6):
        if k == 2:  # then the large-cell classes with the counts-only layout
            b.set_class_launch(1024, 32, 2, REC)
        if k == 4:  # and with 16 lanes, several voxels per lane
            b.set_class_launch(1024, 16, 2, REC)
            b.set_class_launch(400, 16, 1, REC)
        b.step(dt, 1)
        b.sync()
        for i, s in enumerate(specs):
            ne, tl = O.step(orc_desc(s), orc_model(s), states[i], k, 1, dt)
            _compare(members[i], orc_desc(s), states[i], ne, tl, f"member {i} step {k}")
    b.close()
    for t in members:
        t.close()


def test_count_limit_is_still_reported_for_large_cells():
    """A count at 2^30 - 1 that hops: the 16-bit pass hands the cell back and
    the 32-bit pass reports the overflow, as the oracle does."""
    spec = TissueSpec(2, 1, 32, seed=77, init_lambda=(0.0, 0.0, 0.0)).with_model(hopD=1000.0)
    x = np.zeros(spec.state_ints, dtype=np.int32)
    x[0] = 2 ** 30 - 1
    x[3 * spec.V + spec.V + 7] = 3  # cell 1 has a few N molecules and runs the 16-bit pass
    g = Tissue(spec)
    g.write_counts(x, 0)
    g.step(0.1, 1)
    with pytest.raises(T.TissueError) as e:
        g.read_counts()
    assert e.value.code == T.E_OVERFLOW
    with pytest.raises(O.OracleError):
        O.step(orc_desc(spec), orc_model(spec), x.copy(), 0, 1, 0.1)
    g.close()
