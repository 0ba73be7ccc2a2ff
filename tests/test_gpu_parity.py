"""GPU path (through the C ABI) against the CPU oracle, bit for bit.

Integer counts must be identical and every binary64 time identical in all 64
bits: the method is an exact SSA whose arithmetic is fully specified, so there
is exactly one correct trajectory.  Inputs are seeded and synthetic; every
expected value comes from oracle/ on the same inputs.
"""
import numpy as np
import pytest

import oracle as O
from paper_1806_10889_gb300 import workloads as W
from paper_1806_10889_gb300.workloads import TissueSpec
from tests._util import orc_desc, orc_model, poisson_gof, q_rate

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # the gpu marker deselects these on CPU runs
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1806_10889_gb300 import tissue as T  # noqa: E402
from paper_1806_10889_gb300.tissue import Tissue  # noqa: E402


def _bits(x):
    return np.asarray(x, dtype=np.float64).view(np.uint64)


def _compare_step(g: Tissue, d, counts, ne, tl, ctx=""):
    got = g.read_counts()
    gne, gtl = g.read_stats()
    if not np.array_equal(got, counts):
        bad = np.flatnonzero(got != counts)
        V = d.V
        raise AssertionError(f"{ctx}: counts differ at {bad.size} ints; first cell {bad[0] // (3 * V)}")
    assert np.array_equal(gne, ne), f"{ctx}: event counts differ"
    assert np.array_equal(_bits(gtl), _bits(tl)), f"{ctx}: event times differ"


def _run_both(spec: TissueSpec, dt: float, n_steps: int, wpb: int | None = None, every=True,
              config: tuple | None = None):
    d, m = orc_desc(spec), orc_model(spec)
    counts = O.init_counts(d)
    g = Tissue(spec)
    if wpb:
        g.set_launch(wpb)
    if config:
        g.set_launch_config(*config)
    assert np.array_equal(g.read_counts(), counts), "initial counts differ"
    for k in range(n_steps):
        ne, tl = O.step(d, m, counts, k, 1, dt)
        g.step(dt, 1)
        if every or k == n_steps - 1:
            _compare_step(g, d, counts, ne, tl, f"{spec} step {k}")
    g.close()
    return counts


@pytest.mark.parametrize("lam", [(5.0, 5.0, 5.0), (0.3, 50.0, 0.0), (700.0, 1.0, 12.5)])
def test_initial_counts_bit_exact(lam):
    spec = TissueSpec(5, 3, 10, seed=123, tissue_id=77, init_lambda=lam)
    d = orc_desc(spec)
    g = Tissue(spec)
    assert np.array_equal(g.read_counts(), O.init_counts(d))
    g.close()


def test_tiny_config_every_step():
    run = W.tiny()
    _run_both(run.tissue, run.dt, run.n_steps)


STRONG = dict(k_bind=0.05)


@pytest.mark.parametrize("w,h,n,dt", [
    (5, 3, 16, 0.1),    # several warps and blocks, V = 256
    (3, 2, 10, 0.1),    # V = 100: ragged lane blocks, scalar (non-vector) loads
    (2, 2, 32, 0.05),   # V = 1024: 32 voxels per lane
    (4, 1, 2, 0.5),     # V = 4: one voxel per lane, no y-faces
    (1, 3, 7, 0.2),     # V = 49 (odd), no x-faces
    (1, 1, 8, 0.1),     # a lone cell: no faces at all
    (7, 5, 8, 1.0),     # long step, many events
    (6, 4, 16, 0.01),   # short step, few events
])
def test_tiles_and_ragged_shapes(w, h, n, dt):
    spec = TissueSpec(w, h, n, seed=1000 + w * 100 + n, tissue_id=w * h).with_model(**STRONG)
    _run_both(spec, dt, 3)


@pytest.mark.parametrize("wpb", [1, 2, 3, 8, 16])
def test_launch_shape_does_not_change_results(wpb):
    spec = TissueSpec(9, 7, 16, seed=5, tissue_id=3)
    _run_both(spec, 0.1, 2, wpb=wpb, every=False)


PERSISTENT = [(T.KERNEL_PERSISTENT, 32, 4, 0, T.LAYOUT_PREFIX),
              (T.KERNEL_PERSISTENT, 16, 4, 0, T.LAYOUT_PREFIX),
              (T.KERNEL_PERSISTENT, 16, 2, 1, T.LAYOUT_PREFIX),
              (T.KERNEL_PERSISTENT, 32, 1, 3, T.LAYOUT_PREFIX),
              (T.KERNEL_PERSISTENT, 16, 4, 0, T.LAYOUT_RECOMPUTE),
              (T.KERNEL_PERSISTENT, 32, 2, 0, T.LAYOUT_RECOMPUTE),
              (T.KERNEL_PERSISTENT, 16, 1, 2, T.LAYOUT_RECOMPUTE),
              (T.KERNEL_PERSISTENT, 16, 1, 0, T.LAYOUT_PREFIX),
              (T.KERNEL_PERSISTENT, 8, 4, 0, T.LAYOUT_PREFIX),
              (T.KERNEL_PERSISTENT, 8, 2, 0, T.LAYOUT_RECOMPUTE),
              (T.KERNEL_PERSISTENT, 8, 1, 1, T.LAYOUT_PREFIX)]


@pytest.mark.parametrize("config", PERSISTENT)
@pytest.mark.parametrize("w,h,n,dt", [
    (5, 3, 16, 0.1), (3, 2, 10, 0.1), (4, 1, 2, 0.5), (1, 3, 7, 0.2), (7, 5, 8, 1.0),
    (2, 2, 32, 0.05), (3, 2, 30, 0.05), (2, 1, 20, 0.1),
])
def test_persistent_kernel_matches_oracle(config, w, h, n, dt):
    """The persistent work-list kernel, one, two or four cells per warp, any
    grid (down to a single block pulling every cell), gives the oracle's bits."""
    if config[4] == T.LAYOUT_RECOMPUTE and n * n > config[1] ** 2 and \
            not (config[1] == 16 and n * n <= 1024) and not (config[1] == 8 and n * n <= 256):
        pytest.skip("the recompute layout needs V <= lanes^2, or 4 voxels per lane at most")
    lanes, wpb = config[1], config[2]
    blocks_v = 1
    while lanes * blocks_v < n * n:
        blocks_v *= 2
    per_voxel = 20 if config[4] == T.LAYOUT_PREFIX else 12
    if wpb * (32 // lanes) * (512 + per_voxel * lanes * blocks_v) > 227 * 1024:
        pytest.skip("this launch shape does not fit shared memory for these cells")
    spec = TissueSpec(w, h, n, seed=2000 + w * 100 + n, tissue_id=w * h).with_model(**STRONG)
    _run_both(spec, dt, 3, config=config)


def test_launch_config_validation():
    g = Tissue(TissueSpec(2, 2, 32, seed=1))
    with pytest.raises(T.TissueError):  # recompute layout: V = 1024 is 16 voxels per lane at 8 lanes
        g.set_launch_config(T.KERNEL_PERSISTENT, 8, 4, 0, T.LAYOUT_RECOMPUTE)
    # 16 lanes cover up to four voxels each in the recompute layout (V <= 1024)
    g.set_launch_config(T.KERNEL_PERSISTENT, 16, 4, 0, T.LAYOUT_RECOMPUTE)
    with pytest.raises(T.TissueError):
        g.set_launch_config(7, 32, 4, 0)
    with pytest.raises(T.TissueError):
        g.set_launch_config(T.KERNEL_PERSISTENT, 32, 8, 0, T.LAYOUT_RECOMPUTE)  # <= 4 warps
    g.set_launch_config(T.KERNEL_PERSISTENT, 32, 2, 0)
    assert g.launch_config() == (T.KERNEL_PERSISTENT, 32, 2, 0, T.LAYOUT_PREFIX)
    g.close()


@pytest.mark.parametrize("config", [None, (T.KERNEL_PERSISTENT, 16, 4, 0),
                                    (T.KERNEL_PERSISTENT, 32, 4, 0),
                                    (T.KERNEL_PERSISTENT, 16, 4, 0, T.LAYOUT_RECOMPUTE),
                                    (T.KERNEL_PERSISTENT, 8, 2, 0, T.LAYOUT_PREFIX)])
def test_in_voxel_binding_channels(config):
    spec = TissueSpec(3, 3, 6, seed=17).with_model(k_in=0.02, k_off=0.7)
    _run_both(spec, 0.2, 4, config=config)


@pytest.mark.parametrize("config", [None, (T.KERNEL_WARP, 32, 4, 0),
                                    (T.KERNEL_PERSISTENT, 16, 4, 0, T.LAYOUT_RECOMPUTE),
                                    (T.KERNEL_PERSISTENT, 8, 4, 0, T.LAYOUT_PREFIX)])
def test_medium_config_full_tissue(config):
    """64x64 cells of 16x16 voxels at dt = 0.1: the whole tissue, two steps,
    in the default launch shape (the benchmark's) and the warp kernel."""
    run = W.medium(0.1)
    _run_both(run.tissue, run.dt, 2, config=config)


@pytest.mark.parametrize("dt", [0.01, 1.0])
def test_medium_config_other_dt(dt):
    """The medium tissue at the two other step lengths, whole tissue."""
    run = W.medium(dt)
    _run_both(run.tissue, run.dt, 2 if dt < 1.0 else 1)


def _neighbourhood_reference(d, m, c, dt, n_steps):
    """Oracle counts of cell c after steps 0..n_steps-1 of a large tissue,
    computed from the cells that can influence it.  A face carries
    influence one cell per phase along its axis, so a wrong cell at the edge
    of a block of Chebyshev radius K reaches at most one cell further in per
    step.  Simulating the block of radius K = n_steps around c therefore
    leaves c exact.  Returns c's counts and its chi statistics of the last
    step."""
    counts = np.zeros(d.cells * 3 * d.V, dtype=np.int32)
    Wd, Hd = d.width, d.height
    cx, cy = c % Wd, c // Wd
    K = n_steps
    xs = [x for x in range(cx - K, cx + K + 1) if 0 <= x < Wd]
    ys = [y for y in range(cy - K, cy + K + 1) if 0 <= y < Hd]
    for y in ys:
        for x in xs:
            O.init_cell(d, counts, y * Wd + x)
    stats = None
    for k in range(n_steps):
        for y in ys:
            for x in xs:
                st = O.chi_cell(d, m, counts, y * Wd + x, k, dt)
                if y * Wd + x == c:
                    stats = st
        for y in ys:
            for x in xs[:-1]:
                O.sig_face(d, m, counts, y * Wd + x, 0, k, dt)
        for y in ys[:-1]:
            for x in xs:
                O.sig_face(d, m, counts, y * Wd + x, 1, k, dt)
    V = d.V
    return counts[c * 3 * V:(c + 1) * 3 * V].copy(), stats


def test_large_config_sampled_cells():
    """256x256 cells of 32x32 voxels (0.8 GB of state), steps 0 and 1 at
    dt = 0.1, in the launch shape the benchmark times; sampled cells
    (corners, edges, interior) checked against the oracle computed on the
    neighbourhood that can influence them."""
    run = W.large()
    spec = run.tissue
    d, m = orc_desc(spec), orc_model(spec)
    g = Tissue(spec)  # default launch shape, as the benchmark uses
    g.step(run.dt, 2)
    got = g.read_counts()
    gne, gtl = g.read_stats()
    g.close()
    Wd = spec.width
    rng = np.random.default_rng(99)
    samples = [0, Wd - 1, Wd * (Wd - 1), Wd * Wd - 1, Wd // 2, Wd * 7] + \
              [int(x) for x in rng.integers(0, spec.cells, size=6)]
    V = spec.V
    for c in samples:
        ref, (ne, tl) = _neighbourhood_reference(d, m, c, run.dt, 2)
        assert gne[0, c] == ne and _bits(gtl[0, c]) == _bits(tl), c
        assert np.array_equal(got[c * 3 * V:(c + 1) * 3 * V], ref), c


def test_resume_from_checkpoint_is_bit_identical():
    spec = TissueSpec(4, 4, 8, seed=21, tissue_id=5).with_model(**STRONG)
    a = Tissue(spec)
    a.step(0.1, 6)
    want = a.read_counts()
    want_stats = a.read_stats()
    b = Tissue(spec)
    b.step(0.1, 3)
    ckpt = b.read_counts()
    b.close()
    c = Tissue(spec)
    c.write_counts(ckpt, step_index=3)
    c.step(0.1, 3)
    assert c.get_step() == 6
    assert np.array_equal(c.read_counts(), want)
    got_stats = c.read_stats()
    assert np.array_equal(got_stats[0], want_stats[0])
    assert np.array_equal(_bits(got_stats[1]), _bits(want_stats[1]))
    a.close()
    c.close()


def test_rerun_is_bit_identical_and_totals_add_up():
    spec = TissueSpec(6, 6, 16, seed=8)
    runs = []
    for _ in range(2):
        g = Tissue(spec)
        per_step = np.zeros(3, dtype=np.uint64)
        for k in range(3):
            g.step(0.1, 1)
            per_step += g.read_stats()[0].sum(axis=1)
        runs.append((g.read_counts(), g.total_events()))
        assert np.array_equal(runs[-1][1], per_step)
        g.close()
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])


@pytest.mark.parametrize("config", [None, (T.KERNEL_PERSISTENT, 16, 4, 0),
                                    (T.KERNEL_PERSISTENT, 16, 4, 0, T.LAYOUT_RECOMPUTE)])
def test_overflow_is_reported(config):
    spec = TissueSpec(2, 1, 2, seed=1, init_lambda=(0.0, 0.0, 0.0)).with_model(hopD=1000.0)
    g = Tissue(spec)
    if config:
        g.set_launch_config(*config)
    x = np.zeros(spec.state_ints, dtype=np.int32)
    x[0] = 2 ** 30 - 1
    g.write_counts(x)
    g.step(0.1, 1)
    with pytest.raises(T.TissueError) as e:
        g.read_counts()
    assert e.value.code == T.E_OVERFLOW
    # the oracle reports the same condition
    with pytest.raises(O.OracleError):
        O.step(orc_desc(spec), orc_model(spec), x.copy(), 0, 1, 0.1)
    g.close()


def test_step_without_model_and_bad_dt():
    spec = TissueSpec(2, 2, 4, seed=1)
    g = Tissue(spec)
    with pytest.raises(T.TissueError) as e:
        g.step(0.0, 1)
    assert e.value.code == T.E_ARG
    with pytest.raises(T.TissueError):
        g.write_counts(np.full(spec.state_ints, -1, dtype=np.int32))
    g.close()


def test_gpu_ensemble_immigration_death_law():
    """Closed form on the GPU at scale: 64x64 cells of 16x16 voxels with Notch
    only; every voxel is Poisson(m(t)) with m(t) = lam e^-gt + (b/g)(1-e^-gt)."""
    zero = dict(kD=0.0, kN=5.0, gD=0.0, gN=0.1, gR=0.0, hopD=0.0, hopN=1.0, hopR=0.0,
                k_in=0.0, k_off=0.0, k_bind=0.01)
    spec = TissueSpec(64, 64, 16, seed=404, init_lambda=(0.0, 7.0, 0.0)).with_model(**zero)
    g = Tissue(spec)
    g.step(0.5, 30)
    x = g.read_counts().reshape(spec.cells, 3, spec.V)[:, 1, :]
    g.close()
    import math
    gq = q_rate(0.1)
    mean = 7.0 * math.exp(-gq * 15.0) + (q_rate(5.0) / gq) * (1 - math.exp(-gq * 15.0))
    p, z = poisson_gof(x, mean)
    assert p > 0.01 and abs(z) < 3, (p, z)


def _run_from(spec, counts0, dt, n_steps, config=None):
    """GPU and oracle from the same explicit state, compared every step."""
    d, m = orc_desc(spec), orc_model(spec)
    counts = counts0.copy()
    g = Tissue(spec)
    if config:
        g.set_launch_config(*config)
    g.write_counts(counts0, 0)
    for k in range(n_steps):
        ne, tl = O.step(d, m, counts, k, 1, dt)
        g.step(dt, 1)
        _compare_step(g, d, counts, ne, tl, f"{spec} step {k}")
    g.close()
    return counts


@pytest.mark.parametrize("config", [None, (T.KERNEL_WARP, 32, 4, 0),
                                    (T.KERNEL_PERSISTENT, 32, 2, 0, T.LAYOUT_PREFIX),
                                    (T.KERNEL_PERSISTENT, 8, 4, 0, T.LAYOUT_RECOMPUTE)])
def test_empty_tissue_fires_nothing(config):
    """No molecules and no production: total propensity 0 everywhere, so
    every module call ends at once with no event and t_last = 0."""
    spec = TissueSpec(3, 2, 8, seed=5).with_model(kD=0.0, kN=0.0)
    zero = np.zeros(spec.state_ints, dtype=np.int32)
    out = _run_from(spec, zero, 0.1, 2, config)
    assert not out.any()


@pytest.mark.parametrize("config", [None, (T.KERNEL_PERSISTENT, 16, 4, 0, T.LAYOUT_PREFIX),
                                    (T.KERNEL_PERSISTENT, 16, 4, 0, T.LAYOUT_RECOMPUTE)])
def test_counts_at_the_maximum(config):
    """Voxels holding the largest allowed count (2^30 - 1) with rates small
    enough to stay below the propensity limit: the exactly checked
    large-count path, bit for bit."""
    # k_in > 0 lowers the bound below which counts take the unchecked fast
    # path (2^25 here), so these voxels take the checked one; no voxel holds
    # both D and N, so no total comes near 2^52
    spec = TissueSpec(2, 2, 4, seed=6).with_model(kD=0.0, kN=0.0, gD=1e-6, gN=2e-6, gR=0.0,
                                                  hopD=0.0, hopN=0.0, hopR=0.0, k_bind=0.0,
                                                  k_in=1e-9)
    x = np.zeros(spec.state_ints, dtype=np.int32).reshape(spec.cells, 3, spec.V)
    x[:, 0, 3] = (1 << 30) - 1
    x[1, 1, 0] = (1 << 30) - 1
    x[2, 0, :] = 1000
    out = _run_from(spec, x.ravel(), 0.5, 2, config).reshape(spec.cells, 3, spec.V)
    assert out[:, 0, 3].min() < (1 << 30) - 1  # decay happened


def test_tiny_step_length():
    """dt = 1e-9: almost every call ends before its first event."""
    run = W.tiny()
    _run_both(run.tissue, 1e-9, 3)


@pytest.mark.parametrize("lanes,n", [(16, 32), (16, 24), (16, 20), (16, 17), (8, 16), (8, 12),
                                     (8, 9)])
@pytest.mark.parametrize("wpb", [1, 2, 4])
def test_counts_only_layout_with_several_voxels_per_lane(lanes, n, wpb):
    """The counts-only layout with more voxels per block than lanes: each
    block splits into 2 or 4 sub-blocks whose running sums the owning lane
    keeps, and an event recomputes one sub-block, one voxel per lane (16
    lanes: V = 1024, 576, 400, 289; 8 lanes: V = 256, 144, 81; all but the
    first of each with partly empty blocks and sub-blocks), every step
    bit-exact with the oracle."""
    spec = TissueSpec(3, 3, n, seed=300 + n, tissue_id=wpb).with_model(**STRONG)
    _run_both(spec, 0.1, 3, config=(T.KERNEL_PERSISTENT, lanes, wpb, 0, T.LAYOUT_RECOMPUTE))


P_, R_ = T.LAYOUT_PREFIX, T.LAYOUT_RECOMPUTE


@pytest.mark.parametrize("side,n,want", [
    (16, 32, (T.KERNEL_PERSISTENT, 32, 2, 0, P_)),   # 256 cells: the machine is not full
    (46, 32, (T.KERNEL_PERSISTENT, 32, 2, 0, P_)),   # 2,116 cells: one prefix wave
    (47, 32, (T.KERNEL_PERSISTENT, 16, 2, 0, R_)),   # 2,209 cells: counts only
    (77, 16, (T.KERNEL_PERSISTENT, 16, 4, 0, P_)),   # 5,929 cells: one prefix wave
    (78, 16, (T.KERNEL_PERSISTENT, 8, 2, 0, R_)),    # 6,084 cells: counts only
    (128, 8, (T.KERNEL_PERSISTENT, 8, 4, 0, P_)),    # 8x8-voxel cells keep the prefix layout
])
def test_default_launch_by_cell_size_and_count(side, n, want):
    """The default launch takes the counts-only layout past one wave of the
    prefix launch (2,128 cells of 257..1,024 voxels, 6,080 of 65..256)."""
    g = Tissue(TissueSpec(side, side, n, seed=1))
    assert g.launch_config() == want
    g.close()


@pytest.mark.parametrize("side,n", [(47, 32), (78, 16)])
def test_default_counts_only_launch_matches_oracle(side, n):
    """Whole tissues just past the thresholds, on their default (counts-only)
    launch, every step bit-exact with the oracle."""
    _run_both(TissueSpec(side, side, n, seed=40 + n, tissue_id=side), 0.1, 2)
