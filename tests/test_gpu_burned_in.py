"""The GPU against the oracle from burned-in states, where the benchmarks time
their steps: tens of molecules per voxel (about 60 D, 30 N and 10 R in the
medium tissue after 20 time units) instead of the initial Poisson(5), so the
Hill values, the small-count fast path of the voxel totals and the 16-bit
counts of large cells all run in their working regime.

The GPU advances the workload alone; its state is then handed both to a fresh
tissue (tissue_write_counts, checkpoint resume) and to the oracle, and the
following steps must agree bit for bit: counts, per-cell event counts and
binary64 times.  The full 256-tissue batch is checked on members of every
cell size, including its largest tissue of 32x32-voxel cells, after a
batched step.
"""
import numpy as np
import pytest

import oracle as O
from paper_1806_10889_gb300 import workloads as W
from tests._util import orc_desc, orc_model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1806_10889_gb300.batching import Batch  # noqa: E402
from paper_1806_10889_gb300.tissue import Tissue  # noqa: E402


def _bits(x):
    return np.asarray(x, dtype=np.float64).view(np.uint64)


def _same(g, counts, ne, tl, ctx):
    got = g.read_counts()
    if not np.array_equal(got, counts):
        bad = np.flatnonzero(got != counts)
        raise AssertionError(f"{ctx}: counts differ at {bad.size} ints, first cell "
                             f"{bad[0] // (3 * g.spec.V)}")
    gne, gtl = g.read_stats()
    assert np.array_equal(gne, ne), f"{ctx}: event counts differ"
    assert np.array_equal(_bits(gtl), _bits(tl)), f"{ctx}: event times differ"


def test_medium_tissue_after_200_steps_matches_oracle():
    """64x64 cells of 16x16 voxels, dt 0.1: 200 GPU steps (20 time units, the
    benchmark's burn-in), then 2 more steps on the GPU and in the oracle."""
    run = W.medium(0.1)
    spec = run.tissue
    g = Tissue(spec)
    g.step(run.dt, 200)
    state, k0 = g.read_counts(), g.get_step()
    g.close()
    assert k0 == 200
    # the burn-in reached the working regime: far above the initial mean of 5
    per_voxel = state.reshape(spec.cells, 3, spec.V).mean(axis=(0, 2))
    assert per_voxel[0] > 40 and per_voxel[1] > 20, per_voxel
    resumed = Tissue(spec)
    resumed.write_counts(state, step_index=k0)
    d, m = orc_desc(spec), orc_model(spec)
    ref = state.copy()
    for k in range(2):
        ne, tl = O.step(d, m, ref, k0 + k, 1, run.dt)
        resumed.step(run.dt, 1)
        _same(resumed, ref, ne, tl, f"medium step {k0 + k}")
    resumed.close()


def _batch_sample(runs):
    """Members of every cell size: for 8x8 and 16x16 voxels the tissue nearest
    256 cells, for 32x32 voxels the largest tissue and the one nearest 256."""
    pick = set()
    for n in (8, 16, 32):
        idx = [i for i, r in enumerate(runs) if r.tissue.n == n]
        pick.add(min(idx, key=lambda i: (abs(runs[i].tissue.cells - 256), i)))
        if n == 32:
            pick.add(max(idx, key=lambda i: (runs[i].tissue.cells, -i)))
    return sorted(pick)


def test_full_batch_members_after_burn_in_match_oracle():
    """The 256-tissue uneven batch (369,574 cells) advanced 30 batched steps
    (3 time units); then one more batched step, checked for sampled members
    against the oracle from the members' burned-in state."""
    runs = W.batch()
    dt = runs[0].dt
    members = [Tissue(r.tissue) for r in runs]
    b = Batch(members)
    b.step(dt, 30)
    b.sync()
    sample = _batch_sample(runs)
    assert {runs[i].tissue.n for i in sample} == {8, 16, 32}
    assert max(runs[i].tissue.cells for i in sample if runs[i].tissue.n == 32) == \
        max(r.tissue.cells for r in runs if r.tissue.n == 32)
    start = {i: members[i].read_counts() for i in sample}
    k0 = members[0].get_step()
    assert k0 == 30
    b.step(dt, 1)
    b.sync()
    for i in sample:
        spec = runs[i].tissue
        ref = start[i].copy()
        ne, tl = O.step(orc_desc(spec), orc_model(spec), ref, k0, 1, dt)
        _same(members[i], ref, ne, tl, f"batch member {i} ({spec.width}x{spec.height} cells of "
                                       f"{spec.n}x{spec.n} voxels) step {k0}")
    b.close()
    for m in members:
        m.close()


def _block_reference(d, m, state, c, step0, dt, n_steps):
    """Oracle counts of cell c after steps step0 .. step0 + n_steps - 1 of a
    tissue too large for the whole oracle, from the GPU's state at step0: a
    face carries influence one cell per phase along its axis, so simulating
    the block of Chebyshev radius n_steps around c leaves c exact.  Returns
    c's counts and its chi statistics of the last step."""
    V, Wd, Hd = d.V, d.width, d.height
    cx, cy = c % Wd, c // Wd
    xs = [x for x in range(cx - n_steps, cx + n_steps + 1) if 0 <= x < Wd]
    ys = [y for y in range(cy - n_steps, cy + n_steps + 1) if 0 <= y < Hd]
    counts = np.zeros(d.cells * 3 * V, dtype=np.int32)
    for y in ys:
        for x in xs:
            b = (y * Wd + x) * 3 * V
            counts[b:b + 3 * V] = state[b:b + 3 * V]
    stats = None
    for k in range(step0, step0 + n_steps):
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
    return counts[c * 3 * V:(c + 1) * 3 * V].copy(), stats


def test_large_tissue_after_burn_in_sampled_cells_match_oracle():
    """256x256 cells of 32x32 voxels (16-bit counts in shared memory) after 2
    time units, the state the benchmark's large leg times from; 2 more steps,
    sampled cells (corners, edges, interior) checked against the oracle on
    the neighbourhood that can influence them."""
    run = W.large()
    spec = run.tissue
    d, m = orc_desc(spec), orc_model(spec)
    g = Tissue(spec)  # default launch shape, as the benchmark uses
    g.step(run.dt, 20)
    state, k0 = g.read_counts(), g.get_step()
    g.step(run.dt, 2)
    got = g.read_counts()
    gne, gtl = g.read_stats()
    g.close()
    Wd, V = spec.width, spec.V
    rng = np.random.default_rng(101)
    samples = [0, Wd - 1, Wd * (Wd - 1), Wd * Wd - 1, Wd * 100 + 3] + \
              [int(x) for x in rng.integers(0, spec.cells, size=5)]
    for c in samples:
        ref, (ne, tl) = _block_reference(d, m, state, c, k0, run.dt, 2)
        assert gne[0, c] == ne and _bits(gtl[0, c]) == _bits(tl), c
        assert np.array_equal(got[c * 3 * V:(c + 1) * 3 * V], ref), c
