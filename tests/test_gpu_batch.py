"""Batched stepping: many tissues of different sizes and models advance in one
persistent launch per step (captured in a CUDA graph) and every member ends
bit-identical to the oracle and to stepping it alone."""
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


def _bits(x):
    return np.asarray(x, dtype=np.float64).view(np.uint64)


MIX = [TissueSpec(3, 2, 8, seed=3, tissue_id=0).with_model(kD=7.5),
       TissueSpec(5, 4, 16, seed=3, tissue_id=1).with_model(kD=12.0, k_bind=0.05),
       TissueSpec(2, 2, 32, seed=3, tissue_id=2),
       TissueSpec(1, 1, 8, seed=3, tissue_id=3),
       TissueSpec(4, 1, 10, seed=9, tissue_id=4).with_model(k_in=0.01, k_off=0.3),
       TissueSpec(2, 3, 16, seed=3, tissue_id=5).with_model(kD=19.0)]


@pytest.mark.parametrize("steps_per_graph,overlap", [(1, True), (2, True), (1, False)])
def test_batch_matches_oracle_per_member(steps_per_graph, overlap):
    """Both with the cell-size classes overlapped (the default) and with
    them one after another."""
    members = [T.Tissue(s) for s in MIX]
    b = Batch(members)
    b.set_schedule(steps_per_graph)
    b.set_overlap(overlap)
    assert b.info() == (len(MIX), 4, sum(s.cells for s in MIX))
    ref = [O.init_counts(orc_desc(s)) for s in MIX]
    dt = 0.1
    for k in range(3):
        b.step(dt, 1)
        b.sync()
        for i, s in enumerate(MIX):
            ne, tl = O.step(orc_desc(s), orc_model(s), ref[i], k, 1, dt)
            assert np.array_equal(members[i].read_counts(), ref[i]), (k, i)
            gne, gtl = members[i].read_stats()
            assert np.array_equal(gne, ne) and np.array_equal(_bits(gtl), _bits(tl)), (k, i)
    assert all(m.get_step() == 3 for m in members)
    b.close()
    for m in members:
        m.close()


def test_batch_class_launch_shapes_give_the_same_bits():
    results = []
    for lanes, wpb, layout in ((16, 4, 0), (32, 2, 0), (16, 1, 0), (32, 8, 0), (16, 4, 1),
                               (32, 2, 1)):
        members = [T.Tissue(s) for s in MIX]
        b = Batch(members)
        for V in {s.V for s in MIX}:
            if layout == 1 and V > lanes * lanes:
                continue
            b.set_class_launch(V, lanes, wpb, layout)
        b.step(0.2, 4)
        b.sync()
        results.append([m.read_counts() for m in members])
        b.close()
        for m in members:
            m.close()
    for r in results[1:]:
        assert all(np.array_equal(a, c) for a, c in zip(results[0], r))


def test_batch_workload_members_same_alone_and_in_the_mix():
    """The benchmark's uneven batch (side 2..64, n in {8,16,32}, kD per tissue):
    sampled members stepped alone reproduce their in-batch result exactly."""
    runs = W.batch()
    members = [T.Tissue(r.tissue) for r in runs]
    b = Batch(members)
    b.step(0.1, 2)
    b.sync()
    for i in (0, 7, 100, 255):
        alone = T.Tissue(runs[i].tissue)
        alone.step(0.1, 2)
        assert np.array_equal(alone.read_counts(), members[i].read_counts()), i
        ne_a, tl_a = alone.read_stats()
        ne_b, tl_b = members[i].read_stats()
        assert np.array_equal(ne_a, ne_b) and np.array_equal(_bits(tl_a), _bits(tl_b)), i
        alone.close()
    b.close()
    for m in members:
        m.close()


def test_batch_rejects_bad_input():
    a = T.Tissue(MIX[0])
    with pytest.raises(T.TissueError):
        Batch([a, a])
    b = Batch([a])
    with pytest.raises(T.TissueError):
        b.set_class_launch(64, 16, 99, 0)
    with pytest.raises(T.TissueError):
        b.set_class_launch(1024, 16, 4, 0)  # no such class
    with pytest.raises(T.TissueError):
        b.set_class_launch(64, 4, 2, 1)  # lanes must be 16 or 32
    b.close()
    a.close()


def test_batch_timing_and_class_info_change_no_result():
    """Per-class timing (event-record nodes in the captured graph) reports
    positive times that add up within the step, and the trajectory is the
    same with timing on and off."""
    outs = []
    for timing in (False, True):
        members = [T.Tissue(s) for s in MIX]
        b = Batch(members)
        cls = b.classes()
        assert [c["V"] for c in cls] == [1024, 256, 100, 64]
        assert sum(c["cells"] for c in cls) == sum(s.cells for s in MIX)
        for c in cls:
            assert c["lanes_per_cell"] in (8, 16, 32) and c["smem_layout"] in (0, 1)
        if timing:
            b.set_timing(True)
            with pytest.raises(T.TissueError):
                b.read_timing()  # no timed step yet
        for k in range(4):
            if timing:
                b.set_overlap(k < 2)  # overlapped classes, then one after another
            b.step(0.1, 1)
            if timing:
                step_ms, chi_ms, wm_ms, class_ms = b.read_timing()
                assert step_ms > 0 and wm_ms >= 0 and len(class_ms) == len(cls)
                assert all(x > 0 for x in class_ms)
                assert chi_ms <= step_ms * 1.001 and max(class_ms) <= chi_ms * 1.001
                if k >= 2:  # one after another: the classes add up to the chi phase
                    assert abs(sum(class_ms) + wm_ms - chi_ms) <= 0.01 * chi_ms + 0.05
        b.sync()
        outs.append([m.read_counts() for m in members])
        if timing:
            b.set_timing(False)
            with pytest.raises(T.TissueError):
                b.read_timing()
        b.close()
        for m in members:
            m.close()
    assert all(np.array_equal(x, y) for x, y in zip(*outs))


def test_batch_state_io_matches_per_member_io():
    """tissue_batch_write_counts / read_counts: the same states and step
    indices as the per-member calls, a count out of range rejected, and the
    batch steps on from written states as the members would alone."""
    members = [T.Tissue(s) for s in MIX]
    b = Batch(members)
    b.step(0.1, 2)
    b.sync()
    hosts = [torch.empty(s.state_ints, dtype=torch.int32, pin_memory=True) for s in MIX]
    b.read_counts(hosts)
    for h, m in zip(hosts, members):
        assert np.array_equal(h.numpy(), m.read_counts())
    # write back perturbed states at a new step index; step on both ways
    rng = np.random.default_rng(4)
    for h in hosts:
        h.copy_(torch.from_numpy(rng.integers(0, 40, size=h.numel(), dtype=np.int32)))
    alone = [T.Tissue(s) for s in MIX]
    for t, h in zip(alone, hosts):
        t.write_counts(h.numpy(), step_index=11)
    b.write_counts(hosts, step_index=11)
    assert all(m.get_step() == 11 for m in members)
    b.step(0.1, 2)
    b.read_counts(hosts)
    for t, h in zip(alone, hosts):
        t.step(0.1, 2)
        assert np.array_equal(t.read_counts(), h.numpy())
        t.close()
    # a negative count and one above TISSUE_COUNT_MAX are rejected
    for bad in (-1, 2 ** 30):
        h0 = hosts[0].clone().pin_memory()
        h0[5] = bad
        with pytest.raises(T.TissueError) as e:
            b.write_counts([h0] + hosts[1:], step_index=[0] * len(MIX))
        assert e.value.code == T.E_ARG
    b.close()
    for m in members:
        m.close()


def test_overlap_tuning_picks_a_mode_and_keeps_the_trajectory():
    """autotune.tune_overlap steps the batch 4 times, alternating overlapped
    and sequential classes, and leaves the faster set; the members still
    match the oracle bit for bit."""
    from paper_1806_10889_gb300 import autotune
    members = [T.Tissue(s) for s in MIX]
    b = Batch(members)
    dt = 0.1
    res = autotune.tune_overlap(b, dt)
    assert set(res["ms"]) == {"overlapped", "sequential"}
    assert all(v > 0 for v in res["ms"].values())
    assert b.overlap == res["overlap"] and b.timing is False
    assert all(m.get_step() == 4 for m in members)
    b.step(dt, 1)
    b.sync()
    for i, s in enumerate(MIX):
        ref = O.init_counts(orc_desc(s))
        ne, tl = O.step(orc_desc(s), orc_model(s), ref, 0, 5, dt)
        assert np.array_equal(members[i].read_counts(), ref), i
        gne, gtl = members[i].read_stats()
        assert np.array_equal(gne, ne) and np.array_equal(_bits(gtl), _bits(tl)), i
    b.close()
    for m in members:
        m.close()
