"""Host logic: the seeded workload generators are deterministic and in range."""
import math

from paper_1806_10889_gb300 import workloads as W


def test_fixed_configs():
    t = W.tiny()
    assert (t.tissue.width, t.tissue.height, t.tissue.n, t.dt, t.n_steps) == (2, 2, 8, 0.1, 100)
    for dt, steps in ((0.01, 5000), (0.1, 500), (1.0, 50)):
        r = W.medium(dt)
        assert (r.tissue.cells, r.tissue.V, r.n_steps) == (4096, 256, steps)
    L = W.large()
    assert L.tissue.cells == 65536 and L.tissue.V == 1024
    assert L.tissue.state_ints * 4 == 805306368  # 0.8 GB of int32 state


def test_batch_mix_deterministic_and_in_range():
    a, b = W.batch(), W.batch()
    assert a == b and len(a) == 256
    assert all(2 <= r.tissue.width <= 64 and r.tissue.width == r.tissue.height for r in a)
    assert {r.tissue.n for r in a} == {8, 16, 32}
    assert all(5.0 <= r.tissue.model["kD"] <= 20.0 for r in a)
    assert [r.tissue.tissue_id for r in a] == list(range(256))


def test_serving_arrivals():
    reqs = W.serving()
    assert len(reqs) == 500
    gaps = [b.arrival_s - a.arrival_s for a, b in zip(reqs, reqs[1:])]
    assert all(g > 0 for g in gaps)
    assert abs(sum(gaps) / len(gaps) - 0.02) < 0.004
    assert all(1 <= r.replicas <= 64 and 2 <= r.side <= 128 and r.n == 16 for r in reqs)
    med = sorted(r.side for r in reqs)[250]
    assert 12 <= med <= 20
    specs = reqs[7].replica_specs()
    assert all(s.seed == 7 for s in specs) and [s.tissue_id for s in specs] == list(range(reqs[7].replicas))
