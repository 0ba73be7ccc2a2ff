"""Host logic of the server's scheduling policy (no device needed): which
active requests a round advances."""
import pytest

from paper_1806_10889_gb300.serving import Result, Server, _Active, latency_summary
from paper_1806_10889_gb300.workloads import Request


def _active(index, replicas, side, n_steps, done=0):
    req = Request(index, 0.0, replicas, side, 16, n_steps, 0.1)
    res = Result(index, 0.0)
    res.cells = replicas * side * side
    return _Active(req, res, [], done, 0)


def test_srpt_orders_by_remaining_work_and_fills_the_round():
    big = _active(0, 10, 20, 200)           # 4000 cells x 200 steps
    small = _active(1, 1, 4, 200)           # 16 cells
    half_done = _active(2, 10, 20, 200, 190)  # 4000 cells x 10 steps left
    srv = Server(budget_bytes=1, policy="srpt", fill_cells=100)
    assert [a.req.index for a in srv._choose([big, small, half_done])] == [1, 2]
    srv = Server(budget_bytes=1, policy="srpt", fill_cells=10_000)
    assert [a.req.index for a in srv._choose([big, small, half_done])] == [1, 2, 0]
    srv = Server(budget_bytes=1, policy="srpt", fill_cells=1)
    assert [a.req.index for a in srv._choose([big, small, half_done])] == [1]


def test_lockstep_takes_everything_and_ties_break_by_index():
    a, b = _active(5, 1, 4, 10), _active(3, 1, 4, 10)
    assert Server(budget_bytes=1, policy="lockstep")._choose([a, b]) == [a, b]
    assert [x.req.index for x in Server(budget_bytes=1, fill_cells=1)._choose([a, b])] == [3]
    with pytest.raises(ValueError):
        Server(budget_bytes=1, policy="round-robin")


def test_latency_summary_skips_rejected_and_cancelled():
    rs = [Result(i, 0.0, done_s=float(i + 1)) for i in range(4)]
    rs[1].rejected = True
    rs[2].cancelled = True
    s = latency_summary(rs)
    assert s["served"] == 2 and s["rejected"] == 1 and s["cancelled"] == 1
    assert s["p50_s"] == pytest.approx(2.5)
    assert latency_summary([])["served"] == 0
