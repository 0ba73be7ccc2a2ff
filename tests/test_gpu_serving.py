"""Serving: continuous batching under a device-memory budget.  Each request's
result is the same alone and in the mix, bit for bit; the budget is never
exceeded; a request larger than the budget is refused."""
import numpy as np
import pytest

import oracle as O
from paper_1806_10889_gb300.workloads import Request
from tests._util import orc_desc, orc_model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1806_10889_gb300.serving import Server, latency_summary, request_bytes  # noqa: E402

# staggered arrivals (seconds) so later requests join batches already running
REQS = [Request(0, 0.00, 3, 4, 16, 7, 0.1), Request(1, 0.02, 2, 6, 8, 5, 0.1),
        Request(2, 0.04, 4, 3, 16, 9, 0.1), Request(3, 0.05, 1, 5, 32, 4, 0.1),
        Request(4, 0.05, 2, 2, 10, 6, 0.1)]


def test_results_same_alone_and_in_the_mix():
    mix = Server(budget_bytes=1 << 34, chunk_steps=2, keep_counts=True).run(REQS)
    assert all(r.digest for r in mix)
    for req in REQS:
        alone = Server(budget_bytes=1 << 34, chunk_steps=3).run([req])[0]
        assert alone.digest == mix[req.index].digest, req.index
    # and the mix agrees with the oracle for one replica of each request
    for req, res in zip(REQS, mix):
        spec = req.replica_specs()[-1]
        ref = O.init_counts(orc_desc(spec))
        O.step(orc_desc(spec), orc_model(spec), ref, 0, req.n_steps, req.dt)
        assert np.array_equal(res.counts[-1], ref), req.index
    s = latency_summary(mix)
    assert s["served"] == len(REQS) and s["p99_s"] >= s["p50_s"] > 0


def test_budget_admission_and_rejection():
    one = max(request_bytes(r) for r in REQS)
    srv = Server(budget_bytes=one, chunk_steps=2)
    res = srv.run(REQS)
    assert srv.peak_used <= one
    assert all(r.digest and not r.rejected for r in res)
    big = Request(9, 0.0, 64, 40, 16, 2, 0.1)
    srv2 = Server(budget_bytes=request_bytes(big) - 1, chunk_steps=2)
    out = srv2.run([big])
    assert out[0].rejected and latency_summary(out)["served"] == 0


def test_srpt_finishes_small_requests_first_with_the_same_results():
    """With every request arriving at once and a round sized for one
    request, the least remaining work goes first: the small requests finish
    before the large one, and every result equals the lockstep schedule's."""
    reqs = [Request(0, 0.0, 4, 8, 16, 6, 0.1),   # 256 cells
            Request(1, 0.0, 1, 2, 8, 6, 0.1),    # 4 cells
            Request(2, 0.0, 2, 3, 8, 6, 0.1)]    # 18 cells
    srpt = Server(budget_bytes=1 << 34, chunk_steps=2, policy="srpt", fill_cells=1).run(reqs)
    lock = Server(budget_bytes=1 << 34, chunk_steps=2, policy="lockstep").run(reqs)
    assert [r.digest for r in srpt] == [r.digest for r in lock]
    assert srpt[1].done_s < srpt[2].done_s < srpt[0].done_s
    with pytest.raises(ValueError):
        Server(budget_bytes=1, policy="fifo")


def test_cancel_pending_and_active_requests():
    """Cancelling frees the request's memory and leaves every other result
    as it would be alone."""
    reqs = [Request(0, 0.0, 2, 4, 16, 8, 0.1), Request(1, 0.0, 1, 3, 8, 8, 0.1),
            Request(2, 0.0, 1, 2, 8, 8, 0.1)]
    srv = Server(budget_bytes=1 << 34, chunk_steps=2, policy="lockstep")
    srv.cancel(2)  # still pending when the run starts

    def after_round(server, indices):
        if 0 in indices:
            server.cancel(0)  # active: stopped at the next chunk boundary

    res = srv.run(reqs, on_round=after_round)
    assert res[0].cancelled and not res[0].digest
    assert res[2].cancelled and not res[2].digest
    assert not res[1].cancelled and res[1].digest
    alone = Server(budget_bytes=1 << 34, chunk_steps=3).run([reqs[1]])[0]
    assert alone.digest == res[1].digest
    assert srv.used == 0
    s = latency_summary(res)
    assert s["served"] == 1 and s["cancelled"] == 2
