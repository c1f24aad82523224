"""Serving loop: requests that overlap on the device give the same result as alone."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serve():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2305_12161_gb300 import serve as m
    return m


def test_mix_equals_alone_and_admission_respects_budget(serve):
    reqs = [serve.Request(id=0, L=64, t_max=300, replicas=3, seed=11, arrival_s=0.0, K=6),
            serve.Request(id=1, L=128, t_max=120, replicas=2, seed=22, arrival_s=0.0, K=5),
            serve.Request(id=2, L=256, t_max=80, replicas=1, seed=33, arrival_s=0.01, K=4),
            serve.Request(id=3, L=64, t_max=50, replicas=16, seed=44, arrival_s=0.02, K=5),
            serve.Request(id=4, L=512, t_max=20, replicas=1, seed=55, arrival_s=0.03, K=3)]
    # a budget that holds only some requests at once forces queueing on memory (footprints
    # with the kernels the server's autotuner picks for each size)
    srv = serve.QuenchServer(budget_bytes=0, max_slots=3, quantum_mcs=16)
    srv.budget = srv.footprint(reqs[4]) + srv.footprint(reqs[2]) + 1
    results = {r.request.id: r for r in srv.run(reqs)}
    assert sorted(results) == [0, 1, 2, 3, 4]
    assert srv.used == 0
    for req in reqs:
        alone = serve.run_alone(req)
        got = results[req.id]
        assert got.times == alone.times
        assert np.array_equal(got.records, alone.records), req.id
        np.testing.assert_allclose(got.derived, alone.derived, rtol=1e-12, atol=0, equal_nan=True)
        assert got.records[-1, 0, 0] == req.t_max
    s = srv.summary()
    assert s["requests"] == 5 and s["p99_s"] >= s["p50_s"] > 0 and s["updates_per_ns"] > 0


def test_oversized_request_rejected(serve):
    srv = serve.QuenchServer(budget_bytes=1e6)
    with pytest.raises(ValueError):
        srv.submit(serve.Request(id=0, L=256, t_max=10, replicas=1, seed=1))


def test_correlation_scratch_forces_queueing(serve):
    # both L = 512 lattices fit the budget, but only one tensor-core correlation scratch
    # (2 x 512^3 bytes) does: the second request waits until the first has retired
    reqs = [serve.Request(id=i, L=512, t_max=30, replicas=1, seed=70 + i, arrival_s=0.0, K=3) for i in range(2)]
    srv = serve.QuenchServer(budget_bytes=0, max_slots=4, quantum_mcs=8)
    fp = srv.footprint(reqs[0])
    from paper_2305_12161_gb300 import ising
    no_scratch = ising.ising_footprint_bytes(512, 1, corr=ising.CORR_POPCOUNT, **srv.options_for(512))
    assert no_scratch + 2 * 512**3 <= fp
    srv.budget = fp + no_scratch  # the second request's lattices fit, its scratch does not
    res = {r.request.id: r for r in srv.run(reqs)}
    first, second = sorted(res.values(), key=lambda r: r.admitted_s)
    assert second.admitted_s >= first.finished_s
    assert srv.used == 0
    for r in res.values():
        alone = serve.run_alone(r.request)
        assert np.array_equal(r.records, alone.records)
