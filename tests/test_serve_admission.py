"""Admission of the serving loop by HBM footprint (no GPU): the footprint comes from the
library's own accounting, which includes the tensor-core correlation scratch, and the
admitted requests never exceed the budget or the slots."""
import numpy as np
import pytest

from paper_2305_12161_gb300 import ising, serve


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2305_12161_gb300 import _build
    _build.build()
    ising.lib()


def test_footprint_includes_the_correlation_scratch():
    K = 12
    for L, R in ((64, 4), (256, 2), (512, 1), (1024, 3)):
        fp = serve.footprint_bytes(L, R, K)
        own = K * R * (ising.ising_record_len(L) * 8 + 32)
        assert fp == ising.ising_footprint_bytes(L, R) + own
        packed = R * L**3 // 8
        if L >= 512:  # 2 L^3 bytes of e4m3 operands once the first measurement runs
            assert fp >= packed + 2 * L**3
        else:
            assert fp < 2 * packed + own + 4096
    with pytest.raises(ValueError):
        serve.footprint_bytes(96, 1, K)


def test_budget_that_fits_the_lattices_but_not_the_scratch_serialises():
    reqs = [serve.Request(id=i, L=512, t_max=10, replicas=1, seed=i, K=3) for i in range(3)]
    fp = serve.footprint_bytes(512, 1, 3)
    lattice_only = 512**3 // 8
    budget = fp + 2 * lattice_only  # room for all three lattices, but one scratch only
    adm, keep, used = serve.admit(reqs, 0, 0.0, budget, 16, lambda r: serve.footprint_bytes(r.L, r.replicas, r.K))
    assert [r.id for r in adm] == [0] and [r.id for r in keep] == [1, 2] and used == fp
    # once the first retires its bytes the next is admitted
    adm, keep, used = serve.admit(keep, 0, used - fp, budget, 16, lambda r: serve.footprint_bytes(r.L, r.replicas, r.K))
    assert [r.id for r in adm] == [1] and [r.id for r in keep] == [2]


def test_admitted_sum_stays_within_budget_and_slots():
    rng = np.random.default_rng(7)
    Ls = [64, 128, 256, 512, 1024]
    for trial in range(200):
        reqs = [serve.Request(id=i, L=int(rng.choice(Ls)), t_max=100, replicas=int(rng.integers(1, 17)), seed=i,
                              K=12) for i in range(int(rng.integers(1, 30)))]
        fps = {r.id: serve.footprint_bytes(r.L, r.replicas, r.K) for r in reqs}
        budget = float(rng.uniform(1e7, 4e10))
        slots = int(rng.integers(1, 17))
        n_active = int(rng.integers(0, slots + 1))
        used0 = float(rng.uniform(0, budget))
        adm, keep, used = serve.admit(reqs, n_active, used0, budget, slots, lambda r: fps[r.id])
        assert used <= budget
        assert used == pytest.approx(used0 + sum(fps[r.id] for r in adm))
        assert n_active + len(adm) <= slots
        assert sorted(r.id for r in adm + keep) == [r.id for r in reqs]
        # nothing kept could have been admitted at the end (greedy in arrival order)
        if n_active + len(adm) < slots:
            assert all(used + fps[r.id] > budget for r in keep)


def test_options_are_kept_per_request_shape():
    srv = serve.QuenchServer(tune=False, pdl=0)
    a = srv.options_for(256, 3)
    assert a == {"pdl": 0}
    assert srv.options_for(256, 3) is a  # computed once per shape
    assert srv.options_for(256, 4) is not a
    assert set(srv.opts) == {(256, 3), (256, 4)}
    req = serve.Request(id=0, L=256, t_max=10, replicas=3, seed=1, K=4)
    # the launch order of the sweep kernels does not change the device footprint
    assert srv.footprint(req) == serve.footprint_bytes(256, 3, 4) == serve.footprint_bytes(256, 3, 4, pdl=1)
