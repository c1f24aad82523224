"""Parity at the full workload sizes, where the oracle cannot replay whole runs.

* 8 replicas of L=256 (seeds 1..8), 10^4 MCS, 40 log-spaced times: the first times are
  replayed by the oracle outright for every replica; at EVERY recorded time the oracle
  recounts the whole record (M, B and all 3 x 129 D_a(r)) from every replica's GPU state;
  at four spread times the GPU state one MCS earlier is handed to the oracle, which
  advances it one MCS, and all spins must agree.
* One L=2048 lattice in the launch configuration the benchmark times (autotuned sweep
  kernel, tensor-core correlation): the whole initial state against the oracle's
  T = infinity start; at t = 0, 3, 2000 and 10^4 the whole record of the tensor-core path against
  the bit-count path (a different algorithm, oracle-pinned in full at L <= 256) on the
  same state, M and B recounted by the oracle, and D_a(r) recounted by the oracle at the
  tile edges of the tensor-core path (tiles of 128 positions, super-tiles of 256); at
  t = 3 (dense ties), t = 2000 and t = 10^4 (where the benchmark's second leg starts) the
  whole state handed to the oracle, advanced one MCS there, and compared with the GPU's next
  state site by site (8.6e9 spins).
"""
import numpy as np
import pytest

import oracle
from paper_2305_12161_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ising():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2305_12161_gb300 import ising as m
    return m


def _rec_D(rec, L):
    return np.asarray(rec[3:]).reshape(3, L // 2 + 1)


def test_L256_eight_replicas_every_recorded_time(ising):
    L, R, seed = 256, 8, 1
    times = inputs.log_schedule(10_000, 40)
    handoff = {5, 17, 29, 39}  # indices into times: one-MCS oracle advance there
    n_early = 6                # times[:n_early] replayed whole by the oracle
    early = [oracle.run(L, seed, r, times[:n_early])[0] for r in range(R)]
    with ising.Ising(L, replicas=R, seed=seed) as q:
        rec = q.measure()
        for r in range(R):
            s = q.get_spins(r)
            assert np.array_equal(s, oracle.init(L, seed, r)), r
            assert np.array_equal(oracle.record(s, 0), rec[r]), r
            assert np.array_equal(early[r][0], rec[r]), r
        t = 0
        for k, tk in enumerate(times):
            prev = None
            if k in handoff:
                q.sweep(tk - 1 - t)
                prev = [q.get_spins(r) for r in range(R)]
                q.sweep(1)
            else:
                q.sweep(tk - t)
            t = tk
            rec = q.measure()
            assert np.all(rec[:, 0] == tk)
            for r in range(R):
                s = q.get_spins(r)
                assert np.array_equal(oracle.record(s, tk), rec[r]), (r, tk)
                if k < n_early:
                    assert np.array_equal(early[r][k + 1], rec[r]), (r, tk)
                if prev is not None:
                    oracle.sweeps(prev[r], tk - 1, 1, seed + r)
                    assert np.array_equal(prev[r], s), (r, tk)
            del prev


# Distances at which the tensor-core path's tiling changes: 128-position tiles, 256-position
# super-tiles, the half-lattice end; plus the first few and a spread of seeded interior ones.
EDGE_LAGS = [0, 1, 2, 3, 127, 128, 129, 255, 256, 257, 383, 384, 385, 511, 512, 513, 767, 768, 769, 1023, 1024]


def _lags_for(t_hand):
    if t_hand != 2000:
        return EDGE_LAGS
    extra = np.random.default_rng(2048).choice(np.arange(4, 1023), size=24, replace=False)
    return sorted(set(EDGE_LAGS) | set(int(v) for v in extra))


def _check_record(ising, q, qp, A, t_hand, L):
    """Tensor-core record of q's state == bit-count record of the same state (qp), and
    oracle recounts of M, B and D_a(r) at the lags of _lags_for."""
    rec = q.measure()[0]
    qp.set_packed(q.get_packed(0))
    qp.t = q.t
    recp = qp.measure()[0]
    assert np.array_equal(rec, recp), (t_hand, np.flatnonzero(rec != recp)[:8])
    M, B = oracle.magnetisation_bonds(A)
    assert (int(rec[0]), int(rec[1]), int(rec[2])) == (t_hand, M, B), t_hand
    lags = _lags_for(t_hand)
    D = _rec_D(rec, L)
    want = oracle.corr_lags(A, lags)
    for j, r in enumerate(lags):
        assert list(D[:, r]) == list(want[j]), (t_hand, r)


def test_L2048_bench_configuration_full(ising):
    L, S = 2048, 1
    tuned = ising.ising_tune_sweep(L, 1, probe_mcs=8)
    kw = dict(variant=tuned["variant"], tile_y=tuned["tile_y"], tile_z=tuned["tile_z"], depth=tuned["depth"])
    with ising.Ising(L, replicas=1, seed=S, **kw) as q, \
            ising.Ising(L, replicas=1, seed=S, corr=ising.CORR_POPCOUNT) as qp:
        # whole initial state against the oracle's T = infinity start
        A = q.get_spins(0)
        assert np.array_equal(A, oracle.init(L, S, 0))
        _check_record(ising, q, qp, A, 0, L)
        del A
        for t_hand in (3, 2000, 10_000):
            q.sweep(t_hand - q.t)
            A = q.get_spins(0)
            _check_record(ising, q, qp, A, t_hand, L)
            q.sweep(1)
            B = q.get_spins(0)
            oracle.sweeps(A, t_hand, 1, S)
            eq = A == B
            assert eq.all(), (t_hand, int((~eq).sum()))
            del A, B, eq
