"""Parity at the full workload sizes, where the oracle cannot replay whole runs.

* 8 replicas of L=256 (seeds 1..8), 10^4 MCS, 40 log-spaced times: the first times are
  replayed by the oracle outright; at late times the GPU state is handed to the oracle,
  which recounts the record and advances one MCS.
* One L=2048 lattice in the launch configuration the benchmark times: sampled sites of
  the initial state against the addressed Philox bits, sampled sites of two sweeps (one
  dense-tie, one late) against the oracle's site update, and M, B and sampled D_a(r)
  recounted by the oracle from the full GPU state.
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


def test_L256_eight_replicas_ten_thousand_mcs(ising):
    L, R, seed = 256, 8, 1
    times = inputs.log_schedule(10_000, 40)
    recs = []
    with ising.Ising(L, replicas=R, seed=seed) as q:
        recs.append(q.measure())
        t = 0
        for tk in times:
            q.sweep(tk - t)
            t = tk
            recs.append(q.measure())
    recs = np.stack(recs, axis=1)  # [R, 41, RL]
    # early times replayed whole by the oracle (replicas 0 and 7)
    for r in (0, 7):
        want, _ = oracle.run(L, seed, r, times[:4])
        assert np.array_equal(recs[r, :5], want), r
    # late times: hand the GPU state at t_k - 1 to the oracle, advance one MCS
    for r, k in ((0, 25), (3, 39), (7, 39)):
        tk = times[k]
        with ising.Ising(L, replicas=1, seed=seed + r) as q:
            q.sweep(tk - 1)
            s = q.get_spins(0)
            q.sweep(1)
            gpu_next = q.get_spins(0)
        oracle.sweeps(s, tk - 1, 1, seed + r)
        assert np.array_equal(s, gpu_next), (r, tk)
        assert np.array_equal(oracle.record(s, tk), recs[r, k + 1]), (r, tk)


def _sample_sites(L, n, q, rng):
    z = rng.integers(0, L, n)
    y = rng.integers(0, L, n)
    x = 2 * rng.integers(0, L // 2, n) + ((y + z + q) & 1)
    return (x + L * (y + L * z)).astype(np.int64), x, y, z


def _check_sweep(A, B, L, t, S, rng, n=200_000):
    """B must be one MCS of A at sweep index t: red sites from A's neighbours, blue
    sites from the red-updated neighbours (B) and their own old value (A)."""
    Af, Bf = A.reshape(-1), B.reshape(-1)
    i0, *_ = _sample_sites(L, n, 0, rng)
    i0 = np.unique(i0)
    assert np.array_equal(oracle.update_sites(A, 0, t, S, i0), Bf[i0])
    i1, *_ = _sample_sites(L, n, 1, rng)
    i1 = np.unique(i1)
    got = Bf[i1].copy()
    Bf[i1] = Af[i1]  # old values at the sampled blue sites; their neighbours are red
    try:
        assert np.array_equal(oracle.update_sites(B, 1, t, S, i1), got)
    finally:
        Bf[i1] = got


def test_L2048_bench_configuration_sampled(ising):
    L, S = 2048, 1
    rng = np.random.default_rng(2048)
    with ising.Ising(L, replicas=1, seed=S) as q:
        # initial state: sampled sites against the addressed Philox bit (phase 2 + q)
        A = q.get_spins(0)
        for qq in (0, 1):
            idx, x, y, z = _sample_sites(L, 2000, qq, rng)
            h = (x >> 1) + (L // 2) * (y + L * z)
            want = np.array([1 if oracle.rng_bit(S, 0, 2 + qq, int(hh)) else -1 for hh in h], dtype=np.int8)
            assert np.array_equal(A.reshape(-1)[idx], want)
        for t_hand in (3, 2000):
            q.sweep(t_hand - q.t)
            A = q.get_spins(0)
            rec = q.measure()[0]
            q.sweep(1)
            B = q.get_spins(0)
            _check_sweep(A, B, L, t_hand, S, rng)
            # observables of the handed-over state
            M, Bnd = oracle.magnetisation_bonds(A)
            assert (rec[1], rec[2]) == (M, Bnd), t_hand
            H = L // 2
            for r in (1, 2, 17, 1024):
                D = oracle.corr_lag(A, r)
                assert [rec[3 + r], rec[3 + (H + 1) + r], rec[3 + 2 * (H + 1) + r]] == list(D), (t_hand, r)
            del A, B
