"""GPU <-> oracle parity for the Menger-sponge start and the mixed sweep cycle."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ising():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2305_12161_gb300 import ising as m
    return m


@pytest.mark.parametrize("L,k", [(8, 1), (32, 2), (32, 3), (64, 0), (64, 2), (128, 3), (256, 4)])
@pytest.mark.parametrize("form", [0, 1])
def test_menger_start_and_quench(ising, L, k, form):
    if form == 1 and L > 128:
        pytest.skip("plain form covered at smaller L")
    R, seed = 2, 13
    with ising.Ising(L, replicas=R, seed=seed, form=form) as q:
        q.sweep(3)
        q.init_menger(k)
        assert q.t == 0
        for r in range(R):
            assert np.array_equal(q.get_spins(r), oracle.init_menger(L, seed, k, replica=r)), (r, "start")
        q.sweep(4)
        rec = q.measure()
        for r in range(R):
            s = oracle.init_menger(L, seed, k, replica=r)
            oracle.sweeps(s, 0, 4, seed + r)
            assert np.array_equal(q.get_spins(r), s), (r, "after 4 MCS")
            assert np.array_equal(rec[r], oracle.record(s, 4))


@pytest.mark.parametrize("variant,L,depth", [(1, 16, 0), (1, 64, 0), (3, 256, 0), (4, 256, 0), (2, 256, 0),
                                             (5, 256, 0), (5, 256, 11), (5, 256, 1), (5, 256, 9), (5, 512, 11), (5, 512, 27)])
def test_mixed_cycle_vs_oracle(ising, variant, L, depth):
    R, seed = 3, 21
    with ising.Ising(L, replicas=R, seed=seed, variant=variant, depth=depth, cycle=ising.CYCLE_MIXED) as q:
        q.sweep(5)
        rec = q.measure()
        for r in range(R):
            s = oracle.init(L, seed, r)
            oracle.sweeps_mixed(s, 0, 5, seed + r)
            assert np.array_equal(q.get_spins(r), s), r
            assert np.array_equal(rec[r], oracle.record(s, 5))


def test_mixed_cycle_plain_form_and_difference_from_01(ising):
    L, seed = 64, 30
    with ising.Ising(L, replicas=2, seed=seed, form=ising.FORM_PLAIN, cycle=ising.CYCLE_MIXED) as q:
        q.sweep(6)
        for r in range(2):
            s = oracle.init(L, seed, r)
            oracle.sweeps_mixed(s, 0, 6, seed + r)
            assert np.array_equal(q.get_spins(r), s)
        mixed = q.get_spins(0)
    with ising.Ising(L, replicas=1, seed=seed) as q01:
        q01.sweep(6)
        assert not np.array_equal(q01.get_spins(0), mixed)


def test_batch_rejects_mixed_cycle(ising):
    import ctypes
    h = ctypes.c_void_p()
    o = ising.ising_opts()
    ising.lib().ising_default_opts(ctypes.byref(o))
    o.cycle = ising.CYCLE_MIXED
    Ls = (ctypes.c_int * 1)(64)
    Rs = (ctypes.c_int * 1)(1)
    Ss = (ctypes.c_uint64 * 1)(1)
    st = ising.lib().ising_batch_create(ctypes.byref(h), 1, ctypes.cast(Ls, ctypes.c_void_p),
                                        ctypes.cast(Rs, ctypes.c_void_p), ctypes.cast(Ss, ctypes.c_void_p),
                                        ctypes.byref(o))
    assert st == ising.ISING_EINVAL
