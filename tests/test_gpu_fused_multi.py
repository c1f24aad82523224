"""Whole-sweep kernel with several replicas per launch (variant 5, five copy slots).

Up to 16 replicas of one context share a launch (grid.y = replica, each with its own
Philox key, first sublattice and stores), so a context of many small lattices fills the
GPU.  Every replica must follow exactly its own single-lattice trajectory: compared with
one-replica contexts on the half-sweep kernel (oracle-pinned elsewhere) for every replica,
and with the oracle directly for the replicas at the edges of a launch.  The batched form
runs its streamed classes on this kernel when told to (or when its autotuner picks it), in
pairs of sweeps between two stores with an odd last sweep in place.
"""
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


def _single(ising, L, seed, n, **kw):
    with ising.Ising(L, replicas=1, seed=seed, variant=ising.VARIANT_ZFAST, **kw) as p:
        p.sweep(n)
        return p.get_packed(0), p.measure()[0]


# depth 0 / 16: first tiling, five slots (16: z-blocks fitted); 10 / 26: balanced tiling
@pytest.mark.parametrize("depth", [0, 10, 16, 26])
def test_eighteen_replicas_two_launches_per_sweep(ising, depth):
    L, R, seed, n = 256, 18, 40, 5
    with ising.Ising(L, replicas=R, seed=seed, variant=ising.VARIANT_ZFUSE, tile_z=32, depth=depth) as q:
        l0 = q.launch_count()
        q.sweep(n)
        assert q.launch_count() - l0 == 2 * n  # 16 + 2 replicas per sweep
        rec = q.measure()
        for r in range(R):
            pk, prec = _single(ising, L, seed + r, n)
            assert np.array_equal(q.get_packed(r), pk), r
            assert np.array_equal(rec[r], prec), r
        for r in (15, 16):  # last of the first launch, first of the second
            want, spins = oracle.run(L, seed, r, [n], keep_spins=True)
            assert np.array_equal(q.get_spins(r), spins[-1]), r
            assert np.array_equal(rec[r], want[-1]), r


@pytest.mark.parametrize("rule", [1, 2])
def test_rules_with_replicas_per_launch(ising, rule):
    L, R, seed, n = 256, 3, 70, 4
    with ising.Ising(L, replicas=R, seed=seed, tie=rule, variant=ising.VARIANT_ZFUSE, tile_z=64, depth=26) as q:
        q.sweep(n)
        for r in range(R):
            pk, _ = _single(ising, L, seed + r, n, tie=rule)
            assert np.array_equal(q.get_packed(r), pk), (rule, r)


def test_mixed_cycle_first_sublattice_per_replica(ising):
    # the mixed cycle draws each replica's first sublattice from its own key: replicas of one
    # launch start on different sublattices
    L, R, seed, n = 256, 17, 90, 6
    with ising.Ising(L, replicas=R, seed=seed, variant=ising.VARIANT_ZFUSE, tile_z=32, depth=10,
                     cycle=ising.CYCLE_MIXED) as q:
        q.sweep(n)
        for r in range(R):
            pk, _ = _single(ising, L, seed + r, n, cycle=ising.CYCLE_MIXED)
            assert np.array_equal(q.get_packed(r), pk), r
        s = oracle.init(L, seed, 16)
        oracle.sweeps_mixed(s, 0, n, seed + 16)
        assert np.array_equal(q.get_spins(16), s)


@pytest.mark.parametrize("L,R,depth", [(512, 3, 26), (512, 2, 0), (1024, 2, 10), (2048, 2, 26)])
def test_wider_rows_with_replicas_per_launch(ising, L, R, depth):
    seed, n = 3, 3
    with ising.Ising(L, replicas=R, seed=seed, variant=ising.VARIANT_ZFUSE, tile_z=64, depth=depth) as q:
        q.sweep(n)
        rec = q.measure()
        for r in range(R):
            pk, prec = _single(ising, L, seed + r, n)
            assert np.array_equal(q.get_packed(r), pk), (L, r)
            assert np.array_equal(rec[r], prec), (L, r)


def test_batch_streamed_classes_on_the_fused_kernel(ising):
    classes = [(64, 4, 1), (256, 5, 9), (512, 2, 11)]
    with ising.Batch(classes) as b:
        assert b.class_config(0)["variant"] == -1
        b.set_class_config(1, variant=ising.VARIANT_ZFUSE, tile_z=32, depth=26)
        b.set_class_config(2, variant=ising.VARIANT_ZFUSE, tile_z=64, depth=2)
        assert b.class_config(1) == dict(variant=ising.VARIANT_ZFUSE, tile_y=256, tile_z=32, depth=26)
        with pytest.raises(ising.IsingError) as e:
            b.set_class_config(0, variant=ising.VARIANT_ZFUSE)
        assert e.value.status == ising.ISING_EINVAL
    with ising.Batch(classes) as b:
        b.set_class_config(1, variant=ising.VARIANT_ZFUSE, tile_z=32, depth=26)
        b.set_class_config(2, variant=ising.VARIANT_ZFUSE, tile_z=64, depth=2)
        b.sweep(7)  # odd segment: six sweeps between the stores, the last in place
        b.sweep(4)  # even segment
        rec, _ = b.measure_ex()
        for ci, (L, R, seed) in enumerate(classes):
            with ising.Ising(L, replicas=R, seed=seed) as q:
                q.sweep(11)
                qrec = q.measure()
                for r in range(R):
                    assert np.array_equal(b.get_packed(ci, r), q.get_packed(r)), (L, r)
                    assert np.array_equal(b.record_of(rec, ci, r), qrec[r]), (L, r)
        # graph-captured schedule with odd and even segments, replayed after a re-init
        times = [1, 2, 5, 8]
        b.reinit()
        g1, _ = b.run(times)
        b.reinit()
        g2, _ = b.run(times)
        assert np.array_equal(g1, g2)
        for ci, (L, R, seed) in enumerate(classes):
            with ising.Ising(L, replicas=R, seed=seed) as q:
                t = 0
                for k, tk in enumerate(times):
                    q.sweep(tk - t)
                    t = tk
                    qrec = q.measure()
                    for r in range(R):
                        assert np.array_equal(b.record_of(g1[k], ci, r), qrec[r]), (L, r, tk)


@pytest.mark.parametrize("kw", [dict(variant=3, tile_z=8), dict(variant=5, tile_z=8, depth=18),
                                dict(variant=5, tile_z=32, depth=10)])
def test_plain_stream_order_gives_the_same_trajectory(ising, kw):
    # programmatic dependent launch (the default) and plain stream order: same spins
    L, R, seed, n = 256, 3, 55, 7
    got = {}
    for pdl in (0, 1):
        with ising.Ising(L, replicas=R, seed=seed, pdl=pdl, **kw) as q:
            q.sweep(n)
            got[pdl] = [q.get_packed(r) for r in range(R)]
    for a, b in zip(got[0], got[1]):
        assert np.array_equal(a, b)
    want = oracle.init(L, seed, 2)
    oracle.sweeps(want, 0, n, seed + 2)
    with ising.Ising(L, replicas=1, seed=seed + 2) as q:
        q.set_spins(want, 0)
        assert np.array_equal(got[0][2], q.get_packed(0))
