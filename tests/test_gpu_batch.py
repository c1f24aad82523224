"""Batched form: one persistent launch per segment over lattices of uneven L.

Every lattice of a batch must follow exactly its single-lattice trajectory (oracle
parity for small L, bit-identical to the single-context kernels for larger L), whatever
the work list looks like (whole-lattice CTAs, slab groups, tuned weights), and the
graph-captured schedule must equal step-by-step sweeps and measurements.  A slab group
that loses a member must end with ISING_ETIMEOUT after its bounded wait, not hang.
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


def test_small_batch_matches_oracle_at_every_time(ising):
    classes = [(16, 3, 11), (64, 2, 21), (128, 1, 31)]
    times = [1, 3, 7, 12]
    with ising.Batch(classes) as b:
        plan = b.plan()
        assert plan["local_ctas"] >= 1 and plan["groups"] >= 1
        recs = [b.measure_ex()[0]]
        t = 0
        for tk in times:
            b.sweep(tk - t)
            t = tk
            recs.append(b.measure_ex()[0])
        for ci, (L, R, seed) in enumerate(classes):
            for r in range(R):
                want, spins = oracle.run(L, seed, r, times, keep_spins=True)
                for k in range(len(times) + 1):
                    assert np.array_equal(b.record_of(recs[k], ci, r), want[k]), (L, r, k)
                # final state, through the packed checkpoint layout
                with ising.Ising(L, replicas=1, seed=seed + r) as q:
                    q.set_spins(spins[-1], 0)
                    assert np.array_equal(b.get_packed(ci, r), q.get_packed(0)), (L, r)


@pytest.mark.parametrize("streamed", [256, 0])
def test_batch_matches_single_contexts_large(ising, streamed):
    classes = [(64, 8, 1), (192, 2, 5), (256, 2, 9), (512, 1, 11)]
    n = 9
    with ising.Batch(classes) as b:
        b.set_streamed(streamed)
        plan = b.plan()
        if streamed:
            assert b.streamed_classes() == 2 and plan["groups"] >= 1
        else:
            assert b.streamed_classes() == 0 and plan["groups"] >= 3
        assert plan["ctas"] <= plan["capacity"]
        b.sweep(n)
        rec, der = b.measure_ex()
        for ci, (L, R, seed) in enumerate(classes):
            with ising.Ising(L, replicas=R, seed=seed) as q:
                q.sweep(n)
                qrec, qder = q.measure_ex()
                for r in range(R):
                    assert np.array_equal(b.get_packed(ci, r), q.get_packed(r)), (L, r)
                    assert np.array_equal(b.record_of(rec, ci, r), qrec[r])
                o = b.offsets[ci][1]
                np.testing.assert_allclose(der[o:o + R], qder, rtol=1e-12, atol=0, equal_nan=True)


def test_graph_schedule_equals_stepwise(ising):
    classes = [(32, 4, 5), (64, 3, 50), (128, 2, 70)]
    times = [1, 2, 4, 8, 15]
    with ising.Batch(classes) as a:
        step = []
        t = 0
        for tk in times:
            a.sweep(tk - t)
            t = tk
            step.append(a.measure_ex(c=0.5))
    with ising.Batch(classes) as b:
        rec, der = b.run(times, c=0.5)
        assert b.t == times[-1]
        for k in range(len(times)):
            assert np.array_equal(rec[k], step[k][0])
            np.testing.assert_allclose(der[k], step[k][1], rtol=1e-12, atol=0, equal_nan=True)
        # replay of the cached graph after a re-init gives the same schedule again
        b.reinit()
        rec2, der2 = b.run(times, c=0.5)
        assert np.array_equal(rec2, rec)


def test_graph_schedule_device_outputs(ising):
    import torch
    classes = [(64, 2, 3), (256, 1, 4)]
    times = [2, 5]
    with ising.Batch(classes) as a:
        want, _ = a.run(times)
    with ising.Batch(classes) as b:
        rec = torch.empty((len(times), b.record_words), dtype=torch.int64, device="cuda")
        der = torch.empty((len(times), b.lattices, 4), dtype=torch.float64, device="cuda")
        b.run(times, rec=rec, derived=der, device=True)
        b.sync()
        assert np.array_equal(rec.cpu().numpy(), want)


def test_tuned_plan_changes_speed_not_results(ising):
    classes = [(64, 16, 2), (128, 4, 40), (256, 1, 60)]
    with ising.Batch(classes) as a:
        a.sweep(6)
        ref = [a.get_packed(ci, r) for ci, (L, R, s) in enumerate(classes) for r in range(R)]
    with ising.Batch(classes) as b:
        w = b.tune(probe_mcs=2)
        assert w > 0
        t_after = b.t
        kern = b.class_config(2)
        b.reinit()
        b.sweep(6)
        got = [b.get_packed(ci, r) for ci, (L, R, s) in enumerate(classes) for r in range(R)]
        # three work-list rounds of 2 MCS, then for the one streamed class two candidates and
        # the streamed classes after and beside the persistent launch, each timed as a warm-up
        # segment of 2 MCS and a timed one of 4
        assert t_after == 6 + 2 * (2 + 4) + 2 * (2 + 4)
        assert kern["variant"] > 0 and b.class_config(0)["variant"] == -1
        for x, y in zip(got, ref):
            assert np.array_equal(x, y)
        for wl in (0.25, 4.0):
            b.set_weights(wl, 1.0)
            b.reinit()
            b.sweep(6)
            got = [b.get_packed(ci, r) for ci, (L, R, s) in enumerate(classes) for r in range(R)]
            for x, y in zip(got, ref):
                assert np.array_equal(x, y)


def test_streamed_classes_beside_the_persistent_launch(ising):
    # the same trajectories whether the streamed classes run after the persistent launch or
    # beside it on their own streams (step by step and as a captured schedule)
    classes = [(64, 6, 3), (128, 2, 30), (256, 3, 60), (512, 1, 90)]
    times = [1, 4, 7, 12]
    out = {}
    for on in (False, True):
        with ising.Batch(classes) as b:
            b.set_overlap(on)
            assert b.overlap == on
            b.sweep(5)
            b.sweep(4)
            rec, _ = b.measure_ex()
            packed = [b.get_packed(ci, r) for ci, (L, R, _) in enumerate(classes) for r in range(R)]
            b.reinit()
            g, _ = b.run(times)
            out[on] = (rec, packed, g)
    assert np.array_equal(out[False][0], out[True][0])
    for x, y in zip(out[False][1], out[True][1]):
        assert np.array_equal(x, y)
    assert np.array_equal(out[False][2], out[True][2])
    with ising.Batch(classes[2:]) as b:  # streamed classes only: nothing to overlap
        b.set_overlap(True)
        b.sweep(3)
        for ci, (L, R, seed) in enumerate(classes[2:]):
            with ising.Ising(L, replicas=R, seed=seed) as q:
                q.sweep(3)
                for r in range(R):
                    assert np.array_equal(b.get_packed(ci, r), q.get_packed(r))


def test_missing_group_member_times_out_instead_of_hanging(ising):
    import time
    with ising.Batch([(128, 1, 1)]) as b:
        plan = b.plan()
        assert plan["groups"] == 1 and plan["ctas"] > 1
        b.inject_missing_cta(0, timeout_s=0.5)
        t0 = time.time()
        b.sweep(3)
        with pytest.raises(ising.IsingError) as e:
            b.sync()
        assert e.value.status == ising.ISING_ETIMEOUT
        assert time.time() - t0 < 30
        with pytest.raises(ising.IsingError) as e:
            b.sweep(1)
        assert e.value.status == ising.ISING_EPOISONED
    # the device is still usable afterwards
    with ising.Ising(64, replicas=1, seed=1) as q:
        q.sweep(2)
        q.measure()


def test_config4_mix_in_the_bench_configuration(ising):
    # the mixed batch of the benchmark (512 x 64^3 + 64 x 128^3 + 16 x 256^3 + 4 x 512^3, one
    # seed per lattice), tuned work list, 10^4 MCS with 20 log-spaced measurements as one graph:
    # the first and last lattice of every class against a single context measured at the same
    # times (every recorded time), the oracle's recount of their final states, and a one-MCS
    # oracle advance of the final state of one lattice per class
    from paper_2305_12161_gb300 import inputs
    classes = [(64, 512, 1), (128, 64, 513), (256, 16, 577), (512, 4, 593)]
    times = inputs.log_schedule(10_000, 20)
    with ising.Batch(classes) as b:
        b.tune(probe_mcs=4)
        b.reinit()
        rec, der = b.run(times, c=0.5)
        assert b.t == times[-1]
        finals = {}
        for ci, (L, R, seed) in enumerate(classes):
            for r in (0, R - 1):
                with ising.Ising(L, replicas=1, seed=seed + r) as q:
                    t = 0
                    for k, tk in enumerate(times):
                        q.sweep(tk - t)
                        t = tk
                        assert np.array_equal(b.record_of(rec[k], ci, r), q.measure()[0]), (L, r, tk)
                    finals[(ci, r)] = q.get_spins(0)
                assert np.array_equal(oracle.record(finals[(ci, r)], times[-1]), b.record_of(rec[-1], ci, r)), (L, r)
        b.sweep(1)
        for ci, (L, R, seed) in enumerate(classes):
            s = finals[(ci, 0)]
            oracle.sweeps(s, times[-1], 1, seed)
            with ising.Ising(L, replicas=1, seed=seed) as q:
                q.set_spins(s, 0)
                assert np.array_equal(b.get_packed(ci, 0), q.get_packed(0)), L
