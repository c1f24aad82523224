"""GPU <-> oracle parity through the C ABI (bit-exact: spins and int64 records).

Every case runs the CUDA library and the CPU oracle on the same seeded input and
compares element by element.  Sizes are chosen so that the oracle finishes in seconds
while the GPU grids span several tiles (and, for the word variant, a ragged last block).
"""
import numpy as np
import pytest

import oracle
from paper_2305_12161_gb300 import inputs

pytestmark = pytest.mark.gpu

RULES = (0, 1, 2)


@pytest.fixture(scope="module")
def ising():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2305_12161_gb300 import ising as m
    return m


def _run_gpu(ising, L, R, seed, times, keep_spins=True, **opts):
    recs, spins = [], []
    with ising.Ising(L, replicas=R, seed=seed, **opts) as q:
        recs.append(q.measure())
        if keep_spins:
            spins.append([q.get_spins(r) for r in range(R)])
        t = 0
        for tk in times:
            q.sweep(tk - t)
            t = tk
            recs.append(q.measure())
            if keep_spins:
                spins.append([q.get_spins(r) for r in range(R)])
        assert q.t == t
    return np.stack(recs, axis=1), spins  # recs: [R, K+1, RL]


def _compare(ising, L, R, seed, times, rule=0, **opts):
    got, gspins = _run_gpu(ising, L, R, seed, times, tie=rule, **opts)
    for r in range(R):
        want, ospins = oracle.run(L, seed, r, times, rule=rule, keep_spins=True)
        for k in range(len(times) + 1):
            assert np.array_equal(gspins[k][r], ospins[k]), f"spins differ: replica {r}, time index {k}"
        assert np.array_equal(got[r], want), f"records differ: replica {r}"


def test_c1_plain_L32_full_schedule(ising):
    # smallest instance: one L=32 lattice, seed 1, GLAUBER, 1000 MCS, 20 log-spaced times
    times = inputs.log_schedule(1000, 20)
    _compare(ising, 32, 1, 1, times, form=ising.FORM_PLAIN)


def test_c1_packed_L32_full_schedule(ising):
    times = inputs.log_schedule(1000, 20)
    _compare(ising, 32, 1, 1, times, form=ising.FORM_PACKED)


@pytest.mark.parametrize("rule", RULES)
@pytest.mark.parametrize("L", [4, 8, 16, 64, 128])
def test_word_variant_small_L_all_rules(ising, L, rule):
    times = [1, 2, 5, 13, 30]
    _compare(ising, L, 2, 7, times, rule=rule, variant=ising.VARIANT_WORD)


@pytest.mark.parametrize("rule", RULES)
def test_plain_form_all_rules(ising, rule):
    _compare(ising, 64, 2, 11, [1, 3, 9, 20], rule=rule, form=ising.FORM_PLAIN)


@pytest.mark.parametrize("tiles", [(256, 8), (64, 16), (32, 4), (128, 256)])
def test_zmarch_L256_vs_oracle(ising, tiles):
    ty, tz = tiles
    _compare(ising, 256, 1, 3, [1, 2, 4], variant=ising.VARIANT_ZMARCH, tile_y=ty, tile_z=tz)


@pytest.mark.parametrize("tz", [1, 4, 16, 256])
def test_zfast_L256_vs_oracle(ising, tz):
    _compare(ising, 256, 1, 13, [1, 2, 5], variant=ising.VARIANT_ZFAST, tile_z=tz)


@pytest.mark.parametrize("depth", [2, 3, 4])
def test_zdeep_L256_vs_oracle(ising, depth):
    _compare(ising, 256, 1, 14, [1, 2, 5], variant=ising.VARIANT_ZDEEP, tile_z=4, depth=depth)
    _compare(ising, 256, 2, 15, [2], rule=1, variant=ising.VARIANT_ZDEEP, tile_z=1, depth=depth)


def test_zfast_rules_and_replicas_L256(ising):
    for rule in (1, 2):
        _compare(ising, 256, 1, 6, [1, 3], rule=rule, variant=ising.VARIANT_ZFAST)
    _compare(ising, 256, 2, 21, [2], variant=ising.VARIANT_ZFAST, tile_z=8)


@pytest.mark.parametrize("tz", [1, 4, 16, 256])
def test_zfuse_L256_vs_oracle(ising, tz):
    # odd and even sweep counts: the state ends in either of the two stores
    _compare(ising, 256, 1, 16, [1, 2, 5], variant=ising.VARIANT_ZFUSE, tile_z=tz)


@pytest.mark.parametrize("tz", [1, 8, 256])
def test_zfuse_balanced_L256_vs_oracle(ising, tz):
    # 254-row tiles: the second of the two tiles owns two rows and wraps onto the first
    _compare(ising, 256, 1, 18, [1, 2, 5], variant=ising.VARIANT_ZFUSE, tile_z=tz, depth=11)
    _compare(ising, 256, 2, 19, [3], rule=1, variant=ising.VARIANT_ZFUSE, tile_z=tz, depth=8)
    _compare(ising, 256, 1, 20, [2, 3], rule=2, variant=ising.VARIANT_ZFUSE, tile_z=tz, depth=9)
    # z-blocks fitted to the resident CTAs (tiles of unequal depth)
    _compare(ising, 256, 1, 21, [1, 2, 5], variant=ising.VARIANT_ZFUSE, tile_z=tz, depth=27)
    _compare(ising, 256, 2, 22, [3], rule=1, variant=ising.VARIANT_ZFUSE, tile_z=tz, depth=19)


def test_zfuse_rules_and_replicas_L256(ising):
    for rule in (1, 2):
        _compare(ising, 256, 1, 17, [1, 3], rule=rule, variant=ising.VARIANT_ZFUSE, tile_z=32)
    _compare(ising, 256, 3, 22, [3], variant=ising.VARIANT_ZFUSE, tile_z=8)
    # three copy groups in flight, and one (four slots, four CTAs per SM)
    _compare(ising, 256, 2, 23, [1, 4], variant=ising.VARIANT_ZFUSE, tile_z=16, depth=3)
    _compare(ising, 256, 2, 24, [1, 4], variant=ising.VARIANT_ZFUSE, tile_z=2, depth=1)


def test_zmarch_rules_L256(ising):
    for rule in (1, 2):
        _compare(ising, 256, 1, 5, [1, 3], rule=rule, variant=ising.VARIANT_ZMARCH)


def test_replicas_each_follow_seed_plus_r(ising):
    _compare(ising, 64, 5, 100, [1, 4, 10])


def _packed_state(ising, L, R, seed, n, **opts):
    with ising.Ising(L, replicas=R, seed=seed, **opts) as q:
        q.sweep(n)
        return [q.get_packed(r) for r in range(R)], q.measure()


@pytest.mark.parametrize("L", [512, 1024, 2048])
def test_variants_and_tiles_bit_identical(ising, L):
    ref, rec = _packed_state(ising, L, 1, 9, 6, variant=ising.VARIANT_WORD)
    W4 = L // 256
    for ty, tz in ((256 // W4, 32), (128 // W4, 8), (1024 // W4, 64), (32 // W4 if 32 // W4 else 1, L)):
        if ty * W4 < 32 or ty * W4 > 1024 or L % ty:
            continue
        got, grec = _packed_state(ising, L, 1, 9, 6, variant=ising.VARIANT_ZMARCH, tile_y=ty, tile_z=tz)
        assert np.array_equal(got[0], ref[0]), (ty, tz)
        assert np.array_equal(grec, rec)
    for tz in (2, 32, L):
        got, grec = _packed_state(ising, L, 1, 9, 6, variant=ising.VARIANT_ZFAST, tile_z=tz)
        assert np.array_equal(got[0], ref[0]), ("zfast", tz)
        assert np.array_equal(grec, rec)
        for d in (2, 3, 4):
            got, grec = _packed_state(ising, L, 1, 9, 6, variant=ising.VARIANT_ZDEEP, tile_z=tz, depth=d)
            assert np.array_equal(got[0], ref[0]), ("zdeep", tz, d)
            assert np.array_equal(grec, rec)
    for tz in (1, 16, 64, L):
        for d in (0, 1, 3, 9, 11, 19, 25, 26, 27):  # ragged tiles of 256 / W4 - 2 rows in the balanced form
            got, grec = _packed_state(ising, L, 1, 9, 6, variant=ising.VARIANT_ZFUSE, tile_z=tz, depth=d)
            assert np.array_equal(got[0], ref[0]), ("zfuse", tz, d)
            assert np.array_equal(grec, rec)


@pytest.mark.parametrize("rule", RULES)
def test_zfuse_matches_zfast_L512_rules_replicas_odd_count(ising, rule):
    ref, rec = _packed_state(ising, 512, 2, 31, 7, tie=rule, variant=ising.VARIANT_ZFAST)
    for d in (0, 10, 26):
        got, grec = _packed_state(ising, 512, 2, 31, 7, tie=rule, variant=ising.VARIANT_ZFUSE, tile_z=32, depth=d)
        for r in range(2):
            assert np.array_equal(got[r], ref[r]), (r, d)
        assert np.array_equal(grec, rec)


def test_plain_and_packed_forms_identical_L256(ising):
    a, ra = _packed_state(ising, 256, 2, 4, 12, form=ising.FORM_PACKED)
    b, rb = _packed_state(ising, 256, 2, 4, 12, form=ising.FORM_PLAIN)
    for r in range(2):
        assert np.array_equal(a[r], b[r])
    assert np.array_equal(ra, rb)


@pytest.mark.parametrize("L", [4, 16, 32, 64, 128, 256])
def test_measure_on_structured_states(ising, L):
    states = [inputs.uniform_state(L, 1), inputs.uniform_state(L, -1), inputs.neel_state(L),
              inputs.stripe_state(L, max(1, L // 4), "x"), inputs.stripe_state(L, 1, "y", 1),
              inputs.stripe_state(L, 2, "z"), inputs.random_state(L, 3, 0.3),
              inputs.cube_defect_state(L, min(L, 3))]
    with ising.Ising(L, replicas=len(states), seed=1) as q:
        for r, s in enumerate(states):
            q.set_spins(s, r)
        rec, der = q.measure_ex(c=0.5)
        for r, s in enumerate(states):
            assert np.array_equal(q.get_spins(r), s)
            want = oracle.record(s, 0)
            assert np.array_equal(rec[r], want), r
            wd = oracle.derived(L, want, 0.5)
            np.testing.assert_allclose(der[r], wd, rtol=1e-12, atol=0, equal_nan=True)
        rec2, der2 = q.measure_ex(c=0.4, connected=True)
        for r, s in enumerate(states):
            wd = oracle.derived(L, rec2[r], 0.4, connected=True)
            np.testing.assert_allclose(der2[r], wd, rtol=1e-12, atol=0, equal_nan=True)


def test_energy_only_measure_marks_correlations_absent(ising):
    with ising.Ising(64, replicas=2, seed=3) as q:
        q.sweep(5)
        full = q.measure()
        rec, der = q.measure_ex(corr=False)
        assert np.array_equal(rec[:, :3], full[:, :3])
        assert np.all(rec[:, 3:] == -1)
        assert np.all(np.isnan(der[:, 3]))


def test_checkpoint_resume_is_bit_exact(ising):
    with ising.Ising(256, replicas=1, seed=17) as a:
        a.sweep(7)
        ck = a.get_packed(0)
        t = a.t
        a.sweep(5)
        end_a = a.get_packed(0)
    with ising.Ising(256, replicas=1, seed=17) as b:
        b.set_packed(ck, 0)
        b.t = t
        b.sweep(5)
        assert np.array_equal(b.get_packed(0), end_a)


@pytest.mark.parametrize("variant", [3, 5])
def test_checkpoint_async_host_load_is_ordered(ising, variant):
    # asynchronous loads from pinned memory land in stream order: queued sweeps run on the old
    # state first, later sweeps on the loaded one; two loads in a row reuse the staging buffer
    import torch
    L = 256
    with ising.Ising(L, replicas=2, seed=17) as a:
        a.sweep(4)
        w0, w1 = a.get_packed(0), a.get_packed(1)
    p0 = torch.from_numpy(w0.view(np.int32).copy()).pin_memory()
    p1 = torch.from_numpy(w1.view(np.int32).copy()).pin_memory()
    with ising.Ising(L, replicas=2, seed=5, variant=variant) as ref:  # the synchronous path
        ref.sweep(3)
        ref.set_packed(w1, 0)
        ref.set_packed(w0, 1)
        ref.sweep(2)
        ref.set_packed(w0, 0)
        ref.sweep(3)
        want = [ref.get_packed(0), ref.get_packed(1)]
    with ising.Ising(L, replicas=2, seed=5, variant=variant) as q:
        q.sweep(3)
        q.set_packed(p1, 0, asynchronous=True)
        q.set_packed(p0, 1, asynchronous=True)
        q.sweep(2)
        q.set_packed(p0, 0, asynchronous=True)
        q.sweep(3)
        q.sync()
        assert np.array_equal(q.get_packed(0), want[0])
        assert np.array_equal(q.get_packed(1), want[1])
        with pytest.raises(ValueError):
            q.set_packed(w0, 0, asynchronous=True)  # not page-locked
        q.release_scratch()  # frees the staging buffer; the next load allocates it again
        q.set_packed(p1, 1, asynchronous=True)
        q.sync()
        assert np.array_equal(q.get_packed(1), w1)


def test_invalid_spin_values_rejected(ising):
    with ising.Ising(8, replicas=1, seed=1) as q:
        bad = np.ones((8, 8, 8), dtype=np.int8)
        bad[0, 0, 0] = 0
        with pytest.raises(ising.IsingError):
            q.set_spins(bad, 0)
        with pytest.raises(ising.IsingError):
            q.get_spins(3)
        # the context is still usable after argument errors
        q.sweep(1)
        q.measure()


def test_zero_sweeps_and_time(ising):
    with ising.Ising(64, replicas=1, seed=2) as q:
        r0 = q.measure()
        q.sweep(0)
        assert q.t == 0 and np.array_equal(q.measure(), r0)


def test_reinit_equals_fresh_context(ising):
    with ising.Ising(64, replicas=2, seed=5) as a:
        a.sweep(9)
        a.reinit(8)
        assert a.t == 0
        a.sweep(3)
        ra = a.measure()
    with ising.Ising(64, replicas=2, seed=8) as b:
        b.sweep(3)
        assert np.array_equal(b.measure(), ra)


@pytest.mark.parametrize("L", [256, 384, 512, 1024])
def test_tensor_core_correlation_equals_popcount(ising, L):
    R = 2 if L <= 512 else 1
    with ising.Ising(L, replicas=R, seed=3, corr=ising.CORR_POPCOUNT) as a, \
            ising.Ising(L, replicas=R, seed=3, corr=ising.CORR_TENSOR) as b:
        for n in (0, 3, 20):
            a.sweep(n)
            b.sweep(n)
            ra, rb = a.measure(), b.measure()
            assert np.array_equal(ra, rb), n
            # two measurements in a row reuse the scratch and give the same record
            assert np.array_equal(b.measure(), rb)


def test_tensor_core_correlation_closed_forms(ising):
    L = 256
    states = [inputs.neel_state(L), inputs.stripe_state(L, 8, "x"), inputs.stripe_state(L, 3, "z", 1),
              inputs.uniform_state(L, -1)]
    with ising.Ising(L, replicas=len(states), seed=1, corr=ising.CORR_TENSOR) as q:
        for r, s in enumerate(states):
            q.set_spins(s, r)
        rec, der = q.measure_ex()
    for r, s in enumerate(states):
        want = oracle.record(s, 0)
        assert np.array_equal(rec[r], want), r


def test_tensor_core_correlation_rejects_unsupported_sizes(ising):
    with pytest.raises(ising.IsingError):
        ising.Ising(64, replicas=1, seed=1, corr=ising.CORR_TENSOR)


def test_tensor_core_wait_times_out_instead_of_hanging(ising):
    import time
    with ising.Ising(512, replicas=1, seed=2, corr=ising.CORR_TENSOR) as q:
        q.sweep(2)
        good = q.measure()
        q.inject_corr_stall(0.3)
        t0 = time.time()
        with pytest.raises(ising.IsingError) as e:
            q.measure()
        assert e.value.status == ising.ISING_ETIMEOUT
        assert time.time() - t0 < 30
        with pytest.raises(ising.IsingError) as e:
            q.sweep(1)
        assert e.value.status == ising.ISING_EPOISONED
    # the device is still usable, and the same measurement is exact again in a new context
    with ising.Ising(512, replicas=1, seed=2, corr=ising.CORR_TENSOR) as q:
        q.sweep(2)
        assert np.array_equal(q.measure(), good)


@pytest.mark.parametrize("rule", RULES)
def test_plain16_vs_oracle_ragged_rows(ising, rule):
    # L = 192: 12 sixteen-byte chunks per row, so rows straddle warps and the Philox groups
    # of a row (96 compressed indices) straddle rows; L = 16: one chunk per row
    _compare(ising, 192, 1, 17, [1, 2, 5], rule=rule, form=ising.FORM_PLAIN)
    _compare(ising, 16, 2, 3, [1, 4, 30], rule=rule, form=ising.FORM_PLAIN)


@pytest.mark.parametrize("L", [512, 1024])
def test_plain_and_packed_forms_identical_large(ising, L):
    # rows of 32 and 64 chunks: warps inside rows; both cycles
    for cycle in (ising.CYCLE_01, ising.CYCLE_MIXED):
        a, ra = _packed_state(ising, L, 1, 9, 5, form=ising.FORM_PACKED, cycle=cycle)
        b, rb = _packed_state(ising, L, 1, 9, 5, form=ising.FORM_PLAIN, cycle=cycle)
        assert np.array_equal(a[0], b[0]), cycle
        assert np.array_equal(ra, rb), cycle
