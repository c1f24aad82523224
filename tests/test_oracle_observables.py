"""Pins for the oracle's observables and derived lengths (no GPU).

Closed forms: ground states, the Neel state and flat stripes (for which D_a(r), B, the
excess-energy length l_E = w and the correlation length l_C = 3w/4 are known exactly);
identities D_a(0) = 0 and D_x(1) + D_y(1) + D_z(1) = B that tie two independent loops of
the oracle together; the symmetry D_a(r) = D_a(L - r) at r = L/2; the axis assignment
(x is the fastest index) against numpy's roll; and the measurement schedule.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2305_12161_gb300 import inputs


def _D(rec, L):
    return rec[3:].reshape(3, L // 2 + 1)


def _stripe_D(L, w, r):
    # square wave of half-period w: fraction of sites with s(x) != s(x+r)
    rho = r % (2 * w)
    return (rho if rho <= w else 2 * w - rho) * L**3 // w


def test_record_layout_and_length():
    for L in (4, 6, 32):
        assert oracle.record_len(L) == 3 + 3 * (L // 2 + 1)
    rec = oracle.record(inputs.uniform_state(4), t=17)
    assert rec[0] == 17


@pytest.mark.parametrize("sign", [1, -1])
def test_ground_state_record(sign):
    L = 8
    N = L**3
    rec = oracle.record(inputs.uniform_state(L, sign))
    assert rec[1] == sign * N and rec[2] == 0
    assert np.all(_D(rec, L) == 0)
    e, m, lE, lC = oracle.derived(L, rec)
    assert e == -3.0 and m == sign and math.isinf(lE) and math.isnan(lC)


def test_neel_record():
    L = 8
    N = L**3
    rec = oracle.record(inputs.neel_state(L))
    assert rec[1] == 0 and rec[2] == 3 * N
    D = _D(rec, L)
    for r in range(L // 2 + 1):
        assert np.all(D[:, r] == (N if r % 2 else 0))
    e, m, lE, lC = oracle.derived(L, rec)
    assert e == 3.0 and m == 0.0 and lE == pytest.approx(1 / 3)
    # C(0) = 1 >= 0.5 > C(1) = -1: crossing at 0 + 0.5/2 = 0.25
    assert lC == pytest.approx(0.25, abs=1e-12)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("w", [1, 2, 3, 4])
def test_stripe_records(axis, w):
    L = 24
    N = L**3
    s = inputs.stripe_state(L, w, "xyz"[axis])
    rec = oracle.record(s)
    D = _D(rec, L)
    for a in range(3):
        for r in range(L // 2 + 1):
            want = _stripe_D(L, w, r) if a == axis else 0
            assert D[a, r] == want, (a, r)
    assert rec[2] == N // w and rec[1] == 0
    e, m, lE, lC = oracle.derived(L, rec)
    # excess-energy length equals the slab width; C(r) = 1 - (2/3)(r/w) for r <= w,
    # which crosses 1/2 at r = 3w/4 (linear, so the interpolation is exact)
    assert lE == pytest.approx(w, rel=1e-12)
    assert lC == pytest.approx(0.75 * w, rel=1e-12)
    assert e == pytest.approx(-3 + 2 / w, rel=1e-12)


def test_intercept_parameter_and_connected_variant():
    L = 24
    rec = oracle.record(inputs.stripe_state(L, 4, "y"))
    for c in (0.4, 0.6, 0.7):
        # C(r) = 1 - r/6 on [0, 4]: crossing at r = 6(1 - c)
        assert oracle.derived(L, rec, c=c)[3] == pytest.approx(6 * (1 - c), rel=1e-12)
    # C never drops below 1/3 for stripes (its minimum at r = w), so c = 0.3 has no
    # crossing for r <= L/2
    assert math.isnan(oracle.derived(L, rec, c=0.3)[3])
    # a magnetised state: m^2 is subtracted from C in the connected variant
    s = inputs.stripe_state(L, 4, "y")
    s[:, 4:6, :] = 1   # two down planes (y = 4, 5) forced up: m = 4/24
    rec = oracle.record(s)
    e, m, lE, lC = oracle.derived(L, rec, c=0.5, connected=False)
    _, _, _, lC2 = oracle.derived(L, rec, c=0.5 + m * m, connected=False)
    _, _, _, lCc = oracle.derived(L, rec, c=0.5, connected=True)
    assert m != 0 and lCc == pytest.approx(lC2, rel=1e-12)


def test_bond_identities_on_random_states():
    for L, seed in ((6, 0), (10, 1), (16, 2)):
        s = inputs.random_state(L, seed)
        rec = oracle.record(s)
        D = _D(rec, L)
        assert np.all(D[:, 0] == 0)
        assert D[:, 1].sum() == rec[2]
        assert rec[1] == int(s.astype(np.int64).sum())


def test_axis_assignment_against_numpy_roll():
    # x is the fastest-varying index (array axis 2), z the slowest (axis 0)
    L = 10
    s = inputs.random_state(L, 5, p_up=0.3)
    rec = oracle.record(s)
    D = _D(rec, L)
    for a, ax in ((0, 2), (1, 1), (2, 0)):
        for r in range(L // 2 + 1):
            assert D[a, r] == int(np.sum(s != np.roll(s, -r, axis=ax)))


def test_half_distance_symmetry():
    # at r = L/2 the forward and backward partners coincide, and D_a(r) = D_a(L - r)
    # makes the r <= L/2 half the whole information
    L = 12
    s = inputs.random_state(L, 9)
    D = _D(oracle.record(s), L)
    for ax, a in ((2, 0), (1, 1), (0, 2)):
        for r in range(L // 2 + 1):
            assert D[a, r] == int(np.sum(s != np.roll(s, r, axis=ax)))


def test_log_schedule():
    assert inputs.log_schedule(1000, 4) == [1, 10, 100, 1000]
    assert inputs.log_schedule(10, 10) == list(range(1, 11))
    ts = inputs.log_schedule(1000, 20)
    assert ts[0] == 1 and ts[-1] == 1000 and all(b > a for a, b in zip(ts, ts[1:]))
    ts = inputs.log_schedule(10_000, 40)
    assert len(ts) == 40 and ts[-1] == 10_000 and all(b > a for a, b in zip(ts, ts[1:]))
    with pytest.raises(ValueError):
        inputs.log_schedule(3, 4)


def test_run_records_schedule():
    recs, _ = oracle.run(8, seed=1, replica=0, times=[1, 2, 5])
    assert list(recs[:, 0]) == [0, 1, 2, 5]
    # B never rises along a quench
    assert all(b >= a for a, b in zip(recs[1:, 2], recs[:-1, 2]))


@pytest.mark.parametrize("L,seed", [(4, 0), (6, 1), (16, 2), (34, 3)])
def test_line_counting_equals_site_counting(L, seed):
    # the record counts D_a(r) line by line (orc_corr_lags); orc_corr_lag counts the same
    # pairs site by site with periodic wrapping.  Two independent loops over Eq. (2)'s pairs
    # must agree at every distance, including those beyond L/2
    s = inputs.random_state(L, seed, p_up=0.4)
    rec = oracle.record(s)
    D = _D(rec, L)
    for r in range(L // 2 + 1):
        assert list(D[:, r]) == list(oracle.corr_lag(s, r)), r
    allD = oracle.corr_lags(s, list(range(L)))
    for r in range(L):
        assert list(allD[r]) == list(oracle.corr_lag(s, r)), r
    # lags in any order and repeated
    lags = [3, 0, L - 1, 3]
    assert np.array_equal(oracle.corr_lags(s, lags), allD[lags])


def test_line_counting_planted_structure():
    # a single flipped site in a uniform state: every axis has exactly 2 unequal pairs at
    # every distance r = 1..L-1, and 0 at r = 0 -- checks that each line is counted once
    L = 12
    s = inputs.uniform_state(L)
    s[5, 7, 3] = -1
    D = oracle.corr_lags(s, list(range(L)))
    assert np.all(D[0] == 0)
    assert np.all(D[1:] == 2)
    with pytest.raises(ValueError):
        oracle.corr_lags(s, [L])
