"""Pins for the oracle's checkerboard T = 0 dynamics (no GPU).

Each test fixes the oracle to something other than its own code: closed forms (Neel
state, stripes, ground states), the hand-worked 4^3 example of tests/golden/, the exact
bookkeeping identity between the incremental and recounted broken-bond numbers, the
monotone energy of a T = 0 quench, the global spin-flip symmetry of the Glauber rule and
the binomial statistics of the first half-sweep from a T = infinity start.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import TIE_ALWAYS, TIE_GLAUBER, TIE_NEVER
from paper_2305_12161_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RULES = (TIE_GLAUBER, TIE_ALWAYS, TIE_NEVER)


def _M(s):
    return int(s.astype(np.int64).sum())


def _B(s):
    return int(oracle.record(s)[2])


def _golden_cube():
    rows = {}
    with open(os.path.join(GOLDEN, "cube_2x2x2_L4.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            stage, sites, B, M = line.split()
            down = [] if sites == "-" else [tuple(int(v) for v in p.split(",")) for p in sites.split(";")]
            rows[stage] = (down, int(B), int(M))
    return rows


def _state_from_down(L, down):
    s = np.ones((L, L, L), dtype=np.int8)
    for x, y, z in down:
        s[z, y, x] = -1
    return s


def test_hand_worked_cube_glauber():
    g = _golden_cube()
    L = 4
    s = _state_from_down(L, g["start"][0])
    assert (_B(s), _M(s)) == g["start"][1:]
    oracle.half_sweep(s, 0, 0, 0, TIE_GLAUBER)
    assert np.array_equal(s, _state_from_down(L, g["t0_red"][0]))
    assert (_B(s), _M(s)) == g["t0_red"][1:]
    oracle.half_sweep(s, 1, 0, 0, TIE_GLAUBER)
    assert np.array_equal(s, _state_from_down(L, g["t0_blue"][0]))
    assert (_B(s), _M(s)) == g["t0_blue"][1:]
    oracle.half_sweep(s, 0, 1, 0, TIE_GLAUBER)
    assert np.array_equal(s, _state_from_down(L, g["t1_red"][0]))
    assert (_B(s), _M(s)) == g["t1_red"][1:]


def test_hand_worked_cube_always_and_never():
    L = 4
    start = inputs.cube_defect_state(L, 2)
    # NEVER: every cube site is a tie, so nothing moves.
    s = start.copy()
    oracle.sweeps(s, 0, 3, 0, TIE_NEVER)
    assert np.array_equal(s, start)
    # ALWAYS: the red half flips the 4 even cube sites up (tie flips, B stays 24); the 4
    # odd cube sites then have u = 6 and flip: all up after one MCS, B 24 -> 24 -> 0.
    s = start.copy()
    assert _B(s) == 24
    f, dB, _ = oracle.half_sweep(s, 0, 0, 0, TIE_ALWAYS)
    assert (f, dB, _B(s)) == (4, 0, 24)
    f, dB, _ = oracle.half_sweep(s, 1, 0, 0, TIE_ALWAYS)
    assert (f, dB, _B(s)) == (4, -24, 0)
    assert np.all(s == 1)


def test_single_defect_heals_in_its_own_half_sweep():
    L = 4
    for (x, y, z) in [(0, 0, 0), (1, 0, 0), (3, 2, 1), (2, 3, 3)]:
        q = (x + y + z) % 2
        s = np.ones((L, L, L), dtype=np.int8)
        s[z, y, x] = -1
        oracle.half_sweep(s, 1 - q, 0, 9, TIE_GLAUBER)   # other sublattice: no change
        assert s[z, y, x] == -1 and _M(s) == L**3 - 2
        oracle.half_sweep(s, q, 0, 9, TIE_GLAUBER)
        assert np.all(s == 1)


@pytest.mark.parametrize("rule", RULES)
def test_ground_states_are_fixed(rule):
    for sign in (1, -1):
        s = inputs.uniform_state(8, sign)
        oracle.sweeps(s, 0, 4, 3, rule)
        assert np.all(s == sign)


@pytest.mark.parametrize("rule", RULES)
@pytest.mark.parametrize("axis", ["x", "y", "z"])
def test_flat_stripes_are_fixed(rule, axis):
    # A flat slab interface: each spin has u in {1, 2, 4, 5} (never 3), so no move.
    L = 12
    for w in (1, 2, 3, 6):
        for phase in (0, 1):
            s = inputs.stripe_state(L, w, axis, phase)
            ref = s.copy()
            oracle.sweeps(s, 0, 3, 11, rule)
            assert np.array_equal(s, ref)


def test_neel_state_orders_in_one_half_sweep():
    # Every even site of the Neel state has u = 0 (all neighbours down): the red half
    # sweep maps it to all-down; B goes from 3N to 0, M from 0 to -N.
    L = 6
    N = L**3
    s = inputs.neel_state(L)
    assert _B(s) == 3 * N and _M(s) == 0
    f, dB, dM = oracle.half_sweep(s, 0, 0, 1, TIE_GLAUBER)
    assert f == N // 2 and dB == -3 * N and dM == -N
    assert np.all(s == -1)


def test_incremental_bookkeeping_matches_recount_and_energy_never_rises():
    # After every half-sweep the recounted B and M equal the values carried flip by
    # flip (a flip with a aligned neighbours changes B by 2a - 6), and B never rises:
    # same-sublattice sites share no bond and every accepted flip has dE <= 0.
    L = 16
    for rule in RULES:
        s = oracle.init(L, seed=3)
        B, M = _B(s), _M(s)
        for t in range(12):
            for q in (0, 1):
                _, dB, dM = oracle.half_sweep(s, q, t, 3, rule)
                assert dB <= 0
                B2, M2 = _B(s), _M(s)
                assert B2 == B + dB and M2 == M + dM
                B, M = B2, M2


def test_global_spin_flip_symmetry_glauber():
    # new = [u>=4] | ([u==3] & (s ^ r)) is odd under s -> -s with the same random bits,
    # so evolve(-s0) = -evolve(s0) bit for bit.
    L = 16
    s = oracle.init(L, seed=21)
    sbar = (-s).astype(np.int8)
    oracle.sweeps(s, 0, 10, 21, TIE_GLAUBER)
    oracle.sweeps(sbar, 0, 10, 21, TIE_GLAUBER)
    assert np.array_equal(sbar, -s)


def test_first_half_sweep_statistics_from_T_infinity():
    # From an i.i.d. start the red sites see u ~ Binomial(6, 1/2): strict moves
    # (u != 3 and spin misaligned with the majority) have probability 22/64, ties 20/64,
    # and a tie flips with probability 1/2 (its Philox bit).  After the half-sweep each
    # even site carries min(u, 6-u) broken bonds, so E[B] = (N/2) * 132/64.
    L = 64
    N = L**3
    s = oracle.init(L, seed=1)
    z, y, x = np.indices((L, L, L))
    even = (x + y + z) % 2 == 0
    up = (s == 1).astype(np.int64)
    u = sum(np.roll(up, sh, axis=ax) for ax in range(3) for sh in (1, -1))
    before = s.copy()
    oracle.half_sweep(s, 0, 0, 1, TIE_GLAUBER)
    flipped = (s != before) & even
    ue = u[even]
    n = even.sum()
    strict = ((ue <= 2) & (before[even] == 1)) | ((ue >= 4) & (before[even] == -1))
    tie = ue == 3
    # deterministic part: strict sites move, non-tie aligned sites do not
    assert np.array_equal(flipped[even] & ~tie, strict)
    # statistical part
    for frac, p in ((strict.mean(), 22 / 64), (tie.mean(), 20 / 64)):
        assert abs(frac - p) < 5 * np.sqrt(p * (1 - p) / n) * 3  # x3: u's share neighbours
    n_tie = int(tie.sum())
    n_tie_flip = int((flipped[even] & tie).sum())
    assert abs(n_tie_flip - n_tie / 2) < 5 * np.sqrt(n_tie / 4)
    B = _B(s)
    assert abs(B - n * 132 / 64) < 5 * np.sqrt(n * 6 * 0.7)
    assert abs((-3 + 2 * B / N) - (-0.9375)) < 0.01


def test_odd_half_uses_post_red_values():
    # The blue half must see the red sites as updated in the same sweep (01 cycle):
    # after the Neel state's red half every site is down, so the blue half is idle.
    s = inputs.neel_state(4)
    f0, _, _ = oracle.half_sweep(s, 0, 0, 0, TIE_GLAUBER)
    f1, _, _ = oracle.half_sweep(s, 1, 0, 0, TIE_GLAUBER)
    assert (f0, f1) == (32, 0)


def test_sweeps_is_red_then_blue_with_sweep_counter():
    L = 8
    a = oracle.init(L, seed=4)
    b = a.copy()
    oracle.sweeps(a, 5, 3, 4, TIE_GLAUBER)
    for t in (5, 6, 7):
        oracle.half_sweep(b, 0, t, 4, TIE_GLAUBER)
        oracle.half_sweep(b, 1, t, 4, TIE_GLAUBER)
    assert np.array_equal(a, b)


def test_update_sites_matches_full_half_sweep():
    # the site-by-site entry used for lattices too large for a full oracle pass must
    # agree with the half-sweep at every listed site
    L = 16
    s = oracle.init(L, seed=8)
    oracle.sweeps(s, 0, 3, 8, TIE_GLAUBER)
    for q in (0, 1):
        z, y, x = np.indices((L, L, L))
        sites = np.flatnonzero(((x + y + z) % 2 == q).ravel())
        got = oracle.update_sites(s, q, 3, 8, sites)
        full = s.copy()
        oracle.half_sweep(full, q, 3, 8, TIE_GLAUBER)
        assert np.array_equal(got, full.ravel()[sites])
