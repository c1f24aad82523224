"""Pins for the oracle's Menger-sponge start and mixed-cycle order (no GPU).

* Membership against an independent construction: carving a cube by removing, at every
  level, the centre and face-centre sub-cubes of each remaining sub-cube (numpy), and the
  closed form 20^k for the cells kept in a full tile.
* Tile signs and mixed-cycle order bits are balanced (binomial, 5 sigma); k = 0 is an
  i.i.d. start.
* Mixed cycle: each sweep is the two half-sweeps in the drawn order; ground states and
  flat stripes stay fixed; B never rises; the global spin-flip symmetry holds.
"""
import numpy as np
import pytest

import oracle
from paper_2305_12161_gb300 import inputs


def _carved_sponge(k):
    side = 3**k
    keep = np.ones((side, side, side), dtype=bool)
    sub = side
    while sub > 1:
        third = sub // 3
        for ox in range(0, side, sub):
            for oy in range(0, side, sub):
                for oz in range(0, side, sub):
                    for a in range(3):
                        for b in range(3):
                            for c in range(3):
                                if (a == 1) + (b == 1) + (c == 1) >= 2:
                                    keep[ox + a * third:ox + (a + 1) * third,
                                         oy + b * third:oy + (b + 1) * third,
                                         oz + c * third:oz + (c + 1) * third] = False
        sub = third
    return keep


@pytest.mark.parametrize("k", [0, 1, 2])
def test_menger_membership_matches_carving(k):
    carved = _carved_sponge(k)
    side = 3**k
    for a in range(side):
        for b in range(side):
            for c in range(side):
                assert oracle.menger_member(a, b, c, k) == bool(carved[a, b, c]), (a, b, c)


def test_menger_cell_counts_closed_form():
    for k in range(4):
        side = 3**k
        n = sum(oracle.menger_member(a, b, c, k) for a in range(side) for b in range(side) for c in range(side))
        assert n == 20**k


def test_menger_start_structure():
    # L = 27 = 3^3: whole tiles for k <= 3; each tile holds 20^k spins of its sign
    L = 27
    for k in (1, 2, 3):
        s = oracle.init_menger(L, seed=4, k=k)
        side = 3**k
        nT = L // side
        for tz in range(nT):
            for ty in range(nT):
                for tx in range(nT):
                    tile = s[tz * side:(tz + 1) * side, ty * side:(ty + 1) * side, tx * side:(tx + 1) * side]
                    sig = oracle.menger_tile_sign(4, tx + nT * (ty + nT * tz))
                    assert int((tile == sig).sum()) == 20**k
                    assert tile[side // 2, side // 2, side // 2] == -sig  # the centre is a hole


def test_menger_k0_is_iid_and_signs_balanced():
    L = 32
    s = oracle.init_menger(L, seed=9, k=0)
    N = L**3
    assert abs(int(s.astype(np.int64).sum())) < 5 * np.sqrt(N)
    signs = np.array([oracle.menger_tile_sign(3, T) for T in range(4000)])
    assert abs(int(signs.sum())) < 5 * np.sqrt(4000)


def test_menger_truncated_tiles_at_the_edge():
    # L = 32 with k = 3 (side 27): the second tile along each axis is cut to 5 cells
    s = oracle.init_menger(32, seed=2, k=3)
    sig = oracle.menger_tile_sign(2, 1)  # tile (1, 0, 0)
    for x in range(27, 32):
        want = sig if oracle.menger_member(x - 27, 0, 0, 3) else -sig
        assert s[0, 0, x] == want


def test_mixed_order_is_balanced():
    bits = [oracle.mixed_order(7, t) for t in range(2000)]
    assert abs(sum(bits) - 1000) < 5 * np.sqrt(500)


def test_mixed_sweep_is_half_sweeps_in_drawn_order():
    L = 16
    S = 12
    a = oracle.init(L, seed=S)
    b = a.copy()
    oracle.sweeps_mixed(a, 3, 6, S)
    for t in range(3, 9):
        first = oracle.mixed_order(S, t)
        oracle.half_sweep(b, first, t, S)
        oracle.half_sweep(b, 1 - first, t, S)
    assert np.array_equal(a, b)
    # at least one sweep in that window went blue first, so the cycles really differ
    assert any(oracle.mixed_order(S, t) for t in range(3, 9))


def test_mixed_cycle_physics():
    L = 12
    for rule in (0, 1, 2):
        for s0 in (inputs.uniform_state(L, 1), inputs.stripe_state(L, 3, "y")):
            s = s0.copy()
            oracle.sweeps_mixed(s, 0, 5, 3, rule)
            assert np.array_equal(s, s0)
    s = oracle.init(16, seed=5)
    sbar = (-s).astype(np.int8)
    B = oracle.record(s)[2]
    for t in range(8):
        oracle.sweeps_mixed(s, t, 1, 5)
        oracle.sweeps_mixed(sbar, t, 1, 5)
        B2 = oracle.record(s)[2]
        assert B2 <= B
        B = B2
    assert np.array_equal(sbar, -s)
