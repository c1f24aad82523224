"""Pins for the oracle's double-checkerboard update (no GPU).

* Blocks of one site: every red block is an even site and every blue block an odd one, so
  the double checkerboard is the plain checkerboard sweep (01 and mixed cycle), whatever
  the fine order.
* One block spanning the lattice: the blue pass is empty and the sweep is the two
  checkerboard half-sweeps in the fine order (odd first in the 01 cycle, the drawn parity
  first in the mixed cycle).
* Any other tiling equals the composition, block by block in a shuffled order, of the
  separately pinned single-site update applied to each fine sublattice of the block.
* Ground states and flat stripes stay fixed, B never rises, the global spin-flip symmetry
  holds, invalid tilings are refused, and the mixed-cycle fine-order bits are balanced.
"""
import numpy as np
import pytest

import oracle
from paper_2305_12161_gb300 import inputs


@pytest.mark.parametrize("L", [4, 8, 12])
@pytest.mark.parametrize("rule", [0, 1, 2])
def test_unit_blocks_are_the_checkerboard(L, rule):
    S = 7 + L
    a = oracle.init(L, seed=S)
    b = a.copy()
    oracle.sweeps_dcb(a, 2, 4, S, (1, 1, 1), rule=rule)
    oracle.sweeps(b, 2, 4, S, rule)
    assert np.array_equal(a, b)
    a = oracle.init(L, seed=S)
    b = a.copy()
    oracle.sweeps_dcb(a, 0, 5, S, (1, 1, 1), rule=rule, mixed=True)
    oracle.sweeps_mixed(b, 0, 5, S, rule)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("mixed", [False, True])
def test_one_block_is_two_half_sweeps_in_fine_order(mixed):
    L, S = 8, 31
    a = oracle.init(L, seed=S)
    b = a.copy()
    oracle.sweeps_dcb(a, 1, 6, S, (L, L, L), mixed=mixed)
    for t in range(1, 7):
        f0 = oracle.dcb_fine_first(S, t, 0) if mixed else 1
        oracle.half_sweep(b, f0, t, S)
        oracle.half_sweep(b, 1 - f0, t, S)
    assert np.array_equal(a, b)
    if mixed:  # both fine orders occur in that window
        assert len({oracle.dcb_fine_first(S, t, 0) for t in range(1, 7)}) == 2


def _composed_sweep(s, t, S, block, mixed, rng):
    """One double-checkerboard sweep composed of single-site updates, blocks shuffled."""
    L = s.shape[0]
    bx, by, bz = block
    nbx, nby, nbz = L // bx, L // by, L // bz
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    parity = (x + y + z) & 1
    beta = (x // bx) + nbx * ((y // by) + nby * (z // bz))
    colour = ((x // bx) + (y // by) + (z // bz)) & 1
    flat = (x + L * (y + L * z)).astype(np.int64)
    first = oracle.mixed_order(S, t) if mixed else 0
    for c in (first, 1 - first):
        blocks = np.unique(beta[colour == c])
        rng.shuffle(blocks)
        for b in blocks:
            f0 = oracle.dcb_fine_first(S, t, int(b)) if mixed else 1
            for q in (f0, 1 - f0):
                sel = (beta == b) & (parity == q)
                sites = flat[sel]
                s.reshape(-1)[sites] = oracle.update_sites(s, q, t, S, sites)


@pytest.mark.parametrize("block", [(4, 2, 8), (2, 8, 4), (8, 4, 2), (2, 2, 2)])
@pytest.mark.parametrize("mixed", [False, True])
def test_tilings_equal_composed_site_updates(block, mixed):
    L, S = 8, 5
    rng = np.random.default_rng(3)
    a = oracle.init(L, seed=S)
    b = a.copy()
    oracle.sweeps_dcb(a, 0, 3, S, block, mixed=mixed)
    for t in range(3):
        _composed_sweep(b, t, S, block, mixed, rng)
    assert np.array_equal(a, b)


def test_double_checkerboard_differs_from_checkerboard():
    L, S = 8, 9
    a = oracle.init(L, seed=S)
    b = a.copy()
    oracle.sweeps_dcb(a, 0, 4, S, (2, 2, 2))
    oracle.sweeps(b, 0, 4, S)
    assert not np.array_equal(a, b)


def test_invalid_tilings_refused():
    assert oracle.dcb_valid(8, (2, 4, 8))
    assert not oracle.dcb_valid(12, (4, 2, 2))   # 3 blocks along x: same colours would touch
    assert not oracle.dcb_valid(8, (3, 2, 2))    # not a divisor
    assert not oracle.dcb_valid(8, (0, 2, 2))
    s = oracle.init(12, seed=1)
    with pytest.raises(ValueError):
        oracle.sweeps_dcb(s, 0, 1, 1, (4, 2, 2))


def test_fixed_points_monotone_B_and_flip_symmetry():
    L = 12
    for rule in (0, 1, 2):
        for s0 in (inputs.uniform_state(L, -1), inputs.stripe_state(L, 3, "z")):
            for mixed in (False, True):
                s = s0.copy()
                oracle.sweeps_dcb(s, 0, 3, 4, (6, 2, 12), rule=rule, mixed=mixed)
                assert np.array_equal(s, s0)
    s = oracle.init(12, seed=6)
    sbar = (-s).astype(np.int8)
    B = oracle.record(s)[2]
    for t in range(6):
        oracle.sweeps_dcb(s, t, 1, 6, (3, 6, 2), mixed=True)
        oracle.sweeps_dcb(sbar, t, 1, 6, (3, 6, 2), mixed=True)
        B2 = oracle.record(s)[2]
        assert B2 <= B
        B = B2
    assert np.array_equal(sbar, -s)


def test_fine_order_bits_balanced():
    bits = [oracle.dcb_fine_first(11, t, beta) for t in range(20) for beta in range(200)]
    n = len(bits)
    assert abs(sum(bits) - n / 2) < 5 * np.sqrt(n / 4)
