"""Pins for the random-site-flip oracle (Methods, "Random-site-flip update"; Eq. 6).

The rsf dynamics has no parallel counterpart in the library: it is the paper's baseline,
against which the checkerboard's time is rescaled (Supplementary Table of time factors:
checkerboard 1.75, rsf 1).  Pins: uniform site draws and balanced zero-energy bits; the
energy never rises and the incremental bond count equals a recount; ground states and
flat stripes are fixed for every rule; a single defect heals; global spin-flip symmetry;
and, statistically, the paper's time factor between the two dynamics.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2305_12161_gb300 import inputs


def test_site_draws_uniform_and_bits_balanced():
    N = 4096
    n = 1 << 16
    sites = np.empty(n, dtype=np.int64)
    bits = np.empty(n, dtype=np.int64)
    for k in range(n):
        sites[k], bits[k] = oracle.rsf_draw(7, 3, k, N)
    assert sites.min() >= 0 and sites.max() < N
    # 64 bins of 64 sites: chi-square with 63 degrees of freedom, far tail at 120
    counts = np.bincount(sites // 64, minlength=64)
    chi2 = ((counts - n / 64) ** 2 / (n / 64)).sum()
    assert chi2 < 120, chi2
    assert abs(bits.mean() - 0.5) < 5 * 0.5 / np.sqrt(n)
    # counter words: step, sweep and key all change the draw
    assert oracle.rsf_draw(7, 3, 5, N) != oracle.rsf_draw(7, 4, 5, N)
    assert oracle.rsf_draw(7, 3, 5, N) != oracle.rsf_draw(8, 3, 5, N)
    # step numbers beyond 2^32 use the fourth counter word (no wrap onto small k)
    big = 1 << 33
    assert oracle.rsf_draw(7, 3, 5 + (1 << 32), big) != oracle.rsf_draw(7, 3, 5, big)


@pytest.mark.parametrize("rule", [oracle.TIE_GLAUBER, oracle.TIE_ALWAYS, oracle.TIE_NEVER])
def test_energy_never_rises_and_incremental_counts_match(rule):
    L = 12
    s = inputs.random_state(L, 3)
    M0, B0 = oracle.magnetisation_bonds(s)
    for t in range(15):
        f, dB, dM = oracle.sweeps_rsf(s, t, 1, 11, rule)
        M1, B1 = oracle.magnetisation_bonds(s)
        assert B1 - B0 == dB and M1 - M0 == dM
        assert dB <= 0
        assert f >= 0
        if rule == oracle.TIE_NEVER:
            # strict flips only: every flip lowers B by at least 2
            assert dB <= -2 * f
        M0, B0 = M1, B1


@pytest.mark.parametrize("rule", [oracle.TIE_GLAUBER, oracle.TIE_ALWAYS, oracle.TIE_NEVER])
def test_fixed_points(rule):
    L = 12
    for sign in (1, -1):
        s = inputs.uniform_state(L, sign)
        assert oracle.sweeps_rsf(s, 0, 3, 5, rule)[0] == 0
        assert np.all(s == sign)
    for axis in "xyz":
        for w in (1, 2, 3):
            s = inputs.stripe_state(L, w, axis)
            ref = s.copy()
            assert oracle.sweeps_rsf(s, 0, 3, 5, rule)[0] == 0
            assert np.array_equal(s, ref)


def test_single_defect_heals():
    L = 8
    for rule in (oracle.TIE_GLAUBER, oracle.TIE_ALWAYS, oracle.TIE_NEVER):
        s = inputs.uniform_state(L)
        s[3, 4, 5] = -1
        # the defect flips the first time it is proposed (u = 6); the chance of missing it
        # in 40 sweeps is e^-40
        f, dB, dM = oracle.sweeps_rsf(s, 0, 40, 2, rule)
        assert f == 1 and dB == -6 and dM == 2
        assert np.all(s == 1)


def test_global_flip_symmetry_and_sweep_counter():
    L = 10
    s0 = inputs.random_state(L, 4)
    a, b = s0.copy(), (-s0).astype(np.int8)
    oracle.sweeps_rsf(a, 0, 6, 9)
    oracle.sweeps_rsf(b, 0, 6, 9)
    assert np.array_equal(a, -b)
    # n sweeps at once equal n calls of one sweep with the counter advanced
    c = s0.copy()
    for t in range(6):
        oracle.sweeps_rsf(c, t, 1, 9)
    assert np.array_equal(a, c)


def test_sequential_steps_follow_the_draws():
    # the first steps of a sweep, replayed one by one from the draws: each step reads the
    # lattice as the previous steps left it
    L, S, t = 4, 21, 0
    s = inputs.random_state(L, 8)
    want = s.copy()
    N = L**3
    for k in range(N):
        i, bit = oracle.rsf_draw(S, t, k, N)
        x, y, z = i % L, (i // L) % L, i // (L * L)
        nb = [want[z, y, (x + 1) % L], want[z, y, (x - 1) % L], want[z, (y + 1) % L, x], want[z, (y - 1) % L, x],
              want[(z + 1) % L, y, x], want[(z - 1) % L, y, x]]
        u = sum(v == 1 for v in nb)
        if u >= 4:
            want[z, y, x] = 1
        elif u <= 2:
            want[z, y, x] = -1
        elif bit:
            want[z, y, x] = -want[z, y, x]
    oracle.sweeps_rsf(s, t, 1, S)
    assert np.array_equal(s, want)


def test_paper_time_factor_between_checkerboard_and_rsf():
    # Supplementary Table of time factors: checkerboard times are multiplied by 1.75 to
    # match rsf.  The excess-energy length l_E = N/B of the checkerboard at tau agrees with
    # rsf at 1.75 tau within 6%, and differs by more than 12% from rsf at tau (control).
    L, runs = 48, 8
    N = L**3
    taus = (16, 32)

    def rsf(seed, factor):
        s = oracle.init(L, seed)
        out, t = [], 0
        for tau in taus:
            tt = int(round(factor * tau))
            oracle.sweeps_rsf(s, t, tt - t, seed)
            t = tt
            out.append(N / oracle.magnetisation_bonds(s)[1])
        return out

    def cb(seed):
        s = oracle.init(L, seed)
        out, t = [], 0
        for tau in taus:
            oracle.sweeps(s, t, tau - t, seed)
            t = tau
            out.append(N / oracle.magnetisation_bonds(s)[1])
        return out

    seeds = range(101, 101 + runs)
    with ThreadPoolExecutor(8) as ex:
        r175 = np.array(list(ex.map(lambda sd: rsf(sd, 1.75), seeds))).mean(axis=0)
        r1 = np.array(list(ex.map(lambda sd: rsf(sd, 1.0), seeds))).mean(axis=0)
    c = np.array([cb(sd) for sd in seeds]).mean(axis=0)
    for j, tau in enumerate(taus):
        assert abs(c[j] / r175[j] - 1) < 0.06, (tau, c[j], r175[j])
        assert c[j] / r1[j] > 1.12, (tau, c[j], r1[j])
