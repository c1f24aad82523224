"""Statistical cross-check against the paper's published domain-size histogram.

Supplementary Discussion II (figure "domain-size histogram"): 1000 independent L=256 runs of
the 01-cycle checkerboard update, measured at rescaled time 4000 MCS, have a mean domain
size of 19.9 (the n-fold way: 19.8).  The checkerboard's time factor is 1.75 (Supplementary
Table of time factors), so the runs here stop at 2286 checkerboard MCS; seeds 1..1000; l is
the first crossing of the radially averaged C(r) with 1/2.

The paper states neither its radial bin edges nor the exact measurement time of its
log-spaced schedule.  Measured on the same lattices, floor(|k|) bins give an l lower by 0.45
than the round(|k|) bins used here, and l grows about as t^0.45, so a schedule point 4% early
lowers it by 2%.  The band is therefore 5% of the paper's mean.  Two controls show that the
band still separates dynamics: the mixed cycle's slower clock (time factor 1.45 instead of
1.75, so l lower by about (1.45/1.75)^0.45 = 0.92 at the same number of sweeps) and the rule
that never flips at zero energy, which freezes early.
"""
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    vals = {}
    for line in open(os.path.join(HERE, "golden", "ell_hist_L256.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


@pytest.fixture(scope="module")
def ising():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2305_12161_gb300 import ising as m
    return m


def test_mean_domain_size_L256_matches_the_paper(ising):
    g = _golden()
    L, runs = int(g["L"]), int(g["runs"])
    mcs = round(g["rescaled_time_mcs"] / g["checkerboard_factor"])
    assert mcs == 2286
    with ising.Ising(L, replicas=runs, seed=1) as q:
        q.sweep(mcs)
        ell = np.array([q.measure_radial(replica=r)["ell"] for r in range(runs)])
    assert np.isfinite(ell).all()
    mean, sem = float(ell.mean()), float(ell.std(ddof=1) / math.sqrt(runs))
    paper = g["mean_ell_checkerboard"]
    assert sem < 0.15
    assert abs(mean - paper) <= 0.05 * paper, (mean, sem, paper)
    # the n-fold way (rsf dynamics) agrees with the checkerboard at the rescaled time
    assert abs(mean - g["mean_ell_nfold"]) <= 0.05 * g["mean_ell_nfold"]


def test_controls_fall_outside_the_band(ising):
    g = _golden()
    L = int(g["L"])
    mcs = round(g["rescaled_time_mcs"] / g["checkerboard_factor"])
    paper = g["mean_ell_checkerboard"]
    runs = 64
    means = {}
    for name, kw in (("01", {}), ("mixed", dict(cycle=ising.CYCLE_MIXED)), ("never", dict(tie=ising.TIE_NEVER))):
        with ising.Ising(L, replicas=runs, seed=1, **kw) as q:
            q.sweep(mcs)
            ell = np.array([q.measure_radial(replica=r)["ell"] for r in range(runs)])
        means[name] = float(np.nanmean(ell))
    assert abs(means["01"] - paper) <= 0.05 * paper + 0.7  # 64 runs: standard error about 0.33
    assert means["mixed"] < 0.96 * means["01"], means
    assert means["never"] < 0.8 * paper, means


def test_checkerboard_on_gpu_matches_rsf_oracle_at_rescaled_time(ising):
    # Supplementary Table of time factors: the checkerboard's time is multiplied by 1.75 to
    # match the random-site-flip (rsf) dynamics (Methods, "Random-site-flip update").  The
    # GPU checkerboard at tau sweeps (128 lattices of L = 64, seeds 1..128) is compared with
    # the sequential rsf oracle at round(1.75 tau) sweeps (24 lattices, seeds 1001..1024) by
    # the mean excess-energy length l_E = N/B.  Band: 5% (the oracle prototype gives ratios
    # 0.99 to 1.02 for tau = 16..64 with standard errors near 1%).  Control: the rsf oracle
    # at tau itself (time factor 1) is more than 15% below the checkerboard.
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    L, N = 64, 64**3
    taus = (16, 32, 64)
    with ising.Ising(L, replicas=128, seed=1) as q:
        cb = []
        for tau in taus:
            q.sweep(tau - q.t)
            _, der = q.measure_ex(corr=False)
            cb.append(float(der[:, 2].mean()))

    def rsf(seed, factor):
        s = oracle.init(L, seed)
        out, t = [], 0
        for tau in taus:
            tt = int(round(factor * tau))
            oracle.sweeps_rsf(s, t, tt - t, seed)
            t = tt
            out.append(N / oracle.magnetisation_bonds(s)[1])
        return out

    seeds = range(1001, 1025)
    with ThreadPoolExecutor(16) as ex:
        r175 = np.array(list(ex.map(lambda sd: rsf(sd, 1.75), seeds))).mean(axis=0)
        r1 = np.array(list(ex.map(lambda sd: rsf(sd, 1.0), seeds))).mean(axis=0)
    for j, tau in enumerate(taus):
        assert abs(cb[j] / r175[j] - 1) < 0.05, (tau, cb[j], r175[j])
        assert cb[j] / r1[j] > 1.15, (tau, cb[j], r1[j])
