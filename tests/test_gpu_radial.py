"""GPU <-> oracle parity for the radially averaged 3-d correlation C(r) and structure factor S(k).

Every FFT value of G(k) is rounded to its integer.  Double precision: C is exact, so it must
equal the oracle's bit for bit, with no inexact lag; S agrees to the rounding of fp64 FFTs and
of the oracle's direct sums.  Single precision: exact too when no lag is inexact (small L);
otherwise C and S agree within the FFT error model
||delta y||_2 <= 5 u log2(N) ||y||_2 per transform (u = 2^-24): a bin mean of n lags is off by
at most 15 u log2(N) sqrt(N/n) in C and 10 u log2(N) N / sqrt(n) in S.

* L = 4..32: the oracle's brute-force G(k) and direct DFT (T = inf start, after sweeps,
  Menger start, ground state, Neel state, stripes).
* L = 64..256: numpy's fp64 FFT rounded to integers, binned by the same exact rule.
* L = 2048: bin counts 1, 18, 62; C(0) = 1; C(1) from the oracle's single-lag sums over the
  18 vectors of the bin; S(0) = M^2/N; Parseval; fp32 against fp64.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2305_12161_gb300 import inputs

pytestmark = pytest.mark.gpu

U32, U64 = 2.0**-24, 2.0**-53


@pytest.fixture(scope="module")
def ising():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2305_12161_gb300 import ising as m
    return m


def _tol_C(N, n, u):
    return 15 * u * math.log2(N) * np.sqrt(N / np.maximum(n, 1))


def _tol_S(N, n, u):
    return 10 * u * math.log2(N) * N / np.sqrt(np.maximum(n, 1))


def _check_against(res, C, S, n, N, prec, L, c=0.5):
    assert np.array_equal(res["count"], n)
    if prec == 1:
        assert res["inexact"] == 0
        assert np.array_equal(res["C"], C)  # exact integers summed, one division
        assert np.all(np.abs(res["S"] - S) <= _tol_S(N, n, U64) + 4 * N * N * U64)
        want = oracle.radial_length(L, C, c)
        assert (math.isnan(want) and math.isnan(res["ell"])) or res["ell"] == want
    else:
        assert res["inexact"] >= 0
        if res["inexact"] == 0:  # every rounded value was its integer: C exact
            assert np.array_equal(res["C"], C)
        assert np.all(np.abs(res["C"] - C) <= _tol_C(N, n, U32))
        assert np.all(np.abs(res["S"] - S) <= _tol_S(N, n, U32))


def _states(L, seed):
    out = {"init": oracle.init(L, seed, 1)}
    s = oracle.init(L, seed, 1)
    oracle.sweeps(s, 0, 3, seed + 1)
    out["swept"] = s
    out["uniform"] = inputs.uniform_state(L, -1)
    out["neel"] = inputs.neel_state(L)
    out["stripes"] = inputs.stripe_state(L, 2, "y")
    if L >= 9:
        out["menger"] = oracle.init_menger(L, seed, 1, replica=1)
    return out


@pytest.mark.parametrize("L", [4, 8, 16, 32])
def test_radial_small_vs_oracle(ising, L):
    seed = 12
    N = L**3
    with ising.Ising(L, replicas=2, seed=seed) as q:
        for name, s in _states(L, seed).items():
            q.set_spins(s, replica=1)
            C, n = oracle.radial_corr(s)
            S, n2 = oracle.structure_factor(s)
            assert np.array_equal(n, n2)
            for prec in (1, 0):
                res = q.measure_radial(replica=1, precision=prec)
                try:
                    _check_against(res, C, S, n, N, prec, L)
                except AssertionError as e:
                    raise AssertionError(f"{name}, precision {prec}: {e}") from e


def _numpy_radial(s):
    """Independent fp64 reference: numpy FFTs, G rounded to integers, exact bins."""
    L = s.shape[0]
    N = L**3
    F = np.fft.rfftn(s.astype(np.float64))
    P = (F.real**2 + F.imag**2)
    G = np.rint(np.fft.irfftn(P, s=s.shape, axes=(0, 1, 2))).astype(np.int64)
    d = np.arange(L)
    d = np.where(d <= L // 2, d, d - L)
    D = (d[:, None, None] ** 2 + d[None, :, None] ** 2 + d[None, None, :] ** 2).astype(np.int64)
    v = 4 * D
    r = np.floor(np.sqrt(v.astype(np.float64))).astype(np.int64)
    r -= (r * r > v)
    r += ((r + 1) * (r + 1) <= v)
    b = (r + 1) // 2
    nb = oracle.radial_nbins(L)
    n = np.bincount(b.ravel(), minlength=nb)
    sumG = np.zeros(nb, dtype=np.int64)
    np.add.at(sumG, b.ravel(), G.ravel())
    C = np.array([sumG[i] / (float(N) * float(n[i])) if n[i] else 0.0 for i in range(nb)])
    # S over the full spectrum: P of the half spectrum mirrored
    Pf = np.abs(np.fft.fftn(s.astype(np.float64))) ** 2 / N
    S = np.bincount(b.ravel(), weights=Pf.ravel(), minlength=nb) / np.maximum(n, 1)
    return C, S, n


@pytest.mark.parametrize("L", [64, 128, 256])
def test_radial_medium_vs_numpy(ising, L):
    seed = 3
    N = L**3
    with ising.Ising(L, seed=seed) as q:
        q.sweep(5)
        s = q.get_spins(0)
        C, S, n = _numpy_radial(s)
        for prec in (1, 0):
            res = q.measure_radial(precision=prec)
            _check_against(res, C, S, n, N, prec, L)


def test_radial_plain_form(ising):
    L, seed = 32, 5
    with ising.Ising(L, seed=seed, form=ising.FORM_PLAIN) as q:
        q.sweep(2)
        s = q.get_spins(0)
        res = q.measure_radial(precision=1)
    C, n = oracle.radial_corr(s)
    assert np.array_equal(res["C"], C) and np.array_equal(res["count"], n)


def test_radial_scratch_release_and_reuse(ising):
    L, seed = 64, 9
    with ising.Ising(L, seed=seed) as q:
        q.sweep(3)
        a = q.measure_radial(precision=0)
        b = q.measure_radial(precision=1)   # grows the buffer
        q.release_scratch()
        c = q.measure_radial(precision=1)   # allocates again
        d = q.measure_radial(precision=0)   # reuses the larger buffer
    # C sums integers (order-independent); S sums doubles with atomics (last bits may differ)
    assert np.array_equal(b["C"], c["C"]) and np.allclose(b["S"], c["S"], rtol=1e-12, atol=0)
    assert np.array_equal(a["C"], d["C"]) and np.array_equal(a["count"], d["count"])
    assert np.allclose(a["S"], d["S"], rtol=1e-12, atol=0)


def test_radial_rejects_bad_arguments(ising):
    with ising.Ising(16, replicas=2) as q:
        for kw in (dict(replica=2), dict(replica=-1), dict(precision=2)):
            with pytest.raises(ising.IsingError) as e:
                q.measure_radial(**kw)
            assert e.value.status == ising.ISING_EINVAL
        q.sweep(1)  # the context stays usable


def test_radial_L2048(ising):
    L, seed = 2048, 7
    N = L**3
    with ising.Ising(L, seed=seed) as q:
        q.sweep(20)
        r64 = q.measure_radial(precision=1)
        r32 = q.measure_radial(precision=0)
        s = q.get_spins(0)
    n = r64["count"]
    assert n[0] == 1 and n[1] == 18 and n[2] == 62 and int(n.sum()) == N
    assert np.array_equal(r32["count"], n)
    assert r64["inexact"] == 0
    assert r64["C"][0] == 1.0
    # bin 1: the 6 axis lags and the 12 face diagonals (G(-k) = G(k): 9 sums)
    reps = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1), (0, 1, 1), (0, 1, -1)]
    sumG = 2 * sum(oracle.corr_vec(s, *k) for k in reps)
    assert r64["C"][1] == sumG / (float(N) * 18.0)
    M = float(s.sum(dtype=np.int64))
    assert abs(r64["S"][0] - M * M / N) <= 1e-12 * max(1.0, M * M / N)
    assert abs(float((r64["S"] * n).sum()) - N) <= 1e-8 * N
    assert np.all(np.abs(r32["C"] - r64["C"]) <= _tol_C(N, n, U32))
    assert np.all(np.abs(r32["S"] - r64["S"]) <= _tol_S(N, n, U32))
    assert r64["ell"] == oracle.radial_length(L, r64["C"], 0.5)
    assert 1.0 < r64["ell"] < 10.0
