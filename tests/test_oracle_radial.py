"""Pins for the oracle's three-dimensional correlation, structure factor and radial bins (no GPU).

* Integer square root against Python's math.isqrt; every bin satisfies the nearest-integer
  condition max(0, b - 1/2)^2 <= |v|^2 < (b + 1/2)^2 exactly; bin counts against a numpy
  enumeration (bins 0 and 1 hold 1 and 18 vectors).
* G(k): G(0) = N, the sum over all lags is M^2, G(-k) = G(k), the axis lags equal
  N - 2 D_a(r) of the separately pinned axis sums, and the whole array equals numpy's
  inverse FFT of |FFT(s)|^2 (Eq. 3 with a library FFT).
* S: numpy's |FFT(s)|^2 / N in the same bins; Parseval (sum of S over all modes = N);
  S(0) = M^2 / N.
* Closed forms: uniform state (C = 1, S only at k = 0), Neel state (G = N (-1)^(kx+ky+kz),
  S only at the corner mode), flat stripes (triangle-wave G along the stripe normal).
* The radial crossing rule on hand-made C arrays.
* The single-lag G equals the full array's entry for every lag (negative components too).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2305_12161_gb300 import inputs


def test_isqrt():
    vals = list(range(0, 2000)) + [k * k + d for k in (46340, 65535, 3547, 7094) for d in (-1, 0, 1)]
    vals += [3 * 4096**2, 3 * 2048**2 * 4, 2**40 + 12345]
    for v in vals:
        if v >= 0:
            assert oracle.isqrt(v) == math.isqrt(v), v


@pytest.mark.parametrize("L", [4, 8, 12])
def test_bins_nearest_integer_and_counts(L):
    idx = np.arange(L)
    d = np.where(idx <= L // 2, idx, idx - L)
    counts = {}
    for x in range(L):
        for y in range(L):
            for z in range(L):
                D = int(d[x] ** 2 + d[y] ** 2 + d[z] ** 2)
                b = oracle.radial_bin(L, x, y, z)
                lo = (2 * b - 1) ** 2 if b > 0 else 0
                assert lo <= 4 * D < (2 * b + 1) ** 2, (x, y, z, b)
                counts[b] = counts.get(b, 0) + 1
    nb = oracle.radial_nbins(L)
    assert max(counts) == nb - 1
    s = oracle.init(L, 1)
    _, n = oracle.radial_corr(s)
    assert [counts.get(b, 0) for b in range(nb)] == list(n)
    assert n[0] == 1 and n[1] == 18 and n.sum() == L**3


@pytest.mark.parametrize("L,seed", [(4, 1), (8, 2), (12, 3)])
def test_corr3d_identities_and_fft(L, seed):
    s = oracle.init(L, seed)
    N = L**3
    G = oracle.corr3d(s)  # [kz, ky, kx]
    M = int(s.astype(np.int64).sum())
    assert G[0, 0, 0] == N
    assert int(G.sum()) == M * M
    neg = (-np.arange(L)) % L
    assert np.array_equal(G, G[np.ix_(neg, neg, neg)])
    for r in range(L // 2 + 1):
        D = oracle.corr_lag(s, r)  # D_x, D_y, D_z
        assert G[0, 0, r] == N - 2 * D[0]
        assert G[0, r, 0] == N - 2 * D[1]
        assert G[r, 0, 0] == N - 2 * D[2]
    F = np.fft.fftn(s.astype(np.float64))
    G_fft = np.fft.ifftn(np.abs(F) ** 2).real  # sum_i s_i s_(i+k) up to the sign of k
    assert np.allclose(G_fft, G, atol=1e-9 * N)


@pytest.mark.parametrize("L,seed", [(4, 5), (8, 6), (12, 7)])
def test_structure_factor_against_numpy_fft(L, seed):
    s = oracle.init(L, seed)
    N = L**3
    S, n = oracle.structure_factor(s)
    P = np.abs(np.fft.fftn(s.astype(np.float64))) ** 2 / N
    nb = oracle.radial_nbins(L)
    acc = np.zeros(nb)
    cnt = np.zeros(nb, dtype=np.int64)
    for z in range(L):
        for y in range(L):
            for x in range(L):
                b = oracle.radial_bin(L, x, y, z)
                acc[b] += P[z, y, x]
                cnt[b] += 1
    assert np.array_equal(cnt, n)
    assert np.allclose(S, acc / np.maximum(cnt, 1), rtol=1e-10, atol=1e-10)
    assert abs(float((S * n).sum()) - N) < 1e-8 * N           # Parseval
    M = float(s.astype(np.int64).sum())
    assert abs(S[0] - M * M / N) < 1e-9 * N


def test_uniform_and_neel_closed_forms():
    L = 8
    N = L**3
    u = inputs.uniform_state(L, 1)
    C, n = oracle.radial_corr(u)
    assert np.allclose(C, 1.0)
    S, _ = oracle.structure_factor(u)
    assert abs(S[0] - N) < 1e-9 and np.allclose(S[1:], 0.0, atol=1e-9)
    neel = inputs.neel_state(L)
    G = oracle.corr3d(neel)
    z, y, x = np.indices((L, L, L))
    assert np.array_equal(G, N * (-1) ** (x + y + z))
    S, n = oracle.structure_factor(neel)
    bc = oracle.radial_bin(L, L // 2, L // 2, L // 2)
    want = np.zeros_like(S)
    want[bc] = N / n[bc]
    assert np.allclose(S, want, atol=1e-9)


@pytest.mark.parametrize("w", [2, 3])
def test_stripes_triangle_wave(w):
    L = 12
    N = L**3
    s = inputs.stripe_state(L, w, "x")
    G = oracle.corr3d(s)
    for kx in range(L):
        m = kx % (2 * w)
        d = min(m, 2 * w - m)
        assert (G[:, :, kx] == N * (w - 2 * d) // w).all(), kx


def test_radial_length_rule():
    L = 8
    C = np.array([1.0, 0.8, 0.4, 0.2, 0.1, 0.05, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0])
    assert oracle.radial_length(L, C, 0.5) == pytest.approx(1.75)
    assert oracle.radial_length(L, C, 0.8) == pytest.approx(1.0)  # C(1) >= c > C(2)
    assert math.isnan(oracle.radial_length(L, C, 0.01))  # crosses only beyond L/2
    assert oracle.radial_length(L, C, 0.3, sub=0.2) == pytest.approx(1.75)


def test_corr_vec_matches_corr3d():
    L = 8
    s = oracle.init(L, 9)
    G = oracle.corr3d(s)
    for kz in range(L):
        for ky in range(L):
            for kx in range(L):
                assert oracle.corr_vec(s, kx, ky, kz) == G[kz, ky, kx]
    assert oracle.corr_vec(s, -1, 2, -3) == G[(-3) % L, 2, (-1) % L]
