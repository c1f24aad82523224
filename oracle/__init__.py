"""CPU oracle for the zero-temperature checkerboard quench (arXiv:2305.12161).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The product library (``paper_2305_12161_gb300``) never imports it and shares no code
with it.

The arithmetic lives in ``ising_oracle.c`` (one byte per spin, plain loops, every
function citing the passage of the paper it follows); this module compiles it with the
host C compiler and exposes it through ``ctypes``.

Spin arrays are ``numpy.int8`` of shape ``(L, L, L)`` indexed ``[z, y, x]``, so that the
flat C-order index is ``x + L*(y + L*z)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ising_oracle.c")
_LIB = os.path.join(_HERE, "libising_oracle.so")
_lock = threading.Lock()
_lib = None

TIE_GLAUBER, TIE_ALWAYS, TIE_NEVER = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile ``libising_oracle.so`` (with OpenMP when the compiler has it)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cc = os.environ.get("CC", "gcc")
    base = [cc, "-O3", "-std=c11", "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i8p = ctypes.POINTER(ctypes.c_int8)
            f64p = ctypes.POINTER(ctypes.c_double)
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_set_threads.restype = ctypes.c_int
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_philox4x32_10.restype = None
            L.orc_rng_bit.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64]
            L.orc_rng_bit.restype = ctypes.c_int
            L.orc_init.argtypes = [ctypes.c_int, ctypes.c_uint64, i8p]
            L.orc_init.restype = None
            L.orc_half_sweep.argtypes = [ctypes.c_int, i8p, ctypes.c_int, ctypes.c_uint32,
                                         ctypes.c_uint64, ctypes.c_int, i64p, i64p]
            L.orc_half_sweep.restype = ctypes.c_int64
            L.orc_sweeps.argtypes = [ctypes.c_int, i8p, ctypes.c_uint32, ctypes.c_int64,
                                     ctypes.c_uint64, ctypes.c_int]
            L.orc_sweeps.restype = None
            L.orc_record_len.argtypes = [ctypes.c_int]
            L.orc_record_len.restype = ctypes.c_int64
            L.orc_record.argtypes = [ctypes.c_int, i8p, ctypes.c_int64, i64p]
            L.orc_record.restype = None
            L.orc_update_sites.argtypes = [ctypes.c_int, i8p, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64,
                                           ctypes.c_int, i64p, ctypes.c_int64, i8p]
            L.orc_update_sites.restype = None
            L.orc_magnetisation_bonds.argtypes = [ctypes.c_int, i8p, i64p, i64p]
            L.orc_magnetisation_bonds.restype = None
            L.orc_corr_lag.argtypes = [ctypes.c_int, i8p, ctypes.c_int64, i64p]
            L.orc_corr_lag.restype = None
            L.orc_corr_lags.argtypes = [ctypes.c_int, i8p, i64p, ctypes.c_int64, i64p]
            L.orc_corr_lags.restype = None
            L.orc_menger_member.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int]
            L.orc_menger_member.restype = ctypes.c_int
            L.orc_menger_tile_sign.argtypes = [ctypes.c_uint64, ctypes.c_int64]
            L.orc_menger_tile_sign.restype = ctypes.c_int
            L.orc_init_menger.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int, i8p]
            L.orc_init_menger.restype = None
            L.orc_mixed_order.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
            L.orc_mixed_order.restype = ctypes.c_int
            L.orc_sweeps_mixed.argtypes = [ctypes.c_int, i8p, ctypes.c_uint32, ctypes.c_int64,
                                           ctypes.c_uint64, ctypes.c_int]
            L.orc_sweeps_mixed.restype = None
            L.orc_rsf_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_int64, i64p,
                                       ctypes.POINTER(ctypes.c_int)]
            L.orc_rsf_draw.restype = None
            L.orc_sweeps_rsf.argtypes = [ctypes.c_int, i8p, ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint64,
                                         ctypes.c_int, i64p, i64p]
            L.orc_sweeps_rsf.restype = ctypes.c_int64
            L.orc_dcb_valid.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.orc_dcb_valid.restype = ctypes.c_int
            L.orc_dcb_fine_first.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64]
            L.orc_dcb_fine_first.restype = ctypes.c_int
            L.orc_sweeps_dcb.argtypes = [ctypes.c_int, i8p, ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint64,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.orc_sweeps_dcb.restype = ctypes.c_int
            L.orc_isqrt.argtypes = [ctypes.c_int64]
            L.orc_isqrt.restype = ctypes.c_int64
            L.orc_radial_bin.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
            L.orc_radial_bin.restype = ctypes.c_int64
            L.orc_radial_nbins.argtypes = [ctypes.c_int]
            L.orc_radial_nbins.restype = ctypes.c_int64
            L.orc_corr3d.argtypes = [ctypes.c_int, i8p, i64p]
            L.orc_corr3d.restype = None
            L.orc_corr_vec.argtypes = [ctypes.c_int, i8p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
            L.orc_corr_vec.restype = ctypes.c_int64
            L.orc_radial_corr.argtypes = [ctypes.c_int, i8p, f64p, i64p]
            L.orc_radial_corr.restype = None
            L.orc_structure_factor.argtypes = [ctypes.c_int, i8p, f64p, i64p]
            L.orc_structure_factor.restype = None
            L.orc_radial_length.argtypes = [ctypes.c_int, f64p, ctypes.c_double, ctypes.c_double]
            L.orc_radial_length.restype = ctypes.c_double
            L.orc_derived.argtypes = [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_int, f64p]
            L.orc_derived.restype = None
            _lib = L
    return _lib


def _p(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _check_lattice(s: np.ndarray) -> int:
    if s.dtype != np.int8 or s.ndim != 3 or not (s.shape[0] == s.shape[1] == s.shape[2]):
        raise ValueError("spins must be an int8 array of shape (L, L, L)")
    if not s.flags.c_contiguous:
        raise ValueError("spins must be C-contiguous")
    return s.shape[0]


def set_threads(n: int) -> int:
    """Set the OpenMP thread count (<= 0 keeps the current); returns threads in use."""
    return int(lib().orc_set_threads(int(n)))


def philox4x32_10(ctr, key):
    """Philox4x32-10 of a 4-word counter and a 2-word key; returns four uint32."""
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), _p(o, ctypes.c_uint32))
    return [int(v) for v in o]


def rng_bit(S: int, t: int, phase: int, h: int) -> int:
    return int(lib().orc_rng_bit(S % 2**64, t, phase, h))


def init(L: int, seed: int, replica: int = 0) -> np.ndarray:
    """T = infinity start of replica ``replica`` of a run seeded ``seed``."""
    s = np.empty((L, L, L), dtype=np.int8)
    lib().orc_init(L, (seed + replica) % 2**64, _p(s, ctypes.c_int8))
    return s


def half_sweep(s: np.ndarray, q: int, t: int, S: int, rule: int = TIE_GLAUBER):
    """One half-sweep in place; returns (flips, incremental dB, incremental dM)."""
    L = _check_lattice(s)
    dB = ctypes.c_int64(0)
    dM = ctypes.c_int64(0)
    f = lib().orc_half_sweep(L, _p(s, ctypes.c_int8), q, t, S % 2**64, rule,
                             ctypes.byref(dB), ctypes.byref(dM))
    return int(f), int(dB.value), int(dM.value)


def sweeps(s: np.ndarray, t0: int, n: int, S: int, rule: int = TIE_GLAUBER) -> None:
    """``n`` MCS in place, starting at completed-sweep count ``t0``."""
    L = _check_lattice(s)
    lib().orc_sweeps(L, _p(s, ctypes.c_int8), t0, n, S % 2**64, rule)


def menger_member(a: int, b: int, c: int, k: int) -> bool:
    return bool(lib().orc_menger_member(a, b, c, k))


def menger_tile_sign(S: int, T: int) -> int:
    return int(lib().orc_menger_tile_sign(S % 2**64, T))


def init_menger(L: int, seed: int, k: int, replica: int = 0) -> np.ndarray:
    """Menger-sponge start of iteration k (tiles of side 3^k, random sign per tile)."""
    s = np.empty((L, L, L), dtype=np.int8)
    lib().orc_init_menger(L, (seed + replica) % 2**64, k, _p(s, ctypes.c_int8))
    return s


def mixed_order(S: int, t: int) -> int:
    """1 when sweep t of the mixed cycle updates blue (q = 1) first."""
    return int(lib().orc_mixed_order(S % 2**64, t))


def sweeps_mixed(s: np.ndarray, t0: int, n: int, S: int, rule: int = TIE_GLAUBER) -> None:
    L = _check_lattice(s)
    lib().orc_sweeps_mixed(L, _p(s, ctypes.c_int8), t0, n, S % 2**64, rule)


def rsf_draw(S: int, t: int, k: int, N: int):
    """(site, zero-energy bit) of step k of rsf sweep t."""
    i = ctypes.c_int64(0)
    b = ctypes.c_int(0)
    lib().orc_rsf_draw(S % 2**64, t, k, N, ctypes.byref(i), ctypes.byref(b))
    return int(i.value), int(b.value)


def sweeps_rsf(s: np.ndarray, t0: int, n: int, S: int, rule: int = TIE_GLAUBER):
    """``n`` random-site-flip sweeps in place (N sequential proposals each); returns
    (flips, incremental dB, incremental dM).  Sequential: releases the GIL while it runs,
    so independent lattices can be advanced from several Python threads."""
    L = _check_lattice(s)
    dB = ctypes.c_int64(0)
    dM = ctypes.c_int64(0)
    f = lib().orc_sweeps_rsf(L, _p(s, ctypes.c_int8), t0, n, S % 2**64, rule, ctypes.byref(dB), ctypes.byref(dM))
    return int(f), int(dB.value), int(dM.value)


def dcb_valid(L: int, block) -> bool:
    """True when blocks of ``block = (bx, by, bz)`` sites tile an L^3 lattice as a double checkerboard."""
    bx, by, bz = block
    return bool(lib().orc_dcb_valid(L, bx, by, bz))


def dcb_fine_first(S: int, t: int, beta: int) -> int:
    """Parity of the sites block ``beta`` updates first in sweep t of the mixed double checkerboard."""
    return int(lib().orc_dcb_fine_first(S % 2**64, t, beta))


def sweeps_dcb(s: np.ndarray, t0: int, n: int, S: int, block, rule: int = TIE_GLAUBER,
               mixed: bool = False) -> None:
    """n double-checkerboard sweeps (Supp. Methods I A; mixed cycle per I B) with blocks ``(bx, by, bz)``."""
    L = _check_lattice(s)
    bx, by, bz = block
    if lib().orc_sweeps_dcb(L, _p(s, ctypes.c_int8), t0, n, S % 2**64, rule, bx, by, bz, int(bool(mixed))) != 0:
        raise ValueError(f"blocks {block} do not tile L={L} as a double checkerboard")


def isqrt(n: int) -> int:
    return int(lib().orc_isqrt(n))


def radial_bin(L: int, x: int, y: int, z: int) -> int:
    """Radial bin round(|v|) of the lag or mode vector with indices (x, y, z) (minimal images)."""
    return int(lib().orc_radial_bin(L, x, y, z))


def radial_nbins(L: int) -> int:
    return int(lib().orc_radial_nbins(L))


def corr3d(s: np.ndarray) -> np.ndarray:
    """G(k) = sum_i s_i s_(i+k) for every lag, int64 array [kz, ky, kx] (brute force)."""
    L = _check_lattice(s)
    G = np.empty((L, L, L), dtype=np.int64)
    lib().orc_corr3d(L, _p(s, ctypes.c_int8), _p(G, ctypes.c_int64))
    return G


def corr_vec(s: np.ndarray, dx: int, dy: int, dz: int) -> int:
    """G(k) = sum_i s_i s_(i+k) for one lag vector k = (dx, dy, dz)."""
    L = _check_lattice(s)
    return int(lib().orc_corr_vec(L, _p(s, ctypes.c_int8), dx, dy, dz))


def radial_corr(s: np.ndarray):
    """(C(r), n_r): radially averaged G(k)/N and the number of lag vectors per bin."""
    L = _check_lattice(s)
    nb = radial_nbins(L)
    C = np.empty(nb, dtype=np.float64)
    n = np.empty(nb, dtype=np.int64)
    lib().orc_radial_corr(L, _p(s, ctypes.c_int8), _p(C, ctypes.c_double), _p(n, ctypes.c_int64))
    return C, n


def structure_factor(s: np.ndarray):
    """(S(b), n_b): radially averaged |DFT(s)|^2 / N by the direct sum, and modes per bin."""
    L = _check_lattice(s)
    nb = radial_nbins(L)
    S = np.empty(nb, dtype=np.float64)
    n = np.empty(nb, dtype=np.int64)
    lib().orc_structure_factor(L, _p(s, ctypes.c_int8), _p(S, ctypes.c_double), _p(n, ctypes.c_int64))
    return S, n


def radial_length(L: int, C: np.ndarray, c: float = 0.5, sub: float = 0.0) -> float:
    """Crossing of the radial C(r) with c for r <= L/2 (linear interpolation; NaN if none)."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    return float(lib().orc_radial_length(L, _p(C, ctypes.c_double), c, sub))


def record_len(L: int) -> int:
    return int(lib().orc_record_len(L))


def record(s: np.ndarray, t: int = 0) -> np.ndarray:
    """Integer record [t, M, B, D_x(0..L/2), D_y(0..L/2), D_z(0..L/2)]."""
    L = _check_lattice(s)
    rec = np.zeros(record_len(L), dtype=np.int64)
    lib().orc_record(L, _p(s, ctypes.c_int8), t, _p(rec, ctypes.c_int64))
    return rec


def update_sites(s: np.ndarray, q: int, t: int, S: int, sites: np.ndarray, rule: int = TIE_GLAUBER) -> np.ndarray:
    """New values the half-sweep (q, t) gives the listed sites (linear indices on q)."""
    L = _check_lattice(s)
    idx = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty(idx.size, dtype=np.int8)
    lib().orc_update_sites(L, _p(s, ctypes.c_int8), q, t, S % 2**64, rule, _p(idx, ctypes.c_int64), idx.size,
                           _p(out, ctypes.c_int8))
    return out


def magnetisation_bonds(s: np.ndarray):
    """(M, B) of one configuration."""
    L = _check_lattice(s)
    M = ctypes.c_int64(0)
    B = ctypes.c_int64(0)
    lib().orc_magnetisation_bonds(L, _p(s, ctypes.c_int8), ctypes.byref(M), ctypes.byref(B))
    return int(M.value), int(B.value)


def corr_lag(s: np.ndarray, r: int) -> np.ndarray:
    """[D_x(r), D_y(r), D_z(r)] of one configuration."""
    L = _check_lattice(s)
    out = np.zeros(3, dtype=np.int64)
    lib().orc_corr_lag(L, _p(s, ctypes.c_int8), r, _p(out, ctypes.c_int64))
    return out


def corr_lags(s: np.ndarray, lags) -> np.ndarray:
    """[n, 3] array of [D_x(r), D_y(r), D_z(r)] for the lags r (each in [0, L)), counted
    line by line (the counting ``record`` uses)."""
    L = _check_lattice(s)
    lg = np.ascontiguousarray(lags, dtype=np.int64)
    if lg.ndim != 1 or (lg.size and (lg.min() < 0 or lg.max() >= L)):
        raise ValueError("lags must be a 1-d list of values in [0, L)")
    out = np.zeros((lg.size, 3), dtype=np.int64)
    lib().orc_corr_lags(L, _p(s, ctypes.c_int8), _p(lg, ctypes.c_int64), lg.size, _p(out, ctypes.c_int64))
    return out


def derived(L: int, rec: np.ndarray, c: float = 0.5, connected: bool = False) -> np.ndarray:
    """[e, m, l_E, l_C] from one record (double precision)."""
    rec = np.ascontiguousarray(rec, dtype=np.int64)
    if rec.size != record_len(L):
        raise ValueError("record length does not match L")
    out = np.zeros(4, dtype=np.float64)
    lib().orc_derived(L, _p(rec, ctypes.c_int64), c, int(bool(connected)), _p(out, ctypes.c_double))
    return out


def run(L: int, seed: int, replica: int, times, rule: int = TIE_GLAUBER, keep_spins: bool = False):
    """Quench one replica and record at t = 0 and at every t in ``times`` (increasing).

    Returns (records [len(times)+1, record_len], spins or None)."""
    S = (seed + replica) % 2**64
    s = init(L, seed, replica)
    recs = [record(s, 0)]
    spins = [s.copy()] if keep_spins else None
    t = 0
    for tk in times:
        sweeps(s, t, tk - t, S, rule)
        t = tk
        recs.append(record(s, t))
        if keep_spins:
            spins.append(s.copy())
    return np.stack(recs), spins
