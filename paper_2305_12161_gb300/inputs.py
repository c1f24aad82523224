"""Seeded synthetic inputs shared by the library's users, its tests and the oracle's tests.

Nothing here computes any part of the quench: this module only produces the inputs a
run is given — measurement schedules, synthetic lattice states with known structure and
the serving request trace.  It holds none of the method's arithmetic, so both the CUDA
path and the CPU oracle may be fed from it.

Lattice arrays are ``numpy.int8`` of shape ``(L, L, L)`` indexed ``[z, y, x]`` with
values +1 / -1.
"""
from __future__ import annotations

import math

import numpy as np


def log_schedule(t_max: int, K: int) -> list[int]:
    """K strictly increasing measurement times from 1 to ``t_max``, log-spaced.

    t_k = round(t_max ** (k / (K-1))) for k = 0..K-1; a clash with the previous point
    is pushed up by one, and if that pushes past ``t_max`` the points are pulled down
    from the back so that the last one is exactly ``t_max``.  The initial state (t = 0)
    is recorded in addition to these points by every caller.
    """
    if K < 1 or t_max < K:
        raise ValueError("need 1 <= K <= t_max")
    if K == 1:
        return [int(t_max)]
    ts: list[int] = []
    for k in range(K):
        v = int(math.floor(t_max ** (k / (K - 1)) + 0.5))
        if ts:
            v = max(v, ts[-1] + 1)
        ts.append(v)
    ts[-1] = int(t_max)
    for k in range(K - 2, -1, -1):
        if ts[k] >= ts[k + 1]:
            ts[k] = ts[k + 1] - 1
    return ts


def uniform_state(L: int, sign: int = 1) -> np.ndarray:
    """All spins +1 (sign=1) or -1 (sign=-1): a ground state."""
    return np.full((L, L, L), 1 if sign > 0 else -1, dtype=np.int8)


def neel_state(L: int) -> np.ndarray:
    """s = (-1)^(x+y+z): even sites +1, odd sites -1 (every bond broken)."""
    z, y, x = np.indices((L, L, L))
    return np.where((x + y + z) % 2 == 0, 1, -1).astype(np.int8)


def stripe_state(L: int, width: int, axis: str = "x", phase: int = 0) -> np.ndarray:
    """Flat slabs of alternating sign, each ``width`` sites thick along ``axis``."""
    z, y, x = np.indices((L, L, L))
    coord = {"x": x, "y": y, "z": z}[axis]
    return np.where(((coord + phase) // width) % 2 == 0, 1, -1).astype(np.int8)


def cube_defect_state(L: int, size: int, origin=(0, 0, 0), sign: int = -1) -> np.ndarray:
    """All spins -sign except a size^3 cube of spins ``sign`` at ``origin`` (x, y, z)."""
    s = uniform_state(L, -sign)
    ox, oy, oz = origin
    for dz in range(size):
        for dy in range(size):
            for dx in range(size):
                s[(oz + dz) % L, (oy + dy) % L, (ox + dx) % L] = sign
    return s


def random_state(L: int, seed: int, p_up: float = 0.5) -> np.ndarray:
    """I.i.d. spins from numpy's generator (independent of the quench's own Philox start)."""
    rng = np.random.default_rng(seed)
    return np.where(rng.random((L, L, L)) < p_up, 1, -1).astype(np.int8)


def serving_trace(n_requests: int, seed: int = 0, rate_hz: float = 20.0,
                  sizes=(64, 128, 256, 512, 1024), t_log10=(3.0, 5.0),
                  replicas=(1, 16)) -> list[dict]:
    """Poisson stream of quench requests: arrival time (s), L drawn uniformly from
    ``sizes`` (log-uniform in L on that set), t_max = round(10**U[a, b]) MCS, replicas
    uniform on [lo, hi], and a per-request seed."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        out.append({
            "id": i,
            "arrival_s": t,
            "L": int(sizes[rng.integers(len(sizes))]),
            "t_max": int(round(10 ** rng.uniform(*t_log10))),
            "replicas": int(rng.integers(replicas[0], replicas[1] + 1)),
            "seed": int(rng.integers(1, 2**31)),
        })
    return out
