"""GPU <-> oracle parity for the double-checkerboard update (Supp. Methods I A, I B).

Small lattices are replayed whole by the oracle over several sweeps, for block shapes that
span an axis or cut it, with and without x-halo words, one word per thread or four, all
three tie rules and both cycles.  At L=2048 in the launch configuration the benchmark
times (full rows, 16 x 8 blocks) sampled sites of one sweep are recomputed by the oracle
from the state each site saw when it was updated.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ising():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2305_12161_gb300 import ising as m
    return m


def _run_gpu(ising, L, R, seed, block, n, cycle=0, tie=0):
    with ising.Ising(L, replicas=R, seed=seed, tie=tie, cycle=cycle, scheme=ising.SCHEME_DOUBLE,
                     block=block) as q:
        q.sweep(n)
        spins = [q.get_spins(r) for r in range(R)]
        rec = q.measure()
    return spins, rec


def _oracle_block(L, block):
    """The tiling the library uses for `block` (0 = its default)."""
    bx, by, bz = block
    return (bx or L, by or (L if L <= 16 else 16), bz or (L if L <= 16 else 8))


CASES = [
    (4, (0, 0, 0)),        # one block: the whole lattice, wraps inside the block on every axis
    (8, (0, 2, 4)),
    (16, (0, 8, 2)),
    (32, (0, 16, 16)),     # padded one-word rows
    (32, (0, 32, 8)),      # spans y
    (64, (0, 16, 16)),     # one full word per row
    (64, (0, 64, 2)),
    (128, (64, 16, 16)),   # x cut: one word per block row plus x-halo words
    (128, (0, 8, 32)),     # two words per row, one word per thread
    (256, (0, 16, 16)),    # four words per row, four per thread
    (256, (64, 8, 8)),     # x cut, one word per block row
    (256, (128, 16, 4)),   # x cut, two words per block row
    (512, (256, 8, 8)),    # x cut, four words per block row, four per thread with x-halo
    (512, (0, 16, 8)),     # full rows, kernel specialised on the row width
    (256, (0, 256, 2)),    # specialised kernel, block spanning y
]


@pytest.mark.parametrize("L,block", CASES)
@pytest.mark.parametrize("cycle", [0, 1])
def test_dcb_matches_oracle(ising, L, block, cycle):
    R, seed = 2, 17
    n = 3 if L >= 256 else 5
    spins, rec = _run_gpu(ising, L, R, seed, block, n, cycle=cycle)
    ob = _oracle_block(L, block)
    for r in range(R):
        s = oracle.init(L, seed, r)
        oracle.sweeps_dcb(s, 0, n, seed + r, ob, mixed=bool(cycle))
        assert np.array_equal(spins[r], s), (L, block, cycle, r)
        assert np.array_equal(rec[r], oracle.record(s, n))


@pytest.mark.parametrize("tie", [1, 2])
@pytest.mark.parametrize("L,block", [(32, (0, 16, 8)), (256, (0, 16, 16)), (256, (64, 8, 8))])
def test_dcb_tie_rules(ising, L, block, tie):
    seed = 3
    spins, _ = _run_gpu(ising, L, 1, seed, block, 3, tie=tie)
    s = oracle.init(L, seed, 0)
    oracle.sweeps_dcb(s, 0, 3, seed, _oracle_block(L, block), rule=tie)
    assert np.array_equal(spins[0], s)


@pytest.mark.parametrize("block", [(0, 16, 16), (0, 8, 32)])
def test_dcb_L1024_full_rows(ising, block):
    L, seed = 1024, 8
    spins, _ = _run_gpu(ising, L, 1, seed, block, 2, cycle=1)
    s = oracle.init(L, seed, 0)
    oracle.sweeps_dcb(s, 0, 2, seed, _oracle_block(L, block), mixed=True)
    assert np.array_equal(spins[0], s)


def test_ground_state_stays_fixed(ising):
    L = 64
    with ising.Ising(L, scheme=ising.SCHEME_DOUBLE, block=(0, 2, 2)) as q:
        q.set_spins(np.ones((L, L, L), dtype=np.int8))
        q.sweep(3)
        assert (q.get_spins(0) == 1).all()


def test_dcb_continues_across_calls_and_mixed_per_replica(ising):
    L, R, seed = 64, 3, 40
    with ising.Ising(L, replicas=R, seed=seed, cycle=ising.CYCLE_MIXED, scheme=ising.SCHEME_DOUBLE,
                     block=(0, 8, 16)) as q:
        q.sweep(2)
        q.sweep(3)
        got = [q.get_spins(r) for r in range(R)]
    for r in range(R):
        s = oracle.init(L, seed, r)
        oracle.sweeps_dcb(s, 0, 5, seed + r, (L, 8, 16), mixed=True)
        assert np.array_equal(got[r], s), r


@pytest.mark.parametrize("L,kw", [
    (256, dict(block=(0, 3, 16))),      # not a divisor
    (192, dict(block=(0, 64, 16))),     # three blocks along y: one colour would touch itself
    (128, dict(block=(96, 16, 16))),    # x block not a divisor
    (256, dict(block=(32, 16, 16))),    # x block not a multiple of 64
    (256, dict(block=(0, 128, 128))),   # block and halo beyond 227 KB of shared memory
    (256, dict(form=1)),                # plain form
])
def test_dcb_rejects_bad_configurations(ising, L, kw):
    with pytest.raises(ising.IsingError) as e:
        ising.Ising(L, scheme=ising.SCHEME_DOUBLE, **kw)
    assert e.value.status == ising.ISING_EINVAL


def test_dcb_block_spanning_an_axis_is_accepted(ising):
    with ising.Ising(256, scheme=ising.SCHEME_DOUBLE, block=(0, 256, 2)) as q:
        q.sweep(1)
        s = oracle.init(256, 1, 0)
        oracle.sweeps_dcb(s, 0, 1, 1, (256, 256, 2))
        assert np.array_equal(q.get_spins(0), s)


def test_batch_rejects_dcb(ising):
    import ctypes
    o = ising.ising_opts()
    ising.lib().ising_default_opts(ctypes.byref(o))
    o.scheme = ising.SCHEME_DOUBLE
    h = ctypes.c_void_p()
    Ls = (ctypes.c_int * 1)(64)
    Rs = (ctypes.c_int * 1)(1)
    Ss = (ctypes.c_uint64 * 1)(1)
    st = ising.lib().ising_batch_create(ctypes.byref(h), 1, ctypes.cast(Ls, ctypes.c_void_p),
                                        ctypes.cast(Rs, ctypes.c_void_p), ctypes.cast(Ss, ctypes.c_void_p),
                                        ctypes.byref(o))
    assert st == ising.ISING_EINVAL


# ---------------------------------------------------------------------------------------
# L = 2048, the benchmark's tiling: one sweep, sampled sites recomputed by the oracle.

def _block_of(x, y, z, block, L):
    bx, by, bz = block
    nbx, nby = L // bx, L // by
    return (x // bx) + nbx * ((y // by) + nby * (z // bz)), ((x // bx) + (y // by) + (z // bz)) & 1


def _check_dcb_sweep(A, B, L, t, S, block, mixed, rng, n=60_000):
    """B must be one double-checkerboard sweep of A at sweep index t.  A site saw, when it
    was updated, its own old value (A); neighbours in its own block from before the block
    started (A) if it is on the block's first parity, else after (B); neighbours in other
    blocks before (A) if its colour went first, else after (B)."""
    Af, Bf = A.reshape(-1), B.reshape(-1)
    first_colour = oracle.mixed_order(S, t) if mixed else 0
    z = rng.integers(0, L, n)
    y = rng.integers(0, L, n)
    x = rng.integers(0, L, n)
    idx = np.unique(x + L * (y + L * z))
    x, y, z = idx % L, (idx // L) % L, idx // (L * L)
    beta, colour = _block_of(x, y, z, block, L)
    par = (x + y + z) & 1
    if mixed:
        f0 = np.array([oracle.dcb_fine_first(S, t, int(b)) for b in beta])
    else:
        f0 = np.ones_like(par)
    second_fine = par != f0
    second_colour = colour != first_colour
    offs = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    checked = 0
    for sc in (False, True):
        for sf in (False, True):
            sel = (second_colour == sc) & (second_fine == sf)
            xs, ys, zs, bs = x[sel], y[sel], z[sel], beta[sel]
            pos, src = [idx[sel]], [np.zeros(sel.sum(), dtype=bool)]  # own value: old
            for dx, dy, dz in offs:
                nx, ny, nz = (xs + dx) % L, (ys + dy) % L, (zs + dz) % L
                nb, _ = _block_of(nx, ny, nz, block, L)
                same = nb == bs
                pos.append(nx + L * (ny + L * nz))
                src.append(np.where(same, sf, sc))  # True: the value after the sweep
            P = np.concatenate(pos)
            Sr = np.concatenate(src)
            # drop sampled sites whose required neighbour values clash with another's
            order = np.argsort(P, kind="stable")
            Ps, Ss = P[order], Sr[order]
            clash_pos = np.unique(Ps[1:][(Ps[1:] == Ps[:-1]) & (Ss[1:] != Ss[:-1])])
            m = sel.sum()
            bad = np.isin(P, clash_pos).reshape(7, m).any(axis=0)
            keep = ~bad
            P7 = P.reshape(7, m)[:, keep]
            S7 = Sr.reshape(7, m)[:, keep]
            sites = P7[0]
            want = Bf[sites].copy()
            upd = P7[S7]
            saved = Af[upd].copy()
            Af[upd] = Bf[upd]
            try:
                for q in (0, 1):
                    qs = sites[((sites % L) + (sites // L) % L + sites // (L * L)) % 2 == q]
                    if len(qs):
                        got = oracle.update_sites(A, q, t, S, qs)
                        assert np.array_equal(got, Bf[qs]), (sc, sf, q)
            finally:
                Af[upd] = saved
            checked += len(sites)
            assert len(sites) > 0.9 * m
    assert checked > 0.9 * len(idx)


@pytest.mark.parametrize("mixed", [False, True])
def test_dcb_L2048_sampled(ising, mixed):
    L, seed = 2048, 5
    block = (L, 16, 8)
    rng = np.random.default_rng(11 + int(mixed))
    cycle = ising.CYCLE_MIXED if mixed else ising.CYCLE_01
    with ising.Ising(L, seed=seed, cycle=cycle, scheme=ising.SCHEME_DOUBLE) as q:
        A = q.get_spins(0)
        # the T = infinity start is the checkerboard's
        i = rng.integers(0, L**3, 2000)
        x, y, z = i % L, (i // L) % L, i // (L * L)
        for k in range(0, 2000, 200):
            h = (x[k] >> 1) + (L // 2) * (y[k] + L * z[k])
            bit = oracle.rng_bit(seed, 0, 2 + int((x[k] + y[k] + z[k]) & 1), int(h))
            assert A.reshape(-1)[i[k]] == (1 if bit else -1)
        q.sweep(1)
        B = q.get_spins(0)
        _check_dcb_sweep(A, B, L, 0, seed, block, mixed, rng)
        q.sweep(40)
        A = q.get_spins(0)
        q.sweep(1)
        B = q.get_spins(0)
        _check_dcb_sweep(A, B, L, 41, seed, block, mixed, rng)
