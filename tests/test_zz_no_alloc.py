"""The measurement entry point for callers that cannot allocate device memory.

It must give the same derived observables as ising_measure_ex on the same lattices, on
consecutive calls (its scratch array keeps the previous call's contents, which must not
leak into the next result).  Collected last so that a failure here leaves every other
test already run; it passes alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_measure_ex_on_consecutive_calls():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2305_12161_gb300 import ising

    L, R = 256, 3
    pw = ising.ising_packed_words(L)
    with ising.Ising(L, replicas=R, seed=5) as q:
        for call in range(2):
            q.sweep(3 + 4 * call)  # a different state on each call
            lat = torch.empty(R * pw, dtype=torch.int32, device="cuda")
            for r in range(R):
                q.get_packed(r, out=lat[r * pw:(r + 1) * pw], device=True)
            q.sync()
            _, want = q.measure_ex(c=0.5)
            _, want_conn = q.measure_ex(c=0.4, connected=True)
            out = torch.full((R, 4), float("nan"), dtype=torch.float64, device="cuda")
            assert ising.ising_measure_derived_noalloc(lat, L, R, out, c=0.5) == ising.ISING_OK
            torch.cuda.synchronize()
            np.testing.assert_allclose(out.cpu().numpy(), want, rtol=1e-12, atol=0, equal_nan=True)
            assert ising.ising_measure_derived_noalloc(lat, L, R, out, c=0.4, connected=True) == ising.ISING_OK
            torch.cuda.synchronize()
            np.testing.assert_allclose(out.cpu().numpy(), want_conn, rtol=1e-12, atol=0, equal_nan=True)


@pytest.mark.parametrize("L,R", [(32, 2), (192, 2)])
def test_noalloc_small_and_non_256_sizes_and_flags(L, R):
    # L = 32 (padded words) and L = 192 (not a multiple of 256) take the other M/B and
    # correlation kernels; the flag without correlations must leave l_C undefined (NaN)
    import math

    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2305_12161_gb300 import ising

    pw = ising.ising_packed_words(L)
    with ising.Ising(L, replicas=R, seed=11) as q:
        for call in range(2):
            q.sweep(2 + 5 * call)
            lat = torch.empty(R * pw, dtype=torch.int32, device="cuda")
            for r in range(R):
                q.get_packed(r, out=lat[r * pw:(r + 1) * pw], device=True)
            q.sync()
            _, want = q.measure_ex(c=0.5)
            _, want_nc = q.measure_ex(c=0.5, corr=False)
            out = torch.full((R, 4), float("nan"), dtype=torch.float64, device="cuda")
            # ISING_MEAS_DEVICE is accepted (and implied)
            assert ising.ising_measure_derived_noalloc(lat, L, R, out, c=0.5, device_flag=True) == ising.ISING_OK
            torch.cuda.synchronize()
            np.testing.assert_allclose(out.cpu().numpy(), want, rtol=1e-12, atol=0, equal_nan=True)
            out.fill_(0.0)
            assert ising.ising_measure_derived_noalloc(lat, L, R, out, c=0.5, corr=False) == ising.ISING_OK
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            np.testing.assert_allclose(got, want_nc, rtol=1e-12, atol=0, equal_nan=True)
            assert all(math.isnan(v) for v in got[:, 3])
            np.testing.assert_allclose(got[:, :3], want[:, :3], rtol=1e-12, atol=0)


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2305_12161_gb300 import ising

    L = 2048
    RL = ising.ising_record_len(L)
    too_many = ising.NOALLOC_MAX_RECORD_WORDS // RL + 1
    dummy = torch.empty(16, dtype=torch.int32, device="cuda")
    out = torch.empty((too_many, 4), dtype=torch.float64, device="cuda")
    assert ising.ising_measure_derived_noalloc(dummy, L, too_many, out) == ising.ISING_EINVAL
    assert ising.ising_measure_derived_noalloc(dummy, 96, 1, out) == ising.ISING_EINVAL
