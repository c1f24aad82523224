"""C-ABI checks that need no GPU: the library builds, loads and exports every function
declared in include/ising.h, and its host-only entry points behave as documented."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ising_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2305_12161_gb300 import _build, ising
    _build.build()
    return ising.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared("ising.h")
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_record_and_packed_sizes(lib):
    from paper_2305_12161_gb300 import ising
    assert ising.ising_record_len(32) == 3 + 3 * 17
    assert ising.ising_record_len(2048) == 3 + 3 * 1025
    assert ising.ising_record_len(7) == -1 and ising.ising_record_len(2) == -1
    assert ising.ising_packed_words(2048) == 2 * 2048 * 2048 * 32
    assert ising.ising_packed_words(32) == 2 * 32 * 32
    assert ising.ising_packed_words(4) == 2 * 16
    assert ising.ising_packed_words(96) == -1  # packed form: multiples of 64 or 4..32


def test_radial_bins_match_the_oracle(lib):
    import oracle
    from paper_2305_12161_gb300 import ising
    for L in (4, 6, 8, 16, 32, 64, 256, 2048, 4096):
        assert ising.ising_radial_bins(L) == oracle.radial_nbins(L), L
    assert ising.ising_radial_bins(2048) == 1775
    assert ising.ising_radial_bins(7) == -1 and ising.ising_radial_bins(2) == -1


def test_strerror_and_variants(lib):
    from paper_2305_12161_gb300 import ising
    for code in range(0, -7, -1):
        assert isinstance(ising.ising_strerror(code), str) and ising.ising_strerror(code)
    assert ising.ising_variants() == [ising.VARIANT_WORD, ising.VARIANT_ZMARCH, ising.VARIANT_ZFAST,
                                     ising.VARIANT_ZDEEP, ising.VARIANT_ZFUSE]


def test_create_rejects_bad_arguments_before_touching_a_device(lib):
    from paper_2305_12161_gb300 import ising
    h = ctypes.c_void_p()
    for L, R in ((7, 1), (2, 1), (96, 1), (64, 0), (8192, 1)):
        assert lib.ising_create(ctypes.byref(h), L, R, 1) == ising.ISING_EINVAL
        assert h.value is None
    assert lib.ising_create(None, 64, 1, 1) == ising.ISING_EINVAL
    # sweep-kernel configurations no kernel can run
    bad = (dict(L=64, variant=9), dict(L=128, variant=ising.VARIANT_ZFUSE), dict(L=2048, variant=ising.VARIANT_ZFUSE,
           depth=7), dict(L=2048, variant=ising.VARIANT_ZFUSE, tile_z=3), dict(L=2048, variant=ising.VARIANT_ZFAST,
           tile_z=48), dict(L=1024, variant=ising.VARIANT_ZDEEP, depth=5), dict(L=96 * 4, variant=ising.VARIANT_ZFAST),
           dict(L=2048, variant=ising.VARIANT_ZFUSE, depth=33), dict(L=2048, variant=ising.VARIANT_ZFUSE, depth=64),
           dict(L=256, pdl=2), dict(L=256, variant=ising.VARIANT_ZFAST, pdl=-1))
    for kw in bad:
        o = ising.ising_opts()
        lib.ising_default_opts(ctypes.byref(o))
        L = kw.pop("L")
        for k, v in kw.items():
            setattr(o, k, v)
        assert lib.ising_create_ex(ctypes.byref(h), L, 1, 1, ctypes.byref(o)) == ising.ISING_EINVAL, (L, kw)
        assert h.value is None
    # valid ones pass the checks: without a device the call then fails on the device (with one
    # it succeeds)
    good = (dict(L=64), dict(L=256, variant=ising.VARIANT_ZFAST, tile_z=8), dict(L=2048, variant=ising.VARIANT_ZFUSE,
            tile_z=32, depth=3), dict(L=1024, variant=ising.VARIANT_ZFUSE, tile_z=32, depth=10),
            dict(L=512, variant=ising.VARIANT_ZDEEP, tile_z=16, depth=4), dict(L=2048, variant=ising.VARIANT_ZFUSE,
            tile_z=64, depth=27), dict(L=256, variant=ising.VARIANT_ZFAST, pdl=0),
            dict(L=256, variant=ising.VARIANT_ZFUSE, tile_z=8, depth=18, pdl=0))
    for kw in good:
        o = ising.ising_opts()
        lib.ising_default_opts(ctypes.byref(o))
        L = kw.pop("L")
        for k, v in kw.items():
            setattr(o, k, v)
        st = lib.ising_create_ex(ctypes.byref(h), L, 1, 1, ctypes.byref(o))
        assert st in (ising.ISING_OK, ising.ISING_ECUDA), (L, kw, st)
        if st == ising.ISING_OK:
            lib.ising_destroy(h)
        h = ctypes.c_void_p()
    # NULL-safe destroy and NULL-context calls
    assert lib.ising_destroy(None) == ising.ISING_OK
    assert lib.ising_sweep(None, 1) == ising.ISING_EINVAL
    assert lib.ising_measure(None, None) == ising.ISING_EINVAL
    assert lib.ising_sync(None) == ising.ISING_EINVAL


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2305_12161_gb300 import ising
    monkeypatch.setattr(ising, "_LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(ising, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        ising.lib()


def test_batch_create_rejects_bad_arguments(lib):
    from paper_2305_12161_gb300 import ising
    h = ctypes.c_void_p()

    def arr(t, v):
        a = (t * len(v))(*v)
        return ctypes.cast(a, ctypes.c_void_p), a

    for Ls, Rs in (([96], [1]), ([64, 7], [1, 1]), ([64], [0])):
        (pl, a), (pr, b), (ps, c) = arr(ctypes.c_int, Ls), arr(ctypes.c_int, Rs), arr(ctypes.c_uint64, [1] * len(Ls))
        assert lib.ising_batch_create(ctypes.byref(h), len(Ls), pl, pr, ps, None) == ising.ISING_EINVAL
    assert lib.ising_batch_create(ctypes.byref(h), 0, None, None, None, None) == ising.ISING_EINVAL
    assert lib.ising_batch_destroy(None) == ising.ISING_OK
    assert lib.ising_batch_sweep(None, 1) == ising.ISING_EINVAL
    o = ising.ising_opts()
    lib.ising_default_opts(ctypes.byref(o))
    assert o.pdl == 1  # programmatic dependent launch is the default
    assert lib.ising_batch_set_class_opts(None, 0, ctypes.byref(o)) == ising.ISING_EINVAL
    assert lib.ising_batch_get_class_opts(None, 0, ctypes.byref(o)) == ising.ISING_EINVAL
    assert lib.ising_batch_set_overlap(None, 1) == ising.ISING_EINVAL
    assert lib.ising_batch_overlap(None) == -1


def test_footprint_bytes_counts_every_buffer(lib):
    # packed store L^3/8 bytes per replica (1 bit per spin), records (3 + 3(L/2+1)) int64 and
    # 4 doubles per replica, a 16-byte status word; the tensor-core correlation scratch 2 L^3
    # bytes for L >= 512 by default (not for the bit-count method), the fused kernel's second
    # store, and L^3 bytes per replica for the plain form
    from paper_2305_12161_gb300 import ising

    def expect(L, R, fused=False, plain=False, tensor=None):
        tensor = (L >= 512) if tensor is None else tensor
        rec = 8 * R * (3 + 3 * (L // 2 + 1)) + 32 * R + 16
        lat = R * (L**3 // 8 if L >= 64 else 8 * L * L)  # L < 64: one padded 32-bit word per row
        return lat * (2 if fused else 1) + rec + (R * L**3 if plain else 0) + (2 * L**3 if tensor else 0)

    for L, R in ((32, 1), (64, 16), (256, 8), (512, 1), (1024, 3), (2048, 1)):
        assert ising.ising_footprint_bytes(L, R) == expect(L, R), (L, R)
        assert ising.ising_footprint_bytes(L, R, corr=ising.CORR_POPCOUNT) == expect(L, R, tensor=False)
        assert ising.ising_footprint_bytes(L, R, form=ising.FORM_PLAIN) == expect(L, R, plain=True)
    assert ising.ising_footprint_bytes(256, 1, corr=ising.CORR_TENSOR) == expect(256, 1, tensor=True)
    assert ising.ising_footprint_bytes(2048, 1, variant=ising.VARIANT_ZFUSE, tile_z=32, depth=3) == \
        expect(2048, 1, fused=True)
    # what ising_create_ex refuses
    assert ising.ising_footprint_bytes(96, 1) == -1
    assert ising.ising_footprint_bytes(64, 0) == -1
    assert ising.ising_footprint_bytes(128, 1, variant=ising.VARIANT_ZFUSE) == -1
    assert ising.ising_footprint_bytes(128, 1, corr=ising.CORR_TENSOR) == -1
