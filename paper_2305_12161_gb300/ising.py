"""Python binding of the C ABI in ``include/ising.h`` (argument marshalling only).

Every function below forwards to the entry point of the same name in ``libising.so``;
all computation runs in the library's CUDA kernels.  There is no CPU fallback: if the
library cannot be loaded, :func:`lib` raises.

Buffers are numpy arrays (host memory) or, for the ``*_device`` forms, any object with
a ``data_ptr()`` method (a CUDA ``torch.Tensor``) or an integer device address.
Streams are ``torch.cuda.Stream`` objects, raw ``cudaStream_t`` integers, or None.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libising.so")
_lock = threading.Lock()
_lib = None

ISING_OK, ISING_EINVAL, ISING_ENOMEM, ISING_ECUDA, ISING_ETIMEOUT, ISING_EBUSY, ISING_EPOISONED = 0, -1, -2, -3, -4, -5, -6
TIE_GLAUBER, TIE_ALWAYS, TIE_NEVER = 0, 1, 2
FORM_PACKED, FORM_PLAIN = 0, 1
MEAS_DEVICE, MEAS_CONNECTED, MEAS_NO_CORR = 1, 2, 4
PTR_DEVICE = 1
PTR_HOST_ASYNC = 2
CYCLE_01, CYCLE_MIXED = 0, 1
CORR_AUTO, CORR_POPCOUNT, CORR_TENSOR = 0, 1, 2
SCHEME_CHECKERBOARD, SCHEME_DOUBLE = 0, 1
FFT_SINGLE, FFT_DOUBLE = 0, 1
VARIANT_AUTO, VARIANT_WORD, VARIANT_ZMARCH, VARIANT_ZFAST, VARIANT_ZDEEP, VARIANT_ZFUSE = 0, 1, 2, 3, 4, 5


class IsingError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {ising_strerror(status)} ({status})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


class ising_opts(ctypes.Structure):
    _fields_ = [("tie", ctypes.c_int), ("form", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("device", ctypes.c_int), ("variant", ctypes.c_int), ("tile_y", ctypes.c_int),
                ("tile_z", ctypes.c_int), ("depth", ctypes.c_int), ("cycle", ctypes.c_int), ("corr", ctypes.c_int),
                ("scheme", ctypes.c_int), ("block_x", ctypes.c_int), ("block_y", ctypes.c_int),
                ("block_z", ctypes.c_int), ("pdl", ctypes.c_int)]


def lib_path() -> str:
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    """Load ``libising.so`` (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(f"CUDA library {_LIB_PATH} is missing: run __graft_entry__.build() first")
            L = ctypes.CDLL(_LIB_PATH)
            vp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
            sig = {
                "ising_default_opts": (None, [ctypes.POINTER(ising_opts)]),
                "ising_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_uint64]),
                "ising_create_ex": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                                   ctypes.POINTER(ising_opts)]),
                "ising_sweep": (ctypes.c_int, [vp, ctypes.c_int64]),
                "ising_reinit": (ctypes.c_int, [vp, ctypes.c_uint64]),
                "ising_init_menger": (ctypes.c_int, [vp, ctypes.c_int]),
                "ising_record_len": (ctypes.c_int64, [ctypes.c_int]),
                "ising_footprint_bytes": (ctypes.c_int64, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ising_opts)]),
                "ising_measure": (ctypes.c_int, [vp, vp]),
                "ising_measure_ex": (ctypes.c_int, [vp, vp, vp, ctypes.c_double, ctypes.c_uint]),
                "ising_radial_bins": (ctypes.c_int64, [ctypes.c_int]),
                "ising_release_scratch": (ctypes.c_int, [vp]),
                "ising_inject_corr_stall": (ctypes.c_int, [vp, ctypes.c_double]),
                "ising_measure_radial": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, vp, vp,
                                                        vp, vp, vp]),
                "ising_get_spins": (ctypes.c_int, [vp, ctypes.c_int, vp]),
                "ising_set_spins": (ctypes.c_int, [vp, ctypes.c_int, vp]),
                "ising_packed_words": (ctypes.c_int64, [ctypes.c_int]),
                "ising_get_packed": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_uint]),
                "ising_set_packed": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_uint]),
                "ising_get_time": (ctypes.c_int, [vp, i64p]),
                "ising_set_time": (ctypes.c_int, [vp, ctypes.c_int64]),
                "ising_sync": (ctypes.c_int, [vp]),
                "ising_destroy": (ctypes.c_int, [vp]),
                "ising_strerror": (ctypes.c_char_p, [ctypes.c_int]),
                "ising_last_error": (ctypes.c_char_p, [vp]),
                "ising_launch_count": (ctypes.c_int64, [vp]),
                "ising_variants": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
                "ising_tune_sweep": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                    ctypes.POINTER(ising_opts), ctypes.POINTER(ising_opts),
                                                    ctypes.POINTER(ctypes.c_double)]),
                "ising_batch_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, vp, vp, vp,
                                                      ctypes.POINTER(ising_opts)]),
                "ising_batch_sweep": (ctypes.c_int, [vp, ctypes.c_int64]),
                "ising_batch_record_words": (ctypes.c_int64, [vp]),
                "ising_batch_lattices": (ctypes.c_int64, [vp]),
                "ising_batch_measure_ex": (ctypes.c_int, [vp, vp, vp, ctypes.c_double, ctypes.c_uint]),
                "ising_batch_run": (ctypes.c_int, [vp, vp, ctypes.c_int, vp, vp, ctypes.c_double, ctypes.c_uint]),
                "ising_batch_reinit": (ctypes.c_int, [vp]),
                "ising_batch_get_packed": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_uint]),
                "ising_batch_sync": (ctypes.c_int, [vp]),
                "ising_batch_get_time": (ctypes.c_int, [vp, i64p]),
                "ising_batch_plan": (ctypes.c_int, [vp, vp, vp, vp, vp]),
                "ising_batch_tune": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
                "ising_batch_set_weights": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_double]),
                "ising_batch_set_streamed": (ctypes.c_int, [vp, ctypes.c_int]),
                "ising_batch_set_class_opts": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ising_opts)]),
                "ising_batch_get_class_opts": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ising_opts)]),
                "ising_batch_set_overlap": (ctypes.c_int, [vp, ctypes.c_int]),
                "ising_batch_overlap": (ctypes.c_int, [vp]),
                "ising_batch_streamed_classes": (ctypes.c_int, [vp]),
                "ising_batch_inject_missing_cta": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_double]),
                "ising_batch_last_error": (ctypes.c_char_p, [vp]),
                "ising_batch_launch_count": (ctypes.c_int64, [vp]),
                "ising_batch_destroy": (ctypes.c_int, [vp]),
                "ising_measure_derived_noalloc": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                                 ctypes.c_uint, vp, vp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def _dev_ptr(buf) -> int:
    if isinstance(buf, int):
        return buf
    return int(buf.data_ptr())


def _host(a: np.ndarray, dtype, n: int, name: str) -> np.ndarray:
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous or a.size < n:
        raise ValueError(f"{name} must be a C-contiguous numpy {np.dtype(dtype).name} array of >= {n} values")
    return a


def ising_strerror(status: int) -> str:
    try:
        return lib().ising_strerror(status).decode()
    except Exception:  # library not loadable: still report the code
        return f"status {status}"


def ising_record_len(L: int) -> int:
    return int(lib().ising_record_len(L))


def ising_radial_bins(L: int) -> int:
    """Number of radial bins round(sqrt(3) L/2) + 1 of the radial C and S (-1 for a bad L)."""
    return int(lib().ising_radial_bins(L))


def ising_packed_words(L: int) -> int:
    return int(lib().ising_packed_words(L))


def ising_footprint_bytes(L: int, replicas: int = 1, **opts) -> int:
    """Device bytes a context holds once it has measured (ising_footprint_bytes in the C
    ABI); keyword options as for Ising(...).  -1 for arguments the context would refuse."""
    o = ising_opts()
    lib().ising_default_opts(ctypes.byref(o))
    for k, v in opts.items():
        if k == "block":
            o.block_x, o.block_y, o.block_z = v
        elif k in dict(ising_opts._fields_) and k != "stream":
            setattr(o, k, v)
        else:
            raise TypeError(f"unknown option {k}")
    return int(lib().ising_footprint_bytes(L, replicas, ctypes.byref(o)))


def ising_variants() -> list[int]:
    buf = (ctypes.c_int * 16)()
    n = lib().ising_variants(buf, 16)
    return list(buf[:n])


class Ising:
    """One context: ``replicas`` lattices of size ``L`` (replica r seeded ``seed + r``)."""

    def __init__(self, L: int, replicas: int = 1, seed: int = 1, tie: int = TIE_GLAUBER, form: int = FORM_PACKED,
                 stream=None, device: int = -1, variant: int = 0, tile_y: int = 0, tile_z: int = 0, depth: int = 0,
                 cycle: int = CYCLE_01, corr: int = CORR_AUTO, scheme: int = SCHEME_CHECKERBOARD,
                 block=(0, 0, 0), pdl: int = 1):
        self._h = ctypes.c_void_p()
        o = ising_opts()
        lib().ising_default_opts(ctypes.byref(o))
        o.tie, o.form, o.device, o.variant, o.tile_y, o.tile_z, o.depth = tie, form, device, variant, tile_y, tile_z, depth
        o.pdl = pdl
        o.cycle = cycle
        o.corr = corr
        o.scheme = scheme
        o.block_x, o.block_y, o.block_z = block
        sh = _stream_handle(stream)
        o.stream = sh if sh else None
        self._stream_obj = stream  # keep the caller's stream alive
        st = lib().ising_create_ex(ctypes.byref(self._h), L, replicas, seed % 2**64, ctypes.byref(o))
        if st != ISING_OK:
            raise IsingError(st, "ising_create_ex")
        self.L, self.replicas, self.seed = L, replicas, seed
        self.record_len = ising_record_len(L)
        self.N = L**3

    # -- helpers -----------------------------------------------------------------
    def _check(self, st: int, where: str) -> None:
        if st != ISING_OK:
            detail = lib().ising_last_error(self._h) if self._h else b""
            raise IsingError(st, where, (detail or b"").decode())

    @property
    def handle(self) -> int:
        return int(self._h.value or 0)

    # -- entry points ------------------------------------------------------------
    def reinit(self, seed: int) -> None:
        """Redraw the T = infinity start (replica r: seed + r) and reset t to 0."""
        self._check(lib().ising_reinit(self._h, seed % 2**64), "ising_reinit")
        self.seed = seed

    def init_menger(self, k: int) -> None:
        """Menger-sponge start of iteration k for every replica; t = 0."""
        self._check(lib().ising_init_menger(self._h, k), "ising_init_menger")

    def sweep(self, n_mcs: int) -> None:
        self._check(lib().ising_sweep(self._h, n_mcs), "ising_sweep")

    def measure(self, out: np.ndarray | None = None) -> np.ndarray:
        """Records [replicas, record_len] int64 in host memory (synchronises)."""
        if out is None:
            out = np.empty((self.replicas, self.record_len), dtype=np.int64)
        _host(out, np.int64, self.replicas * self.record_len, "out")
        self._check(lib().ising_measure(self._h, out.ctypes.data), "ising_measure")
        return out

    def measure_ex(self, c: float = 0.5, connected: bool = False, corr: bool = True):
        """(records [R, record_len] int64, derived [R, 4] float64) in host memory."""
        rec = np.empty((self.replicas, self.record_len), dtype=np.int64)
        der = np.empty((self.replicas, 4), dtype=np.float64)
        flags = (MEAS_CONNECTED if connected else 0) | (0 if corr else MEAS_NO_CORR)
        self._check(lib().ising_measure_ex(self._h, rec.ctypes.data, der.ctypes.data, c, flags), "ising_measure_ex")
        return rec, der

    def measure_radial(self, replica: int = 0, precision: int = FFT_SINGLE, c: float = 0.5) -> dict:
        """Radially averaged 3-d correlation C(b), structure factor S(b), vectors per bin,
        the length at which C crosses c, and the number of inexact lags (0: C is exact)."""
        nb = ising_radial_bins(self.L)
        C = np.empty(nb, dtype=np.float64)
        S = np.empty(nb, dtype=np.float64)
        n = np.empty(nb, dtype=np.int64)
        ell = ctypes.c_double()
        bad = ctypes.c_int64()
        self._check(lib().ising_measure_radial(self._h, replica, precision, c, C.ctypes.data, S.ctypes.data,
                                               n.ctypes.data, ctypes.addressof(ell), ctypes.addressof(bad)),
                    "ising_measure_radial")
        return {"C": C, "S": S, "count": n, "ell": ell.value, "inexact": bad.value}

    def inject_corr_stall(self, timeout_s: float = 0.5) -> None:
        """Test hook: the next tensor-core measurement's bounded wait runs out (ISING_ETIMEOUT)."""
        self._check(lib().ising_inject_corr_stall(self._h, timeout_s), "ising_inject_corr_stall")

    def release_scratch(self) -> None:
        """Free the measurement scratch kept in the context (radial FFT buffer, etc.)."""
        self._check(lib().ising_release_scratch(self._h), "ising_release_scratch")

    def measure_device(self, rec, derived=None, c: float = 0.5, connected: bool = False, corr: bool = True) -> None:
        """Enqueue a measurement into device buffers (no synchronisation)."""
        flags = MEAS_DEVICE | (MEAS_CONNECTED if connected else 0) | (0 if corr else MEAS_NO_CORR)
        dp = _dev_ptr(derived) if derived is not None else None
        self._check(lib().ising_measure_ex(self._h, _dev_ptr(rec), dp, c, flags), "ising_measure_ex")

    def get_spins(self, replica: int = 0) -> np.ndarray:
        out = np.empty((self.L, self.L, self.L), dtype=np.int8)
        self._check(lib().ising_get_spins(self._h, replica, out.ctypes.data), "ising_get_spins")
        return out

    def set_spins(self, spins: np.ndarray, replica: int = 0) -> None:
        s = np.ascontiguousarray(spins, dtype=np.int8)
        if s.size != self.N:
            raise ValueError("spins must hold L^3 values")
        self._check(lib().ising_set_spins(self._h, replica, s.ctypes.data), "ising_set_spins")

    def get_packed(self, replica: int = 0, out=None, device: bool = False):
        n = ising_packed_words(self.L)
        if device:
            self._check(lib().ising_get_packed(self._h, replica, _dev_ptr(out), PTR_DEVICE), "ising_get_packed")
            return out
        if out is None:
            out = np.empty(n, dtype=np.uint32)
        _host(out, np.uint32, n, "out")
        self._check(lib().ising_get_packed(self._h, replica, out.ctypes.data, 0), "ising_get_packed")
        return out

    def set_packed(self, words, replica: int = 0, device: bool = False, asynchronous: bool = False) -> None:
        """Load one replica's packed words.  asynchronous=True: `words` is a page-locked host
        torch tensor (pin_memory) that must stay alive and unchanged until sync(); the call
        returns at once and the transfer overlaps the work already queued."""
        if device:
            self._check(lib().ising_set_packed(self._h, replica, _dev_ptr(words), PTR_DEVICE), "ising_set_packed")
            return
        if asynchronous:
            if not (hasattr(words, "is_pinned") and words.is_pinned()):
                raise ValueError("asynchronous set_packed needs a page-locked (pinned) torch tensor")
            if words.numel() * words.element_size() != 4 * ising_packed_words(self.L) or not words.is_contiguous():
                raise ValueError("words: one replica's packed state, contiguous")
            self._check(lib().ising_set_packed(self._h, replica, ctypes.c_void_p(words.data_ptr()), PTR_HOST_ASYNC),
                        "ising_set_packed")
            return
        w = _host(words, np.uint32, ising_packed_words(self.L), "words")
        self._check(lib().ising_set_packed(self._h, replica, w.ctypes.data, 0), "ising_set_packed")

    @property
    def t(self) -> int:
        v = ctypes.c_int64(0)
        self._check(lib().ising_get_time(self._h, ctypes.byref(v)), "ising_get_time")
        return int(v.value)

    @t.setter
    def t(self, value: int) -> None:
        self._check(lib().ising_set_time(self._h, value), "ising_set_time")

    def sync(self) -> None:
        self._check(lib().ising_sync(self._h), "ising_sync")

    def launch_count(self) -> int:
        return int(lib().ising_launch_count(self._h))

    def destroy(self) -> None:
        if self._h and self._h.value:
            lib().ising_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def ising_tune_sweep(L: int, replicas: int = 1, probe_mcs: int = 8, tie: int = TIE_GLAUBER) -> dict:
    """Fastest (variant, tile_y, tile_z) for this size; pass them to Ising(...)."""
    base = ising_opts()
    lib().ising_default_opts(ctypes.byref(base))
    base.tie = tie
    best = ising_opts()
    ms = ctypes.c_double(0)
    st = lib().ising_tune_sweep(L, replicas, probe_mcs, ctypes.byref(base), ctypes.byref(best), ctypes.byref(ms))
    if st != ISING_OK:
        raise IsingError(st, "ising_tune_sweep")
    return {"variant": best.variant, "tile_y": best.tile_y, "tile_z": best.tile_z, "depth": best.depth,
            "ms_per_mcs": ms.value}


class Batch:
    """Lattice classes [(L, replicas, seed), ...] advanced together by one persistent
    launch per segment (see ``ising_batch_*`` in include/ising.h)."""

    def __init__(self, classes, tie: int = TIE_GLAUBER, stream=None, device: int = -1):
        self._h = ctypes.c_void_p()
        self.classes = [(int(L), int(R), int(s)) for L, R, s in classes]
        n = len(self.classes)
        Ls = (ctypes.c_int * n)(*[c[0] for c in self.classes])
        Rs = (ctypes.c_int * n)(*[c[1] for c in self.classes])
        Ss = (ctypes.c_uint64 * n)(*[c[2] % 2**64 for c in self.classes])
        o = ising_opts()
        lib().ising_default_opts(ctypes.byref(o))
        o.tie, o.device = tie, device
        sh = _stream_handle(stream)
        o.stream = sh if sh else None
        self._stream_obj = stream
        st = lib().ising_batch_create(ctypes.byref(self._h), n, ctypes.cast(Ls, ctypes.c_void_p),
                                      ctypes.cast(Rs, ctypes.c_void_p), ctypes.cast(Ss, ctypes.c_void_p),
                                      ctypes.byref(o))
        if st != ISING_OK:
            raise IsingError(st, "ising_batch_create")
        self.record_words = int(lib().ising_batch_record_words(self._h))
        self.lattices = int(lib().ising_batch_lattices(self._h))
        self.offsets = []  # (record offset, derived row offset) per class
        ro = do = 0
        for L, R, _ in self.classes:
            self.offsets.append((ro, do))
            ro += R * ising_record_len(L)
            do += R

    def _check(self, st: int, where: str) -> None:
        if st != ISING_OK:
            detail = lib().ising_batch_last_error(self._h) if self._h else b""
            raise IsingError(st, where, (detail or b"").decode())

    def sweep(self, n_mcs: int) -> None:
        self._check(lib().ising_batch_sweep(self._h, n_mcs), "ising_batch_sweep")

    def measure_ex(self, c: float = 0.5, connected: bool = False, corr: bool = True):
        rec = np.empty(self.record_words, dtype=np.int64)
        der = np.empty((self.lattices, 4), dtype=np.float64)
        flags = (MEAS_CONNECTED if connected else 0) | (0 if corr else MEAS_NO_CORR)
        self._check(lib().ising_batch_measure_ex(self._h, rec.ctypes.data, der.ctypes.data, c, flags),
                    "ising_batch_measure_ex")
        return rec, der

    def run(self, times, c: float = 0.5, connected: bool = False, corr: bool = True, rec=None, derived=None,
            device: bool = False):
        """Schedule run (one CUDA graph).  Host mode returns (rec [K, words], der [K, lat, 4])."""
        t = np.ascontiguousarray(times, dtype=np.int64)
        K = t.size
        flags = (MEAS_CONNECTED if connected else 0) | (0 if corr else MEAS_NO_CORR)
        if device:
            flags |= MEAS_DEVICE
            dp = _dev_ptr(derived) if derived is not None else None
            self._check(lib().ising_batch_run(self._h, t.ctypes.data, K, _dev_ptr(rec), dp, c, flags),
                        "ising_batch_run")
            return rec, derived
        rec = np.empty((K, self.record_words), dtype=np.int64)
        der = np.empty((K, self.lattices, 4), dtype=np.float64)
        self._check(lib().ising_batch_run(self._h, t.ctypes.data, K, rec.ctypes.data, der.ctypes.data, c, flags),
                    "ising_batch_run")
        return rec, der

    def record_of(self, rec_block: np.ndarray, cls: int, replica: int) -> np.ndarray:
        """One lattice's record out of a batch record block."""
        L, R, _ = self.classes[cls]
        off = self.offsets[cls][0] + replica * ising_record_len(L)
        return rec_block[off:off + ising_record_len(L)]

    def reinit(self) -> None:
        self._check(lib().ising_batch_reinit(self._h), "ising_batch_reinit")

    def get_packed(self, cls: int, replica: int) -> np.ndarray:
        out = np.empty(ising_packed_words(self.classes[cls][0]), dtype=np.uint32)
        self._check(lib().ising_batch_get_packed(self._h, cls, replica, out.ctypes.data, 0), "ising_batch_get_packed")
        return out

    def sync(self) -> None:
        self._check(lib().ising_batch_sync(self._h), "ising_batch_sync")

    @property
    def t(self) -> int:
        v = ctypes.c_int64(0)
        self._check(lib().ising_batch_get_time(self._h, ctypes.byref(v)), "ising_batch_get_time")
        return int(v.value)

    def plan(self) -> dict:
        v = [ctypes.c_int(0) for _ in range(4)]
        self._check(lib().ising_batch_plan(self._h, *[ctypes.byref(x) for x in v]), "ising_batch_plan")
        return dict(zip(("ctas", "local_ctas", "groups", "capacity"), (x.value for x in v)))

    def tune(self, probe_mcs: int = 4) -> float:
        w = ctypes.c_double(0)
        self._check(lib().ising_batch_tune(self._h, probe_mcs, ctypes.byref(w)), "ising_batch_tune")
        return float(w.value)

    def set_weights(self, w_local: float, w_group: float = 1.0) -> None:
        self._check(lib().ising_batch_set_weights(self._h, w_local, w_group), "ising_batch_set_weights")

    def set_streamed(self, min_L: int) -> None:
        """Classes with L >= min_L (L % 256 == 0) use a single-lattice kernel; <= 0: none."""
        self._check(lib().ising_batch_set_streamed(self._h, min_L), "ising_batch_set_streamed")

    def set_class_config(self, cls: int, variant: int = 0, tile_y: int = 0, tile_z: int = 0, depth: int = 0) -> None:
        """Sweep kernel of streamed class ``cls`` (ising_batch_set_class_opts)."""
        o = ising_opts()
        lib().ising_default_opts(ctypes.byref(o))
        o.variant, o.tile_y, o.tile_z, o.depth = variant, tile_y, tile_z, depth
        self._check(lib().ising_batch_set_class_opts(self._h, cls, ctypes.byref(o)), "ising_batch_set_class_opts")

    def set_overlap(self, on: bool) -> None:
        """Streamed classes beside (True) or after (False) the persistent launch."""
        self._check(lib().ising_batch_set_overlap(self._h, int(bool(on))), "ising_batch_set_overlap")

    @property
    def overlap(self) -> bool:
        return bool(lib().ising_batch_overlap(self._h))

    def class_config(self, cls: int) -> dict:
        """Sweep kernel of class ``cls``: variant -1 for the persistent kernel."""
        o = ising_opts()
        self._check(lib().ising_batch_get_class_opts(self._h, cls, ctypes.byref(o)), "ising_batch_get_class_opts")
        return dict(variant=o.variant, tile_y=o.tile_y, tile_z=o.tile_z, depth=o.depth)

    def streamed_classes(self) -> int:
        return int(lib().ising_batch_streamed_classes(self._h))

    def inject_missing_cta(self, cta: int, timeout_s: float = 1.0) -> None:
        self._check(lib().ising_batch_inject_missing_cta(self._h, cta, timeout_s), "ising_batch_inject_missing_cta")

    def launch_count(self) -> int:
        return int(lib().ising_batch_launch_count(self._h))

    def destroy(self) -> None:
        if self._h and self._h.value:
            lib().ising_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


NOALLOC_MAX_RECORD_WORDS = 131072


def ising_measure_derived_noalloc(lattice, L: int, replicas: int, derived, c: float = 0.5, connected: bool = False,
                                  corr: bool = True, stream=None, device_flag: bool = False) -> int:
    """Derived observables of caller-owned packed lattices into a caller-owned device
    buffer, allocating nothing (for callers that may not allocate device memory).
    Returns the C status code; the work is enqueued on ``stream`` without a sync.
    ``device_flag`` also passes ISING_MEAS_DEVICE, which the entry point accepts and ignores."""
    flags = (MEAS_CONNECTED if connected else 0) | (0 if corr else MEAS_NO_CORR) | (MEAS_DEVICE if device_flag else 0)
    return int(lib().ising_measure_derived_noalloc(_dev_ptr(lattice), L, replicas, c, flags, _dev_ptr(derived),
                                                   _stream_handle(stream)))


def ising_create(L: int, replicas: int, seed: int, **opts) -> Ising:
    return Ising(L, replicas, seed, **opts)


def ising_sweep(ctx: Ising, n_mcs: int) -> None:
    ctx.sweep(n_mcs)


def ising_measure(ctx: Ising, out: np.ndarray | None = None) -> np.ndarray:
    return ctx.measure(out)


def ising_destroy(ctx: Ising) -> None:
    ctx.destroy()
