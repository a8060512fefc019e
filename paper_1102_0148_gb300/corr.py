"""Thin ctypes binding of the C ABI in ``include/corr.h`` (same names).

Argument marshalling only: every step of the correlator runs in the CUDA
kernels of ``libgbcorr.so``.  Buffers may be torch tensors (device or host),
numpy arrays (host) or raw integer addresses.  Importing this module loads
the library and raises ``ImportError`` if it has not been built -- there is
no fallback.
"""

import ctypes
import os

import numpy as np

from .build import LIB_PATH

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -m paper_1102_0148_gb300.build` "
        "(or __graft_entry__.build()); gbcorr has no CPU fallback")

_lib = ctypes.CDLL(LIB_PATH)

CORR_FP32, CORR_FP16, CORR_FP8E4M3, CORR_FP32_SIMT = 0, 1, 2, 3
CORR_OK, CORR_EINVAL, CORR_ENOMEM, CORR_ECUDA, CORR_ETIMEOUT, CORR_ESTATE, CORR_EUNSUPPORTED = (
    0, -1, -2, -3, -4, -5, -6)
CORR_MAX_N = 512
KERNEL_CLASSES = ("fengine", "xengine", "reduce", "dump", "fused")

DTYPES = {"fp32": CORR_FP32, "fp16": CORR_FP16, "fp8": CORR_FP8E4M3, "fp32_simt": CORR_FP32_SIMT}

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int

_SIGS = {
    "corr_create": (_int, [ctypes.POINTER(_vp), _int, _int, _int]),
    "corr_set_stream": (_int, [_vp, _vp]),
    "corr_set_chunk": (_int, [_vp, _i64]),
    "corr_set_tiles": (_int, [_vp, _int, _int, _int, _int]),
    "corr_set_fused": (_int, [_vp, _int]),
    "corr_get_fused": (_int, [_vp, ctypes.POINTER(_int)]),
    "corr_test_fault": (_int, [_vp, _int, ctypes.c_double]),
    "corr_state_bytes": (_int, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "corr_save_state": (_int, [_vp, _vp]),
    "corr_load_state": (_int, [_vp, _vp]),
    "corr_set_corrections": (_int, [_vp, _vp, _vp]),
    "corr_push": (_int, [_vp, _vp, _i64]),
    "corr_dump": (_int, [_vp, _vp, ctypes.POINTER(_i64), _int]),
    "corr_dump_async": (_int, [_vp, _vp, ctypes.POINTER(_i64), _int]),
    "corr_sync": (_int, [_vp]),
    "corr_destroy": (None, [_vp]),
    "corr_last_error": (ctypes.c_char_p, [_vp]),
    "corr_info": (_int, [_vp] + [ctypes.POINTER(_int)] * 5),
    "corr_profile_enable": (_int, [_vp, _int]),
    "corr_profile_read": (_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_double), _int]),
    "corr_debug_spectra": (_int, [_vp, _vp, _i64, _vp]),
    "corr_correlate_noalloc": (_int, [_vp, _i64, _int, _int, _vp, _vp]),
    "corr_set_scales": (_int, [_vp, _vp]),
    "corr_set_sample_delays": (_int, [_vp, _vp]),
    "corr_batch_create": (_int, [ctypes.POINTER(_vp), _int, ctypes.POINTER(_int), ctypes.POINTER(_int), _int]),
    "corr_batch_set_chunk": (_int, [_vp, _i64]),
    "corr_batch_set_tiles": (_int, [_vp, _int, _int, _int, _int]),
    "corr_batch_set_one_launch": (_int, [_vp, _int]),
    "corr_batch_push": (_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_i64)]),
    "corr_batch_dump": (_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_i64), _int]),
    "corr_batch_capture": (_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_i64), ctypes.POINTER(_vp), _int]),
    "corr_batch_replay": (_int, [_vp, ctypes.POINTER(_i64)]),
    "corr_batch_sync": (_int, [_vp]),
    "corr_batch_handle": (_int, [_vp, _int, ctypes.POINTER(_vp)]),
    "corr_batch_get_stream": (_int, [_vp, ctypes.POINTER(_vp)]),
    "corr_batch_destroy": (None, [_vp]),
    "corr_batch_last_error": (ctypes.c_char_p, [_vp]),
    "corr_grad": (_int, [_vp, _vp, _i64, _vp, _vp, _vp, _int, _vp, _vp]),
    "corr_get_scales": (_int, [_vp, _vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


class CorrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def _check(rc, h):
    if rc != CORR_OK:
        msg = _lib.corr_last_error(h)
        raise CorrError(rc, msg.decode() if msg else "")
    return rc


def _addr(buf):
    """Address of a tensor / ndarray / int buffer (None -> NULL)."""
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("buffer must be contiguous")
        return buf.data_ptr()
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("buffer must be C-contiguous")
        return buf.ctypes.data
    raise TypeError(f"unsupported buffer type {type(buf)!r}")


# ----------------------------------------------------------------------------
# Same-name wrappers of the C entry points
# ----------------------------------------------------------------------------

def corr_create(N, K, dtype=CORR_FP32):
    h = _vp()
    dtype = DTYPES.get(dtype, dtype) if isinstance(dtype, str) else dtype
    rc = _lib.corr_create(ctypes.byref(h), int(N), int(K), int(dtype))
    _check(rc, None)
    return h


def corr_set_stream(h, stream):
    s = stream if isinstance(stream, int) or stream is None else stream.cuda_stream
    return _check(_lib.corr_set_stream(h, s), h)


def corr_set_chunk(h, max_spectra):
    return _check(_lib.corr_set_chunk(h, int(max_spectra)), h)


def corr_set_tiles(h, window=0, stages=0, split=0, atoms=0):
    return _check(_lib.corr_set_tiles(h, int(window), int(stages), int(split), int(atoms)), h)


def corr_save_state(h):
    """The running integration's state as a bytes object."""
    n = ctypes.c_size_t(0)
    _check(_lib.corr_state_bytes(h, ctypes.byref(n)), h)
    buf = ctypes.create_string_buffer(n.value)
    _check(_lib.corr_save_state(h, buf), h)
    return buf.raw


def corr_load_state(h, state):
    buf = ctypes.create_string_buffer(state, len(state))
    return _check(_lib.corr_load_state(h, buf), h)


def corr_set_fused(h, on=True):
    return _check(_lib.corr_set_fused(h, 1 if on else 0), h)


def corr_get_fused(h):
    v = _int()
    _check(_lib.corr_get_fused(h, ctypes.byref(v)), h)
    return bool(v.value)


def corr_test_fault(h, kind, wait_limit_s):
    return _check(_lib.corr_test_fault(h, int(kind), float(wait_limit_s)), h)


def corr_set_corrections(h, gains=None, delays=None):
    """gains: complex64 [N] (tensor/ndarray) or float32 [2N]; delays: float32 [N]."""
    return _check(_lib.corr_set_corrections(h, _addr(gains), _addr(delays)), h)


def corr_set_scales(h, scales=None):
    """scales: float32 [N][C] (tensor/ndarray) or None for the automatic choice."""
    return _check(_lib.corr_set_scales(h, _addr(scales)), h)


def corr_get_scales(h, out=None):
    """Current [N][C] pre-cast scales (numpy float32 unless `out` is given)."""
    if out is None:
        info = corr_info(h)
        out = np.empty((info["N"], info["C"]), np.float32)
    _check(_lib.corr_get_scales(h, _addr(out)), h)
    return out


def corr_push(h, samples, n):
    return _check(_lib.corr_push(h, _addr(samples), int(n)), h)


def corr_dump(h, vis, fp64=False):
    n = _i64(0)
    _check(_lib.corr_dump(h, _addr(vis), ctypes.byref(n), 1 if fp64 else 0), h)
    return n.value


def corr_set_sample_delays(h, delays):
    """Integer sample delays per antenna (N int32 in [0, K]; None = off)."""
    if delays is not None and isinstance(delays, (list, tuple, np.ndarray)):
        delays = np.ascontiguousarray(np.asarray(delays, np.int32))
    return _check(_lib.corr_set_sample_delays(h, _addr(delays)), h)


def corr_dump_async(h, vis, fp64=False):
    """Queue the dump into device or page-locked host memory; `vis` is
    complete after the next corr_sync.  Returns the spectra summed."""
    n = _i64(0)
    _check(_lib.corr_dump_async(h, _addr(vis), ctypes.byref(n), 1 if fp64 else 0), h)
    return n.value


def corr_grad(h, samples, n, gains, delays, grad_vis, grad_fp64, grad_gains, grad_delays):
    return _check(_lib.corr_grad(h, _addr(samples), int(n), _addr(gains), _addr(delays),
                                 _addr(grad_vis), 1 if grad_fp64 else 0, _addr(grad_gains),
                                 _addr(grad_delays)), h)


def corr_sync(h):
    return _check(_lib.corr_sync(h), h)


def corr_destroy(h):
    _lib.corr_destroy(h)


def corr_last_error(h=None):
    m = _lib.corr_last_error(h)
    return m.decode() if m else ""


def corr_info(h):
    vals = [_int() for _ in range(5)]
    _check(_lib.corr_info(h, *[ctypes.byref(v) for v in vals]), h)
    return dict(zip(("N", "K", "C", "P", "dtype"), (v.value for v in vals)))


def corr_profile_enable(h, on=True):
    return _check(_lib.corr_profile_enable(h, 1 if on else 0), h)


def corr_profile_read(h):
    """{class: (launches, total_ms)} since the last read (clears the counters)."""
    n = len(KERNEL_CLASSES)
    launches = (_i64 * n)()
    ms = (ctypes.c_double * n)()
    _check(_lib.corr_profile_read(h, launches, ms, n), h)
    return {c: (launches[i], ms[i]) for i, c in enumerate(KERNEL_CLASSES)}


def corr_debug_spectra(h, samples, n, spectra):
    return _check(_lib.corr_debug_spectra(h, _addr(samples), int(n), _addr(spectra)), h)


def corr_correlate_noalloc(samples, n, N, K, vis, stream=None):
    """Allocation-free one-shot correlation into device ``vis`` ([P][C]
    complex64); queued on ``stream`` (torch stream, raw handle or None)."""
    s = stream if isinstance(stream, int) or stream is None else stream.cuda_stream
    return _check(_lib.corr_correlate_noalloc(_addr(samples), int(n), int(N), int(K), _addr(vis), s),
                  None)


def _bcheck(rc, b):
    if rc != CORR_OK:
        m = _lib.corr_batch_last_error(b)
        raise CorrError(rc, m.decode() if m else "")
    return rc


def _ptrs(bufs):
    return (_vp * len(bufs))(*[_addr(x) for x in bufs])


def corr_batch_create(N, K, dtype=CORR_FP32):
    b = _vp()
    n = len(N)
    dtype = DTYPES.get(dtype, dtype) if isinstance(dtype, str) else dtype
    rc = _lib.corr_batch_create(ctypes.byref(b), n, (_int * n)(*N), (_int * n)(*K), int(dtype))
    _check(rc, None)
    return b


def corr_batch_set_chunk(b, max_spectra):
    return _bcheck(_lib.corr_batch_set_chunk(b, int(max_spectra)), b)


def corr_batch_set_tiles(b, window=0, stages=0, split=0, atoms=0):
    return _bcheck(_lib.corr_batch_set_tiles(b, int(window), int(stages), int(split), int(atoms)),
                   b)


def corr_batch_set_one_launch(b, on=True):
    return _bcheck(_lib.corr_batch_set_one_launch(b, 1 if on else 0), b)


def corr_batch_push(b, samples, n):
    return _bcheck(_lib.corr_batch_push(b, _ptrs(samples), (_i64 * len(n))(*n)), b)


def corr_batch_dump(b, vis, fp64=False):
    ns = (_i64 * len(vis))()
    _bcheck(_lib.corr_batch_dump(b, _ptrs(vis), ns, 1 if fp64 else 0), b)
    return list(ns)


def corr_batch_capture(b, samples, n, vis, fp64=False):
    return _bcheck(_lib.corr_batch_capture(b, _ptrs(samples), (_i64 * len(n))(*n), _ptrs(vis),
                                           1 if fp64 else 0), b)


def corr_batch_replay(b, n_modes):
    ns = (_i64 * n_modes)()
    _bcheck(_lib.corr_batch_replay(b, ns), b)
    return list(ns)


def corr_batch_sync(b):
    return _bcheck(_lib.corr_batch_sync(b), b)


def corr_batch_handle(b, mode):
    h = _vp()
    _bcheck(_lib.corr_batch_handle(b, int(mode), ctypes.byref(h)), b)
    return h


def corr_batch_get_stream(b):
    s = _vp()
    _bcheck(_lib.corr_batch_get_stream(b, ctypes.byref(s)), b)
    return s.value or 0


def corr_batch_destroy(b):
    _lib.corr_batch_destroy(b)


def corr_batch_last_error(b):
    m = _lib.corr_batch_last_error(b)
    return m.decode() if m else ""


# ----------------------------------------------------------------------------
# Convenience object
# ----------------------------------------------------------------------------

class Correlator:
    """Owning wrapper: ``with Correlator(44, 512) as c: c.push(x); V, n = c.dump()``."""

    def __init__(self, N, K, dtype=CORR_FP32, chunk=None, stream=None, fused=None):
        if isinstance(dtype, str):
            dtype = DTYPES[dtype]
        self.h = corr_create(N, K, dtype)
        info = corr_info(self.h)
        self.N, self.K, self.C, self.P, self.dtype = (info[k] for k in ("N", "K", "C", "P", "dtype"))
        if chunk is not None:
            corr_set_chunk(self.h, chunk)
        if stream is not None:
            corr_set_stream(self.h, stream)
        if fused is not None:
            corr_set_fused(self.h, fused)

    def set_corrections(self, gains=None, delays=None):
        corr_set_corrections(self.h, gains, delays)

    def set_sample_delays(self, delays=None):
        corr_set_sample_delays(self.h, delays)

    def push(self, samples, n=None):
        """``samples``: uint8 buffer [n/K][N][K/2]; n defaults to its size."""
        if n is None:
            nbytes = samples.numel() if hasattr(samples, "numel") else np.asarray(samples).size
            n = nbytes * 2 // self.N
        corr_push(self.h, samples, n)

    def dump(self, out=None, fp64=False):
        """Returns (V, n_spec); V is ``out`` or a new numpy complex array [P][C]."""
        if out is None:
            out = np.empty((self.P, self.C), np.complex128 if fp64 else np.complex64)
        n = corr_dump(self.h, out, fp64)
        return out, n

    def close(self):
        if self.h is not None:
            corr_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CorrelatorBatch:
    """Several correlators of uneven N and K whose X-engine work shares one
    persistent tensor-core launch per pass (optionally replayed as a CUDA
    graph)."""

    def __init__(self, modes, dtype=CORR_FP32, chunk=None, window=0, stages=0, split=0,
                 one_launch=False):
        self.modes = [tuple(m) for m in modes]
        self.b = corr_batch_create([m[0] for m in self.modes], [m[1] for m in self.modes], dtype)
        self.handles = [corr_batch_handle(self.b, i) for i in range(len(self.modes))]
        self.info = [corr_info(h) for h in self.handles]
        if chunk is not None:
            corr_batch_set_chunk(self.b, chunk)
        if window or stages or split:
            corr_batch_set_tiles(self.b, window, stages, split)
        if one_launch:
            corr_batch_set_one_launch(self.b, True)

    @property
    def stream(self):
        return corr_batch_get_stream(self.b)

    def push(self, samples, n=None):
        if n is None:
            n = [x.numel() * 2 // m[0] for x, m in zip(samples, self.modes)]
        corr_batch_push(self.b, samples, n)

    def dump(self, vis=None, fp64=False):
        if vis is None:
            dt = np.complex128 if fp64 else np.complex64
            vis = [np.empty((i["P"], i["C"]), dt) for i in self.info]
        n = corr_batch_dump(self.b, vis, fp64)
        return vis, n

    def capture(self, samples, vis, n=None, fp64=False):
        if n is None:
            n = [x.numel() * 2 // m[0] for x, m in zip(samples, self.modes)]
        corr_batch_capture(self.b, samples, n, vis, fp64)

    def replay(self):
        return corr_batch_replay(self.b, len(self.modes))

    def sync(self):
        corr_batch_sync(self.b)

    def close(self):
        if self.b is not None:
            corr_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
