"""ctypes binding of libnanodisk.so (include/nanodisk.h).

Argument marshalling only: every step of the computation runs inside the CUDA
library.  The functions keep the C names; pointers may be torch CUDA tensors,
numpy arrays (host buffers) or raw integers.  If the library cannot be built
or loaded the import fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

ND_OK, ND_ERR_ARG, ND_ERR_CUDA, ND_ERR_NOT_CONVERGED, ND_ERR_NO_VORTEX, ND_ERR_TIMEOUT, ND_ERR_NAN = range(7)
ND_FP32, ND_FP64 = 0, 1
ND_GRID_3X = 0x100
ND_METHOD_RK4, ND_METHOD_HEUN = 0, 1

_lock = threading.Lock()
_lib = None


class NDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libnanodisk error {code}: {msg}")
        self.code = code


class nd_disk_desc(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double), ("L", ctypes.c_double), ("a", ctypes.c_double),
                ("Ms", ctypes.c_double), ("A", ctypes.c_double), ("gamma", ctypes.c_double),
                ("alpha", ctypes.c_double), ("hext", ctypes.c_double * 3),
                ("polarity", ctypes.c_int), ("chirality", ctypes.c_int)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_LL = ctypes.c_longlong
_ULL = ctypes.c_ulonglong

SIGNATURES = {
    "nd_create_disk": (_I, [_P, _I, _P, _I, _P]),
    "nd_destroy": (None, [_P]),
    "nd_last_error": (ctypes.c_char_p, []),
    "nd_get_info": (_I, [_P, _P, _P]),
    "nd_replica_layout": (_I, [_P, _I, _P, _P, _P, _P, _P]),
    "nd_disk_mask": (_I, [_P, _I, _P]),
    "nd_units": (_I, [_P, _I, _P]),
    "nd_set_green_tensor": (_I, [_P, _I, _P]),
    "nd_set_damping": (_I, [_P, _P]),
    "nd_set_mask": (_I, [_P, _I, _P]),
    "nd_set_field_schedule": (_I, [_P, _I, _LL, _P]),
    "nd_effective_field": (_I, [_P, _P, _P, _P]),
    "nd_energy": (_I, [_P, _P, _P, _P, _P]),
    "nd_step_rk4": (_I, [_P, _P, _LL, _D, _P]),
    "nd_step_heun": (_I, [_P, _P, _LL, _D, _P, _P, _ULL, _P]),
    "nd_init_vortex": (_I, [_P, _P, _P, _P]),
    "nd_vortex_core": (_I, [_P, _P, _P, _P, _P]),
    "nd_mean_m": (_I, [_P, _P, _P, _P]),
    "nd_relax_constrained": (_I, [_P, _P, _P, _D, _I, _P, _P, _P, _P]),
    "nd_relax_sweep_grad": (_I, [_P, _P, _P, _P, _P, _D, _P, _P, _P]),
    "nd_stats_reset": (_I, [_P, _D, _I, _D, _I]),
    "nd_check_status": (_I, [_P, _P]),
    "nd_selftest_handover_timeout": (_I, [_P, _P]),
    "nd_graph_create": (_I, [_P, _P, _I, _LL, _D, _P, _P, _ULL, _I, _P]),
    "nd_autotune": (_I, [_P, _I, _D, _LL, _P]),
    "nd_autotune_group": (_I, [_P, _P, _I, _D, _LL, _P]),
    "nd_set_plan": (_I, [_P, _I, _I, _I]),
    "nd_plan_info": (_I, [_P, _I, _P, _P, _P, _P, _P, _P]),
    "nd_graph_launch": (_I, [_P, _P]),
    "nd_graph_join": (_I, [_P, _I, _P]),
    "nd_graph_nodes": (_I, [_P, _P]),
    "nd_graph_destroy": (None, [_P]),
    "nd_stats_sample": (_I, [_P, _P, _D, _P]),
    "nd_series_reset": (_I, [_P, _I]),
    "nd_series_sample": (_I, [_P, _P, _P]),
    "nd_series_read": (_I, [_P, _P, _P]),
    "nd_power_spectrum": (_I, [_P, _I, _I, _D, _P, _P, _P, _P]),
    "nd_stats_read": (_I, [_P, _P, _P, _P, _P]),
    "nd_stats_save_bytes": (ctypes.c_size_t, [_P]),
    "nd_stats_save": (_I, [_P, _P, ctypes.c_size_t, _P]),
    "nd_stats_load": (_I, [_P, _P, ctypes.c_size_t, _P]),
    "nd_step_heun_noalloc": (_I, [_P, _I, _P, _LL, _D, _P, _P, _ULL, _P]),
}


def library_path() -> str:
    return _build.LIB


def lib(build: bool = True):
    """Load (building first if stale) libnanodisk.so."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build else _build.LIB
            if not os.path.exists(path):
                raise ImportError(f"libnanodisk.so not found at {path}; run paper_1207_2192_gb300.build.build()")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(x):
    """Raw pointer of a torch tensor, numpy array, ctypes object or int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    return ctypes.cast(x, ctypes.c_void_p).value


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(rc):
    if rc != ND_OK:
        raise NDError(rc, lib().nd_last_error().decode())
    return rc


# ------------------------------------------------------------- C names

def nd_create_disk(disks, replicas_per_disk=None, precision=ND_FP32):
    arr = (nd_disk_desc * len(disks))(*disks)
    rep = None if replicas_per_disk is None else (ctypes.c_int * len(disks))(*replicas_per_disk)
    h = ctypes.c_void_p()
    _check(lib().nd_create_disk(ctypes.cast(arr, _P), len(disks), ctypes.cast(rep, _P) if rep else None, precision,
                                ctypes.byref(h)))
    return h.value


def nd_destroy(h):
    lib().nd_destroy(h)


def nd_last_error():
    return lib().nd_last_error().decode()


def nd_get_info(h):
    n, e = ctypes.c_int(), ctypes.c_longlong()
    _check(lib().nd_get_info(h, ctypes.byref(n), ctypes.byref(e)))
    return n.value, e.value


def nd_replica_layout(h, r):
    D, Dp, P, off, C = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong(), ctypes.c_int()
    _check(lib().nd_replica_layout(h, r, ctypes.byref(D), ctypes.byref(Dp), ctypes.byref(P), ctypes.byref(off),
                                   ctypes.byref(C)))
    return dict(D=D.value, Dpad=Dp.value, P=P.value, offset=off.value, cells=C.value)


def nd_disk_mask(h, d, D):
    out = np.zeros((D, D), dtype=np.uint8)
    _check(lib().nd_disk_mask(h, d, _ptr(out)))
    return out


def nd_units(h, d):
    out = np.zeros(8)
    _check(lib().nd_units(h, d, _ptr(out)))
    return out


def nd_set_green_tensor(h, d, Gq=None):
    g = None if Gq is None else np.ascontiguousarray(Gq, dtype=np.float64)
    _check(lib().nd_set_green_tensor(h, d, _ptr(g)))


def nd_set_damping(h, alpha):
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    _check(lib().nd_set_damping(h, _ptr(a)))


def nd_set_mask(h, d, mask):
    mk = np.ascontiguousarray(mask, dtype=np.uint8)
    _check(lib().nd_set_mask(h, d, _ptr(mk)))


def nd_set_field_schedule(h, d, H=None):
    """Per-step external field H[s] (A/m, shape (n, 3)); None removes it."""
    if H is None:
        _check(lib().nd_set_field_schedule(h, d, 0, None))
        return
    Ha = np.ascontiguousarray(H, dtype=np.float64).reshape(-1, 3)
    _check(lib().nd_set_field_schedule(h, d, len(Ha), _ptr(Ha)))


def nd_effective_field(h, m, b, stream=None):
    _check(lib().nd_effective_field(h, _ptr(m), _ptr(b), _stream(stream)))


def nd_energy(h, m, nrep, stream=None, with_dL=False):
    """Energies in units of J (and dE/dL in J/m when with_dL)."""
    E = np.zeros(nrep)
    dL = np.zeros(nrep) if with_dL else None
    _check(lib().nd_energy(h, _ptr(m), _ptr(E), _ptr(dL), _stream(stream)))
    return (E, dL) if with_dL else E


def nd_step_rk4(h, m, n_steps, dt_seconds, stream=None):
    _check(lib().nd_step_rk4(h, _ptr(m), n_steps, dt_seconds, _stream(stream)))


def nd_step_heun(h, m, n_steps, dt_seconds, T_kelvin, seed, step0=0, stream=None):
    T = np.ascontiguousarray(T_kelvin, dtype=np.float64)
    s = np.ascontiguousarray(seed, dtype=np.uint64)
    _check(lib().nd_step_heun(h, _ptr(m), n_steps, dt_seconds, _ptr(T), _ptr(s), step0, _stream(stream)))


def nd_relax_constrained(h, m, X, nrep, tol=1e-6, max_iter=20000, stream=None, check=True):
    """Constrained relaxation; returns (status, U[B], lambda[B,2], iters[B])."""
    Xa = np.ascontiguousarray(X, dtype=np.float64).reshape(nrep, 2)
    U = np.zeros(nrep)
    lam = np.zeros((nrep, 2))
    it = np.zeros(nrep, dtype=np.int32)
    rc = lib().nd_relax_constrained(h, _ptr(m), _ptr(Xa), tol, max_iter, _ptr(U), _ptr(lam), _ptr(it),
                                    _stream(stream))
    if check and rc not in (ND_OK, ND_ERR_NOT_CONVERGED):
        _check(rc)
    return rc, U, lam, it


def nd_init_vortex(h, m, X0, stream=None):
    X = np.ascontiguousarray(X0, dtype=np.float64)
    _check(lib().nd_init_vortex(h, _ptr(m), _ptr(X), _stream(stream)))


def nd_relax_sweep_grad(h, m, grad, X, lam, nrep, tol=0.0, stream=None):
    """One gradient-driven relaxation sweep; lam ([nrep, 2] float64) is updated
    in place.  Returns (resid [nrep], moved [nrep] bool)."""
    Xa = np.ascontiguousarray(X, dtype=np.float64).reshape(nrep, 2)
    assert lam.dtype == np.float64 and lam.flags["C_CONTIGUOUS"] and lam.shape == (nrep, 2)
    res = np.zeros(nrep)
    moved = np.zeros(nrep, dtype=np.int32)
    _check(lib().nd_relax_sweep_grad(h, _ptr(m), _ptr(grad), _ptr(Xa), _ptr(lam), tol, _ptr(res), _ptr(moved),
                                     _stream(stream)))
    return res, moved.astype(bool)


def nd_vortex_core(h, m, nrep, stream=None, check=False):
    Xc = np.zeros((nrep, 2))
    st = np.zeros(nrep, dtype=np.int32)
    rc = lib().nd_vortex_core(h, _ptr(m), _ptr(Xc), _ptr(st), _stream(stream))
    if rc not in (ND_OK, ND_ERR_NO_VORTEX) or (check and rc != ND_OK):
        _check(rc)
    return Xc, st


def nd_mean_m(h, m, nrep, stream=None):
    out = np.zeros((nrep, 3))
    _check(lib().nd_mean_m(h, _ptr(m), _ptr(out), _stream(stream)))
    return out


def nd_step_heun_noalloc(disk, n_replicas, m, n_steps, dt_seconds, T_kelvin, seed, step0=0, stream=None,
                         check=True):
    """Allocation-free Heun steps (no handle); returns the status code."""
    d = disk if isinstance(disk, nd_disk_desc) else disk.desc()
    T = np.ascontiguousarray(T_kelvin, dtype=np.float64)
    s = np.ascontiguousarray(seed, dtype=np.uint64)
    rc = lib().nd_step_heun_noalloc(ctypes.byref(d), n_replicas, _ptr(m), n_steps, dt_seconds, _ptr(T), _ptr(s),
                                    step0, _stream(stream))
    if check:
        _check(rc)
    return rc


def nd_stats_reset(h, r_max, r_bins, v_max, v_bins):
    _check(lib().nd_stats_reset(h, r_max, r_bins, v_max, v_bins))


def nd_stats_sample(h, m, dt_sample_seconds, stream=None):
    _check(lib().nd_stats_sample(h, _ptr(m), dt_sample_seconds, _stream(stream)))


def nd_stats_read(h, nrep, r_bins, v_bins, stream=None):
    mom = np.zeros((nrep, 7))
    hr = np.zeros((nrep, r_bins), dtype=np.uint64)
    hv = np.zeros((nrep, v_bins), dtype=np.uint64)
    _check(lib().nd_stats_read(h, _ptr(mom), _ptr(hr), _ptr(hv), _stream(stream)))
    return mom, hr, hv


def nd_stats_save(h, stream=None):
    """The statistics accumulators as a bytes record (nd_stats_load restores it)."""
    n = lib().nd_stats_save_bytes(h)
    if n == 0:
        raise NDError(ND_ERR_ARG, "no statistics to save")
    buf = ctypes.create_string_buffer(n)
    _check(lib().nd_stats_save(h, buf, n, _stream(stream)))
    return buf.raw


def nd_stats_load(h, record, stream=None):
    buf = ctypes.create_string_buffer(bytes(record), len(record))
    _check(lib().nd_stats_load(h, buf, len(record), _stream(stream)))


def nd_series_reset(h, capacity):
    _check(lib().nd_series_reset(h, int(capacity)))


def nd_series_sample(h, m, stream=None):
    _check(lib().nd_series_sample(h, _ptr(m), _stream(stream)))


def nd_series_read(h, nrep, capacity):
    """Returns (samples taken, array [nrep][kept][3] of the kept ones)."""
    n = ctypes.c_longlong()
    _check(lib().nd_series_read(h, None, ctypes.byref(n)))
    kept = min(n.value, capacity)
    out = np.zeros((nrep, kept, 3))
    if kept:
        _check(lib().nd_series_read(h, _ptr(out), ctypes.byref(n)))
    return n.value, out


def nd_power_spectrum(h, nrep, component, window, dt_sample_seconds, stream=None):
    """Averaged one-sided periodogram of the recorded <m> series: returns
    (psd [nrep][window/2+1], freq [window/2+1] in Hz, n_windows)."""
    psd = np.zeros((nrep, window // 2 + 1))
    freq = np.zeros(window // 2 + 1)
    nw = ctypes.c_int()
    _check(lib().nd_power_spectrum(h, int(component), int(window), float(dt_sample_seconds), _ptr(psd), _ptr(freq),
                                   ctypes.byref(nw), _stream(stream)))
    return psd, freq, nw.value


def nd_check_status(h, stream=None):
    """Synchronise and return the device status code (ND_OK, ND_ERR_TIMEOUT, ND_ERR_NAN)."""
    return lib().nd_check_status(h, _stream(stream))


def nd_selftest_handover_timeout(h, stream=None):
    """Run the bounded-wait failure path once (see include/nanodisk.h)."""
    _check(lib().nd_selftest_handover_timeout(h, _stream(stream)))


ND_GRAPH_STATS = 1
ND_GRAPH_SERIES = 2


def nd_graph_create(h, m, method, n_steps, dt_seconds, T_kelvin=None, seed=None, step0=0, stats_sample=False):
    """stats_sample: False/True, or a combination of ND_GRAPH_STATS and ND_GRAPH_SERIES."""
    T = None if T_kelvin is None else np.ascontiguousarray(T_kelvin, dtype=np.float64)
    s = None if seed is None else np.ascontiguousarray(seed, dtype=np.uint64)
    g = ctypes.c_void_p()
    _check(lib().nd_graph_create(h, _ptr(m), method, n_steps, dt_seconds, _ptr(T), _ptr(s), step0, int(stats_sample),
                                 ctypes.byref(g)))
    return g.value


def nd_graph_join(parts):
    """One graph replaying the given graphs side by side (the parts must outlive it)."""
    arr = (ctypes.c_void_p * len(parts))(*parts)
    g = ctypes.c_void_p()
    _check(lib().nd_graph_join(ctypes.cast(arr, _P), len(parts), ctypes.byref(g)))
    return g.value


def nd_graph_launch(g, stream=None):
    _check(lib().nd_graph_launch(g, _stream(stream)))


def nd_graph_nodes(g):
    n = ctypes.c_int()
    _check(lib().nd_graph_nodes(g, ctypes.byref(n)))
    return n.value


def nd_graph_destroy(g):
    lib().nd_graph_destroy(g)


def nd_autotune_group(handles, methods, dt_seconds, n_steps=20, stream=None):
    """Tune the plans of several handles timed stepping side by side."""
    hs = (ctypes.c_void_p * len(handles))(*handles)
    ms = (ctypes.c_int * len(methods))(*methods)
    _check(lib().nd_autotune_group(ctypes.cast(hs, _P), ctypes.cast(ms, _P), len(handles), dt_seconds, n_steps,
                                   _stream(stream)))


def nd_autotune(h, method, dt_seconds, n_steps=20, stream=None):
    _check(lib().nd_autotune(h, method, dt_seconds, n_steps, _stream(stream)))


def nd_plan_info(h, cls):
    """dict(P, replicas, plan_rk4, plan_heun, threads_rk4, threads_heun) or None past the last class."""
    v = [ctypes.c_int() for _ in range(6)]
    rc = lib().nd_plan_info(h, cls, *[ctypes.byref(x) for x in v])
    if rc != ND_OK:
        return None
    return dict(zip(["P", "replicas", "plan_rk4", "plan_heun", "threads_rk4", "threads_heun"], [x.value for x in v]))


def nd_set_plan(h, cls, method, plan, check=True):
    rc = lib().nd_set_plan(h, cls, method, plan)
    if check:
        _check(rc)
    return rc
