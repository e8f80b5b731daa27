"""FP64 CPU oracle for the thin-nanodisk micromagnetics hot path.

TEST INFRASTRUCTURE.  This package is the independent reference the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the product package never
does, and this package never imports the product package.

The arithmetic lives in ``nd_oracle.c`` (plain C, double precision, an O(C^2)
direct dipolar sum).  This module compiles it with gcc on first use and wraps
it with ctypes.  Arrays are numpy float64 of shape (3, D, D): component, row
(y index), column (x index).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libndoracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (OpenMP if available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fPIC", "-shared", _SRC,
            "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class Disk(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double), ("L", ctypes.c_double), ("a", ctypes.c_double),
                ("Ms", ctypes.c_double), ("A", ctypes.c_double), ("gamma", ctypes.c_double),
                ("alpha", ctypes.c_double), ("hext", ctypes.c_double * 3),
                ("polarity", ctypes.c_int), ("chirality", ctypes.c_int)]


_D = ctypes.c_double
_P = ctypes.c_void_p
_I = ctypes.c_int


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            sig = {
                "ndo_units": (None, [_D, _D, _D, _D, _D, _P, _P, _P, _P, _P]),
                "ndo_scaled_temperature": (_D, [_D, _D, _D]),
                "ndo_sigma_s": (_D, [_D, _D, _D]),
                "ndo_gyrovector": (_D, [_D, _D, _D, _I]),
                "ndo_omega_G": (_D, [_D, _D, _D, _D, _I]),
                "ndo_kF_from_energies": (_D, [_D, _D, _D]),
                "ndo_p_r": (_D, [_D, _D, _D]),
                "ndo_gyro_mass": (_D, [_D, _D]),
                "ndo_f_V": (_D, [_D, _D, _D]),
                "ndo_omega_from_track": (_D, [_P, _P, _I, _D]),
                "ndo_power_spectrum": (_I, [_P, ctypes.c_long, _I, _D, _P]),
                "ndo_grid_side": (_I, [_D, _D]),
                "ndo_mask": (_I, [_D, _D, _I, _P]),
                "ndo_green": (None, [_D, _D, _D, _P]),
                "ndo_self_factors": (None, [_D, _D, _P, _P]),
                "ndo_model_size": (ctypes.c_size_t, []),
                "ndo_model_init": (_I, [_P, _P]),
                "ndo_model_free": (None, [_P]),
                "ndo_model_D": (_I, [_P]),
                "ndo_model_C": (_I, [_P]),
                "ndo_model_params": (None, [_P, _P]),
                "ndo_model_mask": (None, [_P, _P]),
                "ndo_model_set_alpha": (None, [_P, _D]),
                "ndo_model_set_green": (None, [_P, _P]),
                "ndo_model_set_mask": (_I, [_P, _P]),
                "ndo_model_set_schedule": (_I, [_P, ctypes.c_long, _P, _D]),
                "ndo_rk4_at": (None, [_P, _P, ctypes.c_long, _D, ctypes.c_uint64]),
                "ndo_demag": (None, [_P, _P, _P]),
                "ndo_field": (None, [_P, _P, _P]),
                "ndo_field_parts": (None, [_P, _P, _P, _P]),
                "ndo_field_at": (None, [_P, _P, _P, _I, _P]),
                "ndo_energy": (_D, [_P, _P]),
                "ndo_pair_count": (ctypes.c_long, [_P]),
                "ndo_llg_rhs": (None, [_P, _P, _P, _D, _P]),
                "ndo_rk4": (None, [_P, _P, ctypes.c_long, _D]),
                "ndo_philox4x32_10": (None, [_P, _P, _P]),
                "ndo_thermal_normals": (None, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, _P]),
                "ndo_normals_block": (None, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, _P]),
                "ndo_heun": (None, [_P, _P, ctypes.c_long, _D, _D, ctypes.c_uint64, ctypes.c_uint64]),
                "ndo_init_vortex": (None, [_P, _D, _D, _P]),
                "ndo_vortex_core": (_I, [_P, _P, _P, _P]),
                "ndo_mean_m": (None, [_P, _P, _P]),
                "ndo_constraint": (None, [_P, _P, _P, _P]),
                "ndo_relax_sweep": (_D, [_P, _P, _P, _P, _D]),
                "ndo_relax": (_I, [_P, _P, _P, _D, _I, _D, _P, _P, _P, _P]),
                "ndo_num_threads": (_I, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------- helpers

PERMALLOY = dict(Ms=8.6e5, A=1.3e-11, gamma=1.76e11)


def units(A, Ms, a, L, gamma):
    """(lambda_ex, B0, t0, J, a^2/lambda^2) of Section III.A."""
    out = [ctypes.c_double() for _ in range(5)]
    lib().ndo_units(A, Ms, a, L, gamma, *[ctypes.byref(o) for o in out])
    return tuple(o.value for o in out)


def scaled_temperature(T, A, L):
    return lib().ndo_scaled_temperature(T, A, L)


def sigma_s(alpha, Ts, dtau):
    return lib().ndo_sigma_s(alpha, Ts, dtau)


def gyrovector(L, Ms, gamma, Q):
    return lib().ndo_gyrovector(L, Ms, gamma, Q)


def omega_G(kF, a, L, A, Q):
    return lib().ndo_omega_G(kF, a, L, A, Q)


def kF_from_energies(U0, Ux, x):
    return lib().ndo_kF_from_energies(U0, Ux, x)


def p_r(r, kF, kT):
    return lib().ndo_p_r(r, kF, kT)


def gyro_mass(G, kF):
    return lib().ndo_gyro_mass(G, kF)


def f_V(V, mG, kT):
    return lib().ndo_f_V(V, mG, kT)


def omega_from_track(xc, yc, dtau):
    """Slope of the continuous polar angle of a core track against tau."""
    xc = np.ascontiguousarray(xc, dtype=np.float64)
    yc = np.ascontiguousarray(yc, dtype=np.float64)
    assert xc.shape == yc.shape and xc.ndim == 1
    return lib().ndo_omega_from_track(_ptr(xc), _ptr(yc), len(xc), dtau)


def power_spectrum(x, window, dt):
    """Averaged one-sided periodogram of a series; returns (psd, n_windows)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    psd = np.zeros(window // 2 + 1)
    nw = lib().ndo_power_spectrum(_ptr(x), len(x), window, dt, _ptr(psd))
    return psd, nw


def green(x, y, L):
    g = np.zeros(4)
    lib().ndo_green(x, y, L, _ptr(g))
    return g


def self_factors(L, a):
    nx, nz = ctypes.c_double(), ctypes.c_double()
    lib().ndo_self_factors(L, a, ctypes.byref(nx), ctypes.byref(nz))
    return nx.value, nz.value


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    o = np.zeros(4, dtype=np.uint32)
    lib().ndo_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def thermal_normals(seed, cell, step):
    w = np.zeros(3)
    lib().ndo_thermal_normals(seed, cell, step, _ptr(w))
    return w


def normals_block(seed, step, ncell):
    out = np.zeros((ncell, 3))
    lib().ndo_normals_block(seed, step, ncell, _ptr(out))
    return out


class Model:
    """One disk geometry with its precomputed direct-sum Green's table."""

    def __init__(self, R, L, a=2e-9, Ms=8.6e5, A=1.3e-11, gamma=1.76e11, alpha=0.0,
                 hext=(0.0, 0.0, 0.0), polarity=1, chirality=1):
        self.disk = Disk(R, L, a, Ms, A, gamma, alpha, (ctypes.c_double * 3)(*hext), polarity, chirality)
        self._buf = ctypes.create_string_buffer(lib().ndo_model_size())
        rc = lib().ndo_model_init(ctypes.byref(self.disk), self._buf)
        if rc != 0:
            raise ValueError(f"ndo_model_init failed ({rc})")
        self.D = lib().ndo_model_D(self._buf)
        p = np.zeros(8)
        lib().ndo_model_params(self._buf, _ptr(p))
        self.lambda_ex, self.c, self.B0, self.t0, self.J, self.Nx, self.Nz, C = p
        self.C = int(C)
        self.mask = np.zeros((self.D, self.D), dtype=np.uint8)
        lib().ndo_model_mask(self._buf, _ptr(self.mask))
        self.R, self.L, self.a, self.Ms, self.A, self.gamma = R, L, a, Ms, A, gamma
        self.alpha = alpha

    def __del__(self):
        try:
            lib().ndo_model_free(self._buf)
        except Exception:
            pass

    def set_alpha(self, alpha):
        self.alpha = alpha
        lib().ndo_model_set_alpha(self._buf, alpha)

    def set_green(self, Gq):
        """Replace the Green's table by a quarter table [4][D][D] of a^2 G at
        displacements (dx, dy) >= 0 (components xx, yy, xy, zz; self terms at
        the origin), extended to negative displacements by symmetry."""
        Gq = np.ascontiguousarray(Gq, dtype=np.float64)
        assert Gq.shape == (4, self.D, self.D), Gq.shape
        lib().ndo_model_set_green(self._buf, _ptr(Gq))

    def quarter_table(self):
        """The closed-form quarter table of Sec. II.B for this geometry, built
        from the oracle's Green's function and self factors."""
        q = np.zeros((4, self.D, self.D))
        for dy in range(self.D):
            for dx in range(self.D):
                if dx == 0 and dy == 0:
                    q[:, 0, 0] = (-self.Nx, -self.Nx, 0.0, -self.Nz)
                else:
                    q[:, dy, dx] = green(dx * self.a, dy * self.a, self.L) * self.a ** 2
        return q

    def _state(self, m):
        m = np.ascontiguousarray(m, dtype=np.float64)
        assert m.shape == (3, self.D, self.D), m.shape
        return m

    def dtau(self, dt_seconds):
        return self.gamma * self.B0 * dt_seconds

    def demag(self, m):
        m = self._state(m)
        h = np.zeros_like(m)
        lib().ndo_demag(self._buf, _ptr(m), _ptr(h))
        return h

    def field(self, m):
        m = self._state(m)
        b = np.zeros_like(m)
        lib().ndo_field(self._buf, _ptr(m), _ptr(b))
        return b

    def field_at(self, m, cells):
        """Induction at flat cell indices j*D+i (direct sum), shape (n, 3)."""
        m = self._state(m)
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        out = np.zeros((len(cells), 3))
        lib().ndo_field_at(self._buf, _ptr(m), _ptr(cells), len(cells), _ptr(out))
        return out

    def field_parts(self, m):
        m = self._state(m)
        ex, hM = np.zeros_like(m), np.zeros_like(m)
        lib().ndo_field_parts(self._buf, _ptr(m), _ptr(ex), _ptr(hM))
        return ex, hM

    def energy(self, m):
        return lib().ndo_energy(self._buf, _ptr(self._state(m)))

    def pair_count(self):
        return lib().ndo_pair_count(self._buf)

    def llg_rhs(self, m, b, alpha):
        m, b = self._state(m), self._state(b)
        f = np.zeros_like(m)
        lib().ndo_llg_rhs(self._buf, _ptr(m), _ptr(b), alpha, _ptr(f))
        return f

    def rk4(self, m, nsteps, dtau, step0=0):
        """RK4 steps step0 .. step0 + nsteps - 1 (the index selects a scheduled field)."""
        m = self._state(m).copy()
        lib().ndo_rk4_at(self._buf, _ptr(m), nsteps, dtau, step0)
        return m

    def set_mask(self, mask):
        """Replace the disk mask by any cell set of the D x D grid."""
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        assert mk.shape == (self.D, self.D)
        self.C = lib().ndo_model_set_mask(self._buf, _ptr(mk))
        lib().ndo_model_mask(self._buf, _ptr(self.mask))

    def set_schedule(self, hs):
        """Per-step external field H_ext(s) in A/m, shape (n, 3); None clears."""
        if hs is None:
            lib().ndo_model_set_schedule(self._buf, 0, None, self.Ms)
            return
        hs = np.ascontiguousarray(hs, dtype=np.float64).reshape(-1, 3)
        lib().ndo_model_set_schedule(self._buf, len(hs), _ptr(hs), self.Ms)

    def heun(self, m, nsteps, dtau, Ts, seed, step0=0):
        m = self._state(m).copy()
        lib().ndo_heun(self._buf, _ptr(m), nsteps, dtau, Ts, seed, step0)
        return m

    def init_vortex(self, x0, y0):
        m = np.zeros((3, self.D, self.D))
        lib().ndo_init_vortex(self._buf, x0, y0, _ptr(m))
        return m

    def vortex_core(self, m):
        xc, rv = np.zeros(2), np.zeros(2)
        st = lib().ndo_vortex_core(self._buf, _ptr(self._state(m)), _ptr(xc), _ptr(rv))
        return st, xc, rv

    def mean_m(self, m):
        out = np.zeros(3)
        lib().ndo_mean_m(self._buf, _ptr(self._state(m)), _ptr(out))
        return out

    def constraint(self, m, X):
        X = np.asarray(X, dtype=np.float64)
        out = np.zeros(2)
        lib().ndo_constraint(self._buf, _ptr(self._state(m)), _ptr(X), _ptr(out))
        return out

    def relax_sweep(self, m, X, lam, eta=0.5):
        m = self._state(m).copy()
        X = np.asarray(X, dtype=np.float64).copy()
        lam = np.asarray(lam, dtype=np.float64).copy()
        res = lib().ndo_relax_sweep(self._buf, _ptr(m), _ptr(X), _ptr(lam), eta)
        return m, lam, res

    def relax(self, m, X, tol=1e-10, max_iter=20000, eta=0.5, lam=(0.0, 0.0)):
        m = self._state(m).copy()
        X = np.asarray(X, dtype=np.float64).copy()
        lam = np.asarray(lam, dtype=np.float64).copy()
        U, it, res = ctypes.c_double(), ctypes.c_int(), ctypes.c_double()
        st = lib().ndo_relax(self._buf, _ptr(m), _ptr(X), tol, max_iter, eta, ctypes.byref(U), _ptr(lam),
                             ctypes.byref(it), ctypes.byref(res))
        return dict(status=st, m=m, U=U.value, lam=lam, iters=it.value, resid=res.value)

    def cell_centres(self):
        """(x, y) arrays of cell centres in metres, shape (D, D)."""
        idx = (np.arange(self.D) - 0.5 * (self.D - 1)) * self.a
        return np.meshgrid(idx, idx, indexing="xy")


def num_threads():
    return lib().ndo_num_threads()
