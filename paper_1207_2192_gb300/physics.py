"""Host-side analysis on top of the library calls: the force constant k_F
from constrained relaxations (Eq. Ux), its thickness derivative by the
envelope theorem, the gyrotropic frequency from a core trajectory, and the
Thiele relation (Eq. OG).  The field, relaxations and energies run in the
CUDA library; this module only fits numbers."""
from __future__ import annotations

import math

import numpy as np

from ._binding import ND_ERR_NOT_CONVERGED, ND_OK, nd_energy


def kF_map(h, xs, tol=1e-6, max_iter=40000, stream=None):
    """Relax one replica per core position x (along x, metres) of a
    single-disk handle with len(xs) replicas and fit U(x) = U(0) + kF x^2/2.

    Returns dict with U (J units), U_J (joules), kF_fit (N/m, least squares
    over x^2 with the x = 0 point), kF_2pt (from the first nonzero x),
    dkF_dL (N/m^2, envelope theorem on the same two states), lam, iters.
    """
    xs = np.asarray(xs, dtype=np.float64)
    assert h.B == len(xs) and xs[0] == 0.0
    X = np.stack([xs, np.zeros_like(xs)], 1)
    m = h.empty_device()
    h.init_vortex(m, X)
    rc, U, lam, it = h.relax(m, X, tol=tol, max_iter=max_iter, stream=stream)
    if rc not in (ND_OK, ND_ERR_NOT_CONVERGED):
        raise RuntimeError(f"relaxation failed ({rc})")
    E, dEdL = nd_energy(h.h, m, h.B, stream, with_dL=True)
    J = h.units[0][4]
    UJ = E * J
    xn = xs / 1e-9                                   # fit in nanometres (well conditioned)
    A = np.stack([np.ones_like(xn), 0.5 * xn ** 2], 1)
    coef, *_ = np.linalg.lstsq(A, UJ, rcond=None)
    coef[1] /= 1e-18                                 # J/nm^2 -> J/m^2
    x1 = xs[1]
    kF_2pt = 2.0 * (UJ[1] - UJ[0]) / x1 ** 2
    dkF_dL = 2.0 * (dEdL[1] - dEdL[0]) / x1 ** 2
    return dict(U=E, U_J=UJ, kF_fit=coef[1], kF_2pt=kF_2pt, dkF_dL=dkF_dL, dEdL=dEdL, lam=lam, iters=it,
                converged=(rc == ND_OK), state=m)


def dkF_d_aspect(dkF_dL, R):
    """d kF / d(L/R) at fixed radius and mask: R dkF/dL."""
    return R * dkF_dL


def omega_from_core(xc, yc, dtau):
    """Dimensionless angular frequency of gyrotropic motion: slope of the
    unwrapped polar angle of the core position against tau (least squares)."""
    phi = np.unwrap(np.arctan2(np.asarray(yc), np.asarray(xc)))
    t = np.arange(len(phi)) * dtau
    return np.polyfit(t, phi, 1)[0]


def omega_thiele(kF, a, L, A, Q=1):
    """Omega_G = -kF a^2 / (4 pi L A Q) (Eq. OG)."""
    return -kF * a * a / (4.0 * math.pi * L * A * Q)


def spectrum_peak(freq, psd, kmin=1):
    """Frequency of the largest peak of a power spectrum (bins k >= kmin),
    refined by a parabola through the logarithms of the peak bin and its two
    neighbours."""
    freq, psd = np.asarray(freq, dtype=np.float64), np.asarray(psd, dtype=np.float64)
    k = kmin + int(np.argmax(psd[kmin:]))
    if k <= 0 or k >= len(psd) - 1:
        return float(freq[k])
    a, b, c = np.log(psd[k - 1:k + 2])
    den = a - 2 * b + c
    d = 0.0 if den == 0 else 0.5 * (a - c) / den
    return float(freq[k] + d * (freq[1] - freq[0]))


MU0 = 4.0e-7 * math.pi


def geometry_sweep(Rs, Ls, a=2e-9, tol=1e-5, max_iter=60000, precision=None, stream=None):
    """Force constant, Thiele frequency and thickness derivative of a set of
    disks (Sec. IV's scan of f_G, k_F/L and Omega_G against L/R), all in one
    handle: two replicas per disk, cores pinned at X = 0 and X = 2a, relaxed
    in one batched call over every size class.

    Returns one dict per disk with R, L, aspect = L/R, kF (N/m, two-point
    Eq. Ux), kF_per_L, kF_scaled = kF / (mu0 Ms^2 L^2 / R) (the paper's fit
    reads ~0.878), Omega (Thiele, Eq. OG, per time unit), f_G (Hz), dkF_dL
    (envelope theorem), iters and converged."""
    from . import Disk, Nanodisk
    from ._binding import ND_FP32
    disks = [Disk(R, L, a=a) for R, L in zip(Rs, Ls)]
    h = Nanodisk(disks, [2] * len(disks), ND_FP32 if precision is None else precision)
    X = np.zeros((h.B, 2))
    X[1::2, 0] = 2 * a
    m = h.empty_device()
    h.init_vortex(m, X, stream=stream)
    rc, U, lam, it = h.relax(m, X, tol=tol, max_iter=max_iter, stream=stream)
    if rc not in (ND_OK, ND_ERR_NOT_CONVERGED):
        raise RuntimeError(f"relaxation failed ({rc})")
    E, dEdL = nd_energy(h.h, m, h.B, stream, with_dL=True)
    out = []
    for d, disk in enumerate(disks):
        J = h.units[d][4]
        t0 = h.units[d][3]
        i0, i1 = 2 * d, 2 * d + 1
        kF = 2.0 * (E[i1] - E[i0]) * J / (2 * a) ** 2
        om = omega_thiele(kF, a, disk.L, disk.A)
        out.append(dict(R=disk.R, L=disk.L, aspect=disk.L / disk.R, kF=kF, kF_per_L=kF / disk.L,
                        kF_scaled=kF / (MU0 * disk.Ms ** 2 * disk.L ** 2 / disk.R), Omega=om,
                        f_G=abs(om) / (2 * math.pi) / t0, dkF_dL=2.0 * (dEdL[i1] - dEdL[i0]) / (2 * a) ** 2,
                        iters=(int(it[i0]), int(it[i1])), converged=bool(it[i0] < max_iter and it[i1] < max_iter)))
    return out
