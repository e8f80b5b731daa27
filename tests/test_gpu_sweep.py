"""Batched geometry sweep (Sec. IV's scan of k_F and Omega_G against L/R):
nine disks of three thicknesses and three radii relaxed in one call over the
on-chip and global size classes.

* Every relaxation converges; k_F > 0; k_F rises with L at fixed R and falls
  with R at fixed L.
* The force constants follow the paper's scaling k_F ~ 0.878 mu0 Ms^2 L^2/R:
  the median ratio within 15%, every disk within a factor 0.5..1.4 (the
  paper's constant is one fit over its whole range).
* Batched dynamics of three disks (undamped RK4 from X = 2a, <m_y> spectra,
  one CUDA graph): the gyration frequencies match the Thiele frequencies of
  the static k_F to the 0-15% the constraint reading leaves (the static k_F
  is systematically low).
"""
import math

import numpy as np
import pytest

import paper_1207_2192_gb300 as nd
from paper_1207_2192_gb300 import Disk, Nanodisk
from paper_1207_2192_gb300.physics import geometry_sweep, spectrum_peak

pytestmark = pytest.mark.gpu


def test_sweep_force_constants_follow_the_paper_scaling():
    Rs = [30e-9, 60e-9, 120e-9] * 3
    Ls = [5e-9] * 3 + [10e-9] * 3 + [20e-9] * 3
    res = geometry_sweep(Rs, Ls)
    for r in res:
        print(f"R={r['R']*1e9:5.0f} nm L={r['L']*1e9:4.0f} nm L/R={r['aspect']:.3f} kF={r['kF']:.4e} N/m "
              f"kF/(mu0 Ms^2 L^2/R)={r['kF_scaled']:.3f} f_G={r['f_G']/1e9:.3f} GHz iters={r['iters']}")
        assert r["converged"] and r["kF"] > 0
    kF = np.array([r["kF"] for r in res]).reshape(3, 3)           # [L][R]
    assert np.all(np.diff(kF, axis=0) > 0)                        # thicker: stiffer
    assert np.all(np.diff(kF, axis=1) < 0)                        # wider: softer
    # the paper's fitted constant is a single number over its range; here it
    # drifts from ~0.55 (L/R = 0.67) to ~1.1 (L/R = 0.04)
    scaled = np.array([r["kF_scaled"] for r in res])
    assert np.median(scaled) == pytest.approx(0.878, rel=0.15)
    assert np.all((scaled > 0.5 * 0.878) & (scaled < 1.4 * 0.878))


def test_batched_gyration_frequencies_match_thiele():
    a = 2e-9
    geoms = [(30e-9, 5e-9), (30e-9, 10e-9), (60e-9, 20e-9)]
    stat = geometry_sweep([g[0] for g in geoms], [g[1] for g in geoms])
    h = Nanodisk([Disk(R, L, alpha=0.0) for R, L in geoms], None, nd.ND_FP32)
    X = np.array([[2 * a, 0.0]] * len(geoms))
    m = h.empty_device()
    h.init_vortex(m, X)
    rc, *_ = h.relax(m, X, tol=1e-5, max_iter=60000)
    assert rc == nd.ND_OK
    t0 = h.units[0][3]
    dtau, every, window = 0.04, 250, 1024                         # a sample every 10 time units
    nd.nd_series_reset(h.h, window)
    g = nd.nd_graph_create(h.h, m, nd.ND_METHOD_RK4, every, dtau * t0, stats_sample=nd.ND_GRAPH_SERIES)
    for _ in range(window):
        nd.nd_graph_launch(g)
    nd.nd_graph_destroy(g)
    psd, freq, nw = nd.nd_power_spectrum(h.h, h.B, 1, window, every * dtau * t0)
    assert nw == 1 and nd.nd_check_status(h.h) == nd.ND_OK
    for r, s in enumerate(stat):
        f = spectrum_peak(freq, psd[r])
        print(f"R={s['R']*1e9:.0f} nm L={s['L']*1e9:.0f} nm: f_G dynamic {f/1e9:.4f} GHz, Thiele {s['f_G']/1e9:.4f} GHz")
        # the static k_F of the constraint reading (c6) sits 5-12% below the
        # value the dynamics imply, more so for thicker disks
        assert 1.0 <= f / s["f_G"] <= 1.15
