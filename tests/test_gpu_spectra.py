"""Time series of <m> and their power spectra on the GPU (Sec. V: the
thermal spectra of <m_x> whose peaks give the gyrotropic frequency).

* A series of prescribed uniform states: the recorded <m> equals the
  prescribed values, and the averaged periodogram equals the FP64 oracle's
  (a direct DFT of each window, pinned by Parseval and a pure tone) and
  numpy's FFT of the prescribed series under the same definition.
* Graph replays with ND_GRAPH_SERIES append one sample each, equal to <m>.
* Physics: the peak of the <m_y> spectrum of a released undamped vortex is
  the gyrotropic frequency of its core trajectory in the same run.
"""
import math

import numpy as np
import pytest
import torch

import paper_1207_2192_gb300 as nd
from paper_1207_2192_gb300 import Disk, Nanodisk
from paper_1207_2192_gb300.physics import omega_from_core, spectrum_peak

pytestmark = pytest.mark.gpu


def numpy_psd(x, window, dt):
    """The documented estimator written out with numpy's FFT."""
    nwin = len(x) // window
    acc = np.zeros(window // 2 + 1)
    for w in range(nwin):
        seg = x[w * window:(w + 1) * window]
        X = np.fft.rfft(seg - seg.mean())
        acc += np.abs(X) ** 2
    psd = acc / nwin * dt / window
    psd[1:-1] *= 2
    return psd, np.arange(window // 2 + 1) / (window * dt)


def test_power_spectrum_of_prescribed_series_matches_oracle(O):
    disk = Disk(10e-9, 3e-9)
    h = Nanodisk([disk], [2], nd.ND_FP32)
    D = h.layout[0]["D"]
    mask = h.mask(0).astype(bool)
    n, window, dt = 1024 + 37, 256, 2.5e-12
    t = np.arange(n)
    f = np.array([[0.031, 0.2], [0.125, 0.0625]])           # cycles per sample: in-plane angle, m_z
    series = np.zeros((2, n, 3))
    for r in range(2):
        th = 2 * np.pi * f[r, 0] * t + 0.3 * r
        z = 0.4 * np.sin(2 * np.pi * f[r, 1] * t)
        s = np.sqrt(1 - z * z)
        series[r] = np.stack([s * np.cos(th), s * np.sin(th), z], 1)
    nd.nd_series_reset(h.h, 2048)
    for i in range(n):
        grids = []
        for r in range(2):
            g = np.zeros((3, D, D))
            for c in range(3):
                g[c][mask] = series[r, i, c]
            grids.append(g)
        nd.nd_series_sample(h.h, h.to_device(grids))
    taken, got = nd.nd_series_read(h.h, 2, 2048)
    assert taken == n and got.shape == (2, n, 3)
    # the recorded values are the prescribed ones up to their FP32 storage
    assert np.max(np.abs(got - series)) < 1e-7
    for comp in range(3):
        psd, freq, nw = nd.nd_power_spectrum(h.h, 2, comp, window, dt)
        assert nw == n // window
        for r in range(2):
            # the recorded series (FP32 states averaged in FP64) is the input of both
            orc, nwo = O.power_spectrum(got[r, :, comp], window, dt)
            assert nwo == nw
            assert np.max(np.abs(psd[r] - orc)) <= 1e-10 * orc.max()
            ref, fref = numpy_psd(series[r, :, comp], window, dt)
            assert np.allclose(freq, fref, rtol=1e-14)
            assert np.max(np.abs(psd[r] - ref)) <= 1e-6 * ref.max()
    # the in-plane angle's frequency is the peak of the <m_x> spectrum (to
    # within a bin: 0.031 cycles per sample falls between bins 7 and 8)
    psd, freq, _ = nd.nd_power_spectrum(h.h, 2, 0, window, dt)
    assert abs(spectrum_peak(freq, psd[0]) - f[0, 0] / dt) <= freq[1]
    with pytest.raises(nd.NDError):
        nd.nd_power_spectrum(h.h, 2, 0, 2048, dt)            # not a supported window
    nd.nd_series_reset(h.h, 100)
    with pytest.raises(nd.NDError):
        nd.nd_power_spectrum(h.h, 2, 0, 64, dt)              # fewer samples than one window


def test_graph_replays_append_series_samples():
    disk = Disk(30e-9, 5e-9, alpha=0.01)
    h = Nanodisk([disk], [3], nd.ND_FP32)
    m = h.empty_device()
    h.init_vortex(m, np.array([[4e-9, 0.0], [0.0, 3e-9], [-2e-9, -2e-9]]))
    nd.nd_series_reset(h.h, 8)
    g = nd.nd_graph_create(h.h, m, nd.ND_METHOD_RK4, 20, 2e-14, stats_sample=nd.ND_GRAPH_SERIES)
    means = []
    for _ in range(3):
        nd.nd_graph_launch(g)
        torch.cuda.synchronize()
        means.append(h.mean_m(m))
    nd.nd_graph_destroy(g)
    taken, got = nd.nd_series_read(h.h, 3, 8)
    assert taken == 3
    for i in range(3):
        assert np.allclose(got[:, i, :], means[i], rtol=0, atol=1e-12)


def test_gyration_frequency_from_the_magnetisation_spectrum():
    """R = 30 nm, L = 5 nm released from X = 2a with alpha = 0 (RK4): the
    peak of the <m_y> spectrum equals the core's gyration frequency in the
    same run, and both agree with the paper's tau_G ~ 2020 (Sec. IV.B)."""
    a = 2e-9
    h = Nanodisk([Disk(30e-9, 5e-9, alpha=0.0)], [1], nd.ND_FP32)
    m = h.empty_device()
    h.init_vortex(m, [[2 * a, 0.0]])
    rc, *_ = h.relax(m, [[2 * a, 0.0]], tol=1e-5, max_iter=60000)
    assert rc == nd.ND_OK
    t0 = h.units[0][3]
    dtau, every, window = 0.04, 500, 1024                   # a sample every 20 time units
    nd.nd_series_reset(h.h, window)
    xs, ys = [], []
    for _ in range(window):
        h.rk4(m, every, dtau * t0)
        nd.nd_series_sample(h.h, m)
        Xc, st = h.vortex_core(m)
        assert st[0] == 0
        xs.append(Xc[0, 0]); ys.append(Xc[0, 1])
    dts = every * dtau * t0
    psd, freq, nw = nd.nd_power_spectrum(h.h, 1, 1, window, dts)
    assert nw == 1
    f_psd = spectrum_peak(freq, psd[0])
    om = omega_from_core(xs, ys, every * dtau)              # radians per time unit
    f_core = abs(om) / (2 * math.pi) / t0
    tau_psd = 1.0 / (f_psd * t0)
    print(f"f_psd={f_psd:.5e} Hz  f_core={f_core:.5e} Hz  tau_G(psd)={tau_psd:.0f}")
    assert f_psd == pytest.approx(f_core, rel=0.01)
    assert tau_psd == pytest.approx(2020.0, rel=0.05)
