"""Variants of the geometry and the drive (Sec. II.A): non-circular elements
(nd_set_mask: a square, an ellipse, an annulus) and a time-dependent external
field (nd_set_field_schedule: a field pulse), through the C ABI against the
FP64 oracle given the same mask or schedule."""
import numpy as np
import pytest
import torch

import ndsynth
import paper_1207_2192_gb300 as nd
from paper_1207_2192_gb300 import Disk, Nanodisk

pytestmark = pytest.mark.gpu

TOL = {nd.ND_FP32: 1e-5, nd.ND_FP64: 1e-11}


def rel(a, b, mask):
    return np.linalg.norm((np.asarray(a) - np.asarray(b)) * mask) / np.linalg.norm(np.asarray(b) * mask)


def shapes(D):
    idx = np.arange(D) - 0.5 * (D - 1)
    x, y = np.meshgrid(idx, idx, indexing="xy")
    r = 0.5 * D
    return {"square": np.ones((D, D), np.uint8),
            "ellipse": ((x / r) ** 2 + (y / (0.55 * r)) ** 2 <= 1).astype(np.uint8),
            "annulus": ((x * x + y * y <= r * r) & (x * x + y * y >= (0.4 * r) ** 2)).astype(np.uint8)}


@pytest.mark.parametrize("prec", [nd.ND_FP32, nd.ND_FP64])
@pytest.mark.parametrize("R", [13e-9, 30e-9, 70e-9])          # P = 32, 64 (on chip) and 256 (global path)
@pytest.mark.parametrize("shape", ["square", "ellipse", "annulus"])
def test_masked_field_and_energy_match_oracle(O, prec, R, shape):
    disk = Disk(R, 6e-9, hext=(1e4, -2e4, 5e3))
    h = Nanodisk([disk], [2], prec)
    model = O.Model(R, disk.L, hext=disk.hext)
    mk = shapes(model.D)[shape]
    h.set_mask(0, mk)
    model.set_mask(mk)
    assert np.array_equal(h.mask(0), mk)
    assert h.layout[0]["cells"] == model.C == int(mk.sum())
    grids = [ndsynth.random_unit_vectors(model.D, seed=s) for s in (5, 6)]      # nonzero outside the mask too
    b = h.unpack(h.field(h.to_device(grids)))
    E = h.energy(h.to_device(grids))
    stored = h.unpack(h.to_device(grids))            # the states as the handle's precision holds them
    for g, bg, Eg, gs in zip(grids, b, E, stored):
        ref = model.field(g * mk)
        assert rel(bg, ref, mk) < TOL[prec]
        assert np.all(bg[:, mk == 0] == 0)
        assert Eg == pytest.approx(model.energy(gs * mk), rel=1e-12)


@pytest.mark.parametrize("prec", [nd.ND_FP32, nd.ND_FP64])
@pytest.mark.parametrize("R", [30e-9, 70e-9])
def test_masked_trajectories_match_oracle(O, prec, R):
    """RK4 and Heun on an elliptical element, and its vortex core."""
    disk = Disk(R, 6e-9, alpha=0.05)
    h = Nanodisk([disk], [1], prec)
    model = O.Model(R, disk.L, alpha=disk.alpha)
    mk = shapes(model.D)["ellipse"]
    h.set_mask(0, mk)
    model.set_mask(mk)
    g = model.init_vortex(2e-9, -1e-9)
    dt = 1e-14
    m = h.to_device([g])
    h.rk4(m, 3, dt)
    ref = model.rk4(g, 3, model.dtau(dt))
    out = h.unpack(m)[0]
    assert rel(out - g, ref - g, mk) < 20 * TOL[prec]
    m = h.to_device([g])
    h.heun(m, 3, dt, [300.0], [9], step0=4)
    ref = model.heun(g, 3, model.dtau(dt), O.scaled_temperature(300.0, disk.A, disk.L), 9, 4)
    out = h.unpack(m)[0]
    assert rel(out - g, ref - g, mk) < 20 * TOL[prec]
    Xc, st = h.vortex_core(h.to_device([g]))
    so, xo, _ = model.vortex_core(g)
    assert st[0] == 0 and so == 0
    assert np.allclose(Xc[0], xo, rtol=0, atol=1e-12 * disk.R)


def pulse(n_on, n_total, H):
    hs = np.zeros((n_total, 3))
    hs[:n_on] = H
    return hs


@pytest.mark.parametrize("prec", [nd.ND_FP32, nd.ND_FP64])
@pytest.mark.parametrize("R", [30e-9, 70e-9])
def test_field_pulse_trajectories_match_oracle(O, prec, R):
    """An in-plane field pulse for the first steps (the paper's way of
    displacing the core before a release), then the static field; RK4 and
    Heun against the oracle with the same schedule, run in two calls."""
    disk = Disk(R, 6e-9, alpha=0.02, hext=(0.0, 0.0, 2e3))
    h = Nanodisk([disk], [2], prec)
    model = O.Model(R, disk.L, alpha=disk.alpha, hext=disk.hext)
    hs = pulse(3, 5, (4e4, -1e4, 0.0))
    h.set_field_schedule(0, hs)
    model.set_schedule(hs)
    g = model.init_vortex(0.0, 1e-9)
    dt = 2e-14
    m = h.to_device([g, g])
    h.rk4(m, 2, dt)                      # steps 0, 1
    h.rk4(m, 5, dt)                      # steps 2 .. 6: the pulse ends inside this call
    ref = model.rk4(g, 7, model.dtau(dt))
    out = h.unpack(m)
    for r in range(2):
        assert rel(out[r] - g, ref - g, model.mask) < 20 * TOL[prec]
    # the pulse matters: the same steps without it end elsewhere
    assert rel(ref, O.Model(R, disk.L, alpha=disk.alpha, hext=disk.hext).rk4(g, 7, model.dtau(dt)), model.mask) > 1e-6
    m = h.to_device([g, g])
    Ts = O.scaled_temperature(200.0, disk.A, disk.L)
    h.heun(m, 4, dt, [200.0, 200.0], [1, 2], step0=1)     # steps 1 .. 4
    out = h.unpack(m)
    for r in range(2):
        ref = model.heun(g, 4, model.dtau(dt), Ts, r + 1, 1)
        assert rel(out[r] - g, ref - g, model.mask) < 20 * TOL[prec]


def test_field_schedule_in_graph_replays_and_removal(O):
    """RK4 graph replays advance the schedule's step index like consecutive
    calls; removing the schedule restores the static field."""
    disk = Disk(30e-9, 5e-9, alpha=0.02)
    hs = pulse(6, 6, (0.0, 3e4, 0.0))
    ha = Nanodisk([disk], [1], nd.ND_FP32)
    hb = Nanodisk([disk], [1], nd.ND_FP32)
    model = O.Model(disk.R, disk.L, alpha=disk.alpha)
    g = model.init_vortex(1e-9, 0.0)
    ma, mb = ha.to_device([g]), hb.to_device([g])
    ha.set_field_schedule(0, hs)
    hb.set_field_schedule(0, hs)
    gr = nd.nd_graph_create(ha.h, ma, nd.ND_METHOD_RK4, 2, 2e-14, step0=0)
    for _ in range(4):
        nd.nd_graph_launch(gr)             # steps 0-1, 2-3, 4-5, 6-7
    nd.nd_graph_destroy(gr)
    for _ in range(4):
        hb.rk4(mb, 2, 2e-14)               # the handle's RK4 step index advances per call
    torch.cuda.synchronize()
    assert bool((ma == mb).all())
    model.set_schedule(hs)
    ref = model.rk4(g, 8, model.dtau(2e-14))
    assert rel(ha.unpack(ma)[0] - g, ref - g, model.mask) < 20 * TOL[nd.ND_FP32]
    model.set_schedule(None)
    hb.set_field_schedule(0, None)
    mc = hb.to_device([g])
    hb.rk4(mc, 3, 2e-14)
    ref = model.rk4(g, 3, model.dtau(2e-14))
    assert rel(hb.unpack(mc)[0] - g, ref - g, model.mask) < 20 * TOL[nd.ND_FP32]
