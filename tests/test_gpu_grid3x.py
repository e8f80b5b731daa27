"""The non-power-of-two padded grids (ND_GRID_3X) P = 192 = 8 x 24 for disks
of 65..96 cells and P = 200 = 10 x 20 (radix-5 register DFTs, ten-lane FFT
groups) for disks of 97..100 cells, against the FP64 oracle's direct sum: any
P >= 2D - 1 gives the linear convolution exactly (the paper's power-of-two
rule of Sec. II.B is a convenience), so the field, trajectories and
relaxation sweeps must match the oracle to the same tolerances as on the
power-of-two grids."""
import numpy as np
import pytest

import ndsynth
import paper_1207_2192_gb300 as nd
from paper_1207_2192_gb300 import Disk, Nanodisk

pytestmark = pytest.mark.gpu

TOL = {nd.ND_FP32: 1e-5, nd.ND_FP64: 1e-11}


def rel(a, b, mask):
    return np.linalg.norm((np.asarray(a) - np.asarray(b)) * mask) / np.linalg.norm(np.asarray(b) * mask)


def traj_ok(out, ref, start, mask, prec, C):
    """Trajectory error against 20x the field tolerance times the change over
    the run, plus the rounding of the stored state (~1e-7 per FP32 component)."""
    change = np.linalg.norm((ref - start) * mask)
    floor = (1e-7 if prec == nd.ND_FP32 else 1e-15) * np.sqrt(3 * C)
    return np.linalg.norm((out - ref) * mask) <= 20 * TOL[prec] * change + floor


@pytest.mark.parametrize("prec", [nd.ND_FP32, nd.ND_FP64])
@pytest.mark.parametrize("R", [65e-9, 81e-9, 96e-9])          # D = 65 (the smallest), 81 (odd), 96 (the largest)
def test_grid192_field_matches_direct_sum(O, prec, R):
    disk = Disk(R, 9e-9, hext=(1e4, 2e4, -1e4))
    h = Nanodisk([disk], [2], prec, grid3x=True)
    assert h.layout[0]["P"] == 192
    assert Nanodisk([disk], [1], prec).layout[0]["P"] == 256      # without the flag
    model = O.Model(R, disk.L, hext=disk.hext)
    grids = [ndsynth.random_unit_vectors(model.D, seed=s) * model.mask for s in (1, 2)]
    b = h.unpack(h.field(h.to_device(grids)))
    for g, bg in zip(grids, b):
        assert rel(bg, model.field(g), model.mask) < TOL[prec]


@pytest.mark.parametrize("prec", [nd.ND_FP32, nd.ND_FP64])
@pytest.mark.parametrize("R", [97e-9, 99e-9, 100e-9])   # D = 97 (the smallest, odd), 99, 100 (the largest)
def test_grid200_field_matches_direct_sum(O, prec, R):
    disk = Disk(R, 9e-9, hext=(1e4, 2e4, -1e4))
    h = Nanodisk([disk], [2], prec, grid3x=True)
    assert h.layout[0]["P"] == 200
    assert Nanodisk([disk], [1], prec).layout[0]["P"] == 256      # without the flag
    model = O.Model(R, disk.L, hext=disk.hext)
    grids = [ndsynth.random_unit_vectors(model.D, seed=s) * model.mask for s in (3, 4)]
    b = h.unpack(h.field(h.to_device(grids)))
    for g, bg in zip(grids, b):
        assert rel(bg, model.field(g), model.mask) < TOL[prec]


@pytest.mark.parametrize("prec", [nd.ND_FP32, nd.ND_FP64])
@pytest.mark.parametrize("R", [90e-9, 100e-9])                 # P = 192, 200
def test_grid3x_trajectories_match_oracle(O, prec, R):
    disk = Disk(R, 10e-9, alpha=0.02)
    h = Nanodisk([disk], [2], prec, grid3x=True)
    assert h.layout[0]["P"] == (192 if R < 97e-9 else 200)
    model = O.Model(disk.R, disk.L, alpha=disk.alpha)
    g = model.init_vortex(3e-9, -2e-9)
    dt = 1e-14
    m = h.to_device([g, g])
    h.rk4(m, 2, dt)
    ref = model.rk4(g, 2, model.dtau(dt))
    start = h.unpack(h.to_device([g]))[0]
    for out in h.unpack(m):
        assert traj_ok(out, ref, start, model.mask, prec, model.C)
    m = h.to_device([g, g])
    h.heun(m, 3, dt, [300.0, 300.0], [4, 5], step0=2)
    Ts = O.scaled_temperature(300.0, disk.A, disk.L)
    for r, out in enumerate(h.unpack(m)):
        ref = model.heun(g, 3, model.dtau(dt), Ts, 4 + r, 2)
        assert traj_ok(out, ref, start, model.mask, prec, model.C)


def test_grid3x_relaxation_sweeps_and_mixed_classes(O):
    """Relaxation sweeps on the P = 192 and P = 200 classes inside a handle
    that also holds an on-chip class (D = 30, P = 64) and a P = 256 class
    (D = 110)."""
    ds = [Disk(30e-9, 10e-9), Disk(70e-9, 10e-9), Disk(110e-9, 10e-9), Disk(98e-9, 10e-9)]
    h = Nanodisk(ds, [1, 1, 1, 1], nd.ND_FP32, grid3x=True)
    assert [h.layout[r]["P"] for r in range(4)] == [64, 192, 256, 200]
    X = np.array([[2e-9, 0.0], [2.5e-9, 1e-9], [0.0, -2e-9], [1.5e-9, 1.5e-9]])
    grids = [O.Model(d.R, d.L).init_vortex(0.0, 0.0) for d in ds]
    m = h.to_device(grids)
    rc, U, lam, it = h.relax(m, X, tol=1e-300, max_iter=3)
    out = h.unpack(m)
    start = h.unpack(h.to_device(grids))
    for r, d in enumerate(ds):
        model = O.Model(d.R, d.L)
        mm, lm = start[r], np.zeros(2)
        for _ in range(3):
            mm, lm, _ = model.relax_sweep(mm, X[r], lm)
        assert np.max(np.abs(out[r] - mm)) < 2e-4
        assert np.allclose(lam[r], lm, rtol=2e-3, atol=2e-3 * max(1e-3, np.abs(lm).max()))
    # a Heun step of every class
    m = h.to_device(grids)
    h.heun(m, 2, 1e-14, [300.0] * 4, [7, 8, 9, 10], step0=0)
    out = h.unpack(m)
    for r, d in enumerate(ds):
        model = O.Model(d.R, d.L)
        ref = model.heun(start[r], 2, model.dtau(1e-14), O.scaled_temperature(300.0, d.A, d.L), 7 + r, 0)
        assert traj_ok(out[r], ref, start[r], model.mask, nd.ND_FP32, model.C)
