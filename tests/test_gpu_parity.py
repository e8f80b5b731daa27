"""GPU parity: the CUDA library against the FP64 oracle, element by element,
on the same seeded inputs, through the C ABI.

Tolerances (relative L2 over the disk cells, unless stated):
  FP64: 1e-11 for fields and short trajectories, FP32: 1e-5 (the target
  accuracy of the method's FP32 field); energies are evaluated in FP64 by both
  sides and agree to 1e-12 relative; integer decisions (vortex plaquette) are
  taken in FP64 by both sides and must agree exactly.
"""
import numpy as np
import pytest

import ndsynth
import paper_1207_2192_gb300 as nd
from paper_1207_2192_gb300 import Disk, Nanodisk

pytestmark = pytest.mark.gpu

TOL = {nd.ND_FP32: 1e-5, nd.ND_FP64: 1e-11}


def rel(a, b, mask):
    a = np.asarray(a) * mask
    b = np.asarray(b) * mask
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def oracle_model(O, disk: Disk):
    return O.Model(disk.R, disk.L, disk.a, disk.Ms, disk.A, disk.gamma, disk.alpha, disk.hext, disk.polarity,
                   disk.chirality)


# geometries spanning every padded size class: (R, L) -> D, P
GEOMS = [
    (3e-9, 4e-9),      # D=3,  P=16 (tiny, ragged)
    (7e-9, 5e-9),      # D=7,  P=16
    (13e-9, 3e-9),     # D=13, P=32 (odd D)
    (30e-9, 5e-9),     # D=30, P=64  (config 1)
    (33e-9, 8e-9),     # D=33, P=128 (just above a class boundary)
    (50e-9, 10e-9),    # D=50, P=128 (config 3)
    (60e-9, 10e-9),    # D=60, P=128 (config 2)
    (70e-9, 12e-9),    # D=70, P=256 (global path)
]


@pytest.mark.parametrize("prec", [nd.ND_FP32, nd.ND_FP64])
@pytest.mark.parametrize("R,L", GEOMS)
def test_effective_field_matches_direct_sum(O, prec, R, L):
    disk = Disk(R, L, hext=(1.5e4, -2.0e4, 3.0e4))
    h = Nanodisk([disk], [2], prec)
    model = oracle_model(O, disk)
    assert h.layout[0]["D"] == model.D and h.layout[0]["cells"] == model.C
    assert np.array_equal(h.mask(0), model.mask)
    grids = [ndsynth.random_unit_vectors(model.D, seed=s) * model.mask for s in (1, 2)]
    m = h.to_device(grids)
    b = h.unpack(h.field(m))
    for g, bg in zip(grids, b):
        ref = model.field(g)
        assert rel(bg, ref, model.mask) < TOL[prec]
        assert np.all(bg[:, model.mask == 0] == 0)


def test_field_ignores_values_outside_disk(O):
    disk = Disk(20e-9, 5e-9)
    h = Nanodisk([disk], [1], nd.ND_FP64)
    model = oracle_model(O, disk)
    g = ndsynth.random_unit_vectors(model.D, seed=4)            # nonzero outside the disk
    b = h.unpack(h.field(h.to_device([g])))[0]
    ref = model.field(g * model.mask)
    assert rel(b, ref, model.mask) < 1e-11


def test_host_buffers_match_device_buffers(O):
    disk = Disk(25e-9, 5e-9)
    h = Nanodisk([disk], [3], nd.ND_FP32)
    model = oracle_model(O, disk)
    grids = [ndsynth.random_unit_vectors(model.D, seed=s) * model.mask for s in range(3)]
    host = h.pack(grids)
    bh = np.zeros_like(host)
    nd.nd_effective_field(h.h, host, bh)
    bd = h.field(h.to_device(grids)).cpu().numpy()
    assert np.array_equal(bh, bd)


@pytest.mark.parametrize("prec", [nd.ND_FP32, nd.ND_FP64])
@pytest.mark.parametrize("R,L,nsteps", [(12e-9, 5e-9, 1), (12e-9, 5e-9, 25), (30e-9, 5e-9, 3), (50e-9, 10e-9, 2),
                                        (70e-9, 12e-9, 2)])
def test_rk4_matches_oracle(O, prec, R, L, nsteps):
    disk = Disk(R, L, alpha=0.05, hext=(0, 0, 2e4))
    h = Nanodisk([disk], [1], prec)
    model = oracle_model(O, disk)
    g = model.init_vortex(2.5e-9, -1.0e-9)
    g = (ndsynth.perturbed(g, 0.05, seed=3) * model.mask)
    g /= np.where(model.mask, np.linalg.norm(g, axis=0), 1.0)
    dt = 2e-14
    m = h.to_device([g])
    h.rk4(m, nsteps, dt)
    out = h.unpack(m)[0]
    ref = model.rk4(g, nsteps, model.dtau(dt))
    assert np.max(np.abs(out - ref)) < 10 * TOL[prec]
    assert rel(out - g, ref - g, model.mask) < 20 * TOL[prec]


@pytest.mark.parametrize("prec", [nd.ND_FP32, nd.ND_FP64])
@pytest.mark.parametrize("R,L,nsteps,T", [(12e-9, 5e-9, 1, 300.0), (12e-9, 5e-9, 20, 300.0), (30e-9, 5e-9, 4, 300.0),
                                          (50e-9, 10e-9, 3, 300.0), (50e-9, 10e-9, 3, 0.0), (70e-9, 12e-9, 2, 400.0)])
def test_heun_matches_oracle(O, prec, R, L, nsteps, T):
    disk = Disk(R, L, alpha=0.02)
    h = Nanodisk([disk], [2], prec)
    model = oracle_model(O, disk)
    g = model.init_vortex(0.0, 0.0)
    dt = 1e-14
    seeds = [7, 123456789012345]
    m = h.to_device([g, g])
    h.heun(m, nsteps, dt, [T, T], seeds, step0=11)
    out = h.unpack(m)
    Ts = O.scaled_temperature(T, disk.A, disk.L)
    for r in range(2):
        ref = model.heun(g, nsteps, model.dtau(dt), Ts, seeds[r], 11)
        assert np.max(np.abs(out[r] - ref)) < 10 * TOL[prec]
        assert rel(out[r] - g, ref - g, model.mask) < 20 * TOL[prec]
    if T > 0:
        assert not np.allclose(out[0], out[1])


def test_heun_resume_is_bit_identical(O):
    disk = Disk(20e-9, 5e-9, alpha=0.02)
    h = Nanodisk([disk], [1], nd.ND_FP32)
    model = oracle_model(O, disk)
    g = model.init_vortex(1e-9, 0.0)
    a = h.to_device([g])
    h.heun(a, 10, 1e-14, [300.0], [5], step0=0)
    b = h.to_device([g])
    h.heun(b, 4, 1e-14, [300.0], [5], step0=0)
    h.heun(b, 6, 1e-14, [300.0], [5], step0=4)
    assert bool((a == b).all())


@pytest.mark.parametrize("prec", [nd.ND_FP32, nd.ND_FP64])
@pytest.mark.parametrize("R,L", [(7e-9, 5e-9), (30e-9, 5e-9), (60e-9, 10e-9), (70e-9, 12e-9)])
def test_energy_matches_oracle(O, prec, R, L):
    disk = Disk(R, L, hext=(2e4, 0, -1e4))
    h = Nanodisk([disk], [2], prec)
    model = oracle_model(O, disk)
    grids = [model.init_vortex(2e-9, 1e-9), ndsynth.random_unit_vectors(model.D, seed=8) * model.mask]
    m = h.to_device(grids)
    E = h.energy(m)
    exact = h.unpack(m)       # the state as stored (FP32-rounded for FP32 handles)
    for r in range(2):
        ref = model.energy(exact[r])
        assert E[r] == pytest.approx(ref, rel=1e-12, abs=1e-9)


@pytest.mark.parametrize("prec", [nd.ND_FP32, nd.ND_FP64])
def test_init_vortex_and_core_match_oracle(O, prec):
    disk = Disk(30e-9, 5e-9)
    X0 = np.array([[3.3e-9, -1.7e-9], [-6.0e-9, 4.2e-9], [0.0, 0.0]])
    h = Nanodisk([disk], [3], prec)
    model = oracle_model(O, disk)
    m = h.empty_device()
    h.init_vortex(m, X0)
    grids = h.unpack(m)
    for r in range(3):
        ref = model.init_vortex(*X0[r])
        assert np.max(np.abs(grids[r] - ref)) < (1e-6 if prec == nd.ND_FP32 else 1e-13)
    # perturb to make the core estimator work on a noisy state
    noisy = [ndsynth.perturbed(g, 0.2, seed=10 + r) * model.mask for r, g in enumerate(grids)]
    m2 = h.to_device(noisy)
    Xc, st = h.vortex_core(m2)
    exact = h.unpack(m2)
    for r in range(3):
        s_ref, xc_ref, _ = model.vortex_core(exact[r])
        assert st[r] == (0 if s_ref == 0 else nd.ND_ERR_NO_VORTEX)
        if s_ref == 0:
            assert np.allclose(Xc[r], xc_ref, rtol=0, atol=1e-12 * disk.R)


def test_core_reports_no_vortex(O):
    disk = Disk(20e-9, 5e-9)
    h = Nanodisk([disk], [1], nd.ND_FP32)
    model = oracle_model(O, disk)
    g = np.zeros((3, model.D, model.D)); g[0] = model.mask
    Xc, st = h.vortex_core(h.to_device([g]))
    assert st[0] == nd.ND_ERR_NO_VORTEX


def test_mean_m_matches_oracle(O):
    disk = Disk(30e-9, 5e-9)
    h = Nanodisk([disk], [2], nd.ND_FP32)
    model = oracle_model(O, disk)
    grids = [model.init_vortex(4e-9, 0.0), ndsynth.random_unit_vectors(model.D, seed=2) * model.mask]
    m = h.to_device(grids)
    mm = h.mean_m(m)
    exact = h.unpack(m)
    for r in range(2):
        assert np.allclose(mm[r], model.mean_m(exact[r]), atol=1e-12)


def test_uneven_batch_matches_oracle(O):
    """Disks of different radius and thickness (three FFT size classes) in one
    handle: every replica matches its own oracle."""
    disks = [Disk(9e-9, 2e-9), Disk(21e-9, 3e-9), Disk(40e-9, 6e-9), Disk(26e-9, 5.2e-9)]
    h = Nanodisk(disks, [1, 2, 1, 1], nd.ND_FP32)
    grids, models = [], []
    for r in range(h.B):
        mdl = oracle_model(O, disks[h.rep_disk[r]])
        models.append(mdl)
        grids.append(ndsynth.random_unit_vectors(mdl.D, seed=30 + r) * mdl.mask)
    b = h.unpack(h.field(h.to_device(grids)))
    for r in range(h.B):
        assert rel(b[r], models[r].field(grids[r]), models[r].mask) < 1e-5
