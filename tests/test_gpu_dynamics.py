"""Long-trajectory checks against the FP64 oracle and the paper:

* Config 1 (Sec. III.A): an undamped FP64 RK4 run of 2000 steps at
  dt = 5 fs conserves the energy to better than 12 digits, and its final
  state matches the oracle's run from the same relaxed state.
* Omega_G (Eq. OG, dynamic side): the gyration frequency of a released
  vortex, from the core track of the GPU run and of the oracle's run from the
  same relaxed state, each with its own estimator, agrees to 1e-3.
* k_F of the batched geometry sweep (Eq. Ux), one disk of each size class
  (on-chip P = 64 and 128, global path P = 256), against the oracle's
  relaxations to 1e-3.
"""
import math

import numpy as np
import pytest

import paper_1207_2192_gb300 as nd
from paper_1207_2192_gb300 import Disk, Nanodisk
from paper_1207_2192_gb300.physics import geometry_sweep, omega_from_core

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def disk_30_5(O):
    """R = 30 nm, L = 5 nm (configs 1, Sec. IV.B) relaxed by the oracle with
    the core pinned at X = (3 nm, 0) and at X = (2a, 0)."""
    model = O.Model(30e-9, 5e-9)
    out = {}
    for X in (3e-9, 4e-9):
        r = model.relax(model.init_vortex(X, 0.0), (X, 0.0), tol=1e-10, max_iter=40000)
        assert r["status"] == 0
        out[X] = r["m"]
    return model, out


def test_config1_fp64_rk4_conserves_energy_and_matches_oracle(O, disk_30_5):
    model, relaxed = disk_30_5
    g = relaxed[3e-9]
    disk = Disk(30e-9, 5e-9, alpha=0.0)
    h = Nanodisk([disk], [1], nd.ND_FP64)
    m = h.to_device([g])
    dt = 5e-15
    assert model.dtau(dt) == pytest.approx(0.0066512, rel=1e-4)
    E0 = h.energy(m)[0]
    drift = 0.0
    for _ in range(4):
        h.rk4(m, 500, dt)
        drift = max(drift, abs(h.energy(m)[0] - E0) / abs(E0))
    print(f"config 1: E0 = {E0:.12f} J-units, max relative drift over 2000 steps = {drift:.2e}")
    assert drift <= 1e-12                               # Sec. III.A: better than 12 digits
    out = h.unpack(m)[0]
    n = np.sqrt((out ** 2).sum(0))[model.mask.astype(bool)]
    assert np.max(np.abs(n - 1)) < 1e-14
    ref = model.rk4(g, 2000, model.dtau(dt))
    assert np.max(np.abs(out - ref)) < 1e-10
    change = np.linalg.norm((ref - g) * model.mask)
    assert change > 1e-4
    assert np.linalg.norm((out - ref) * model.mask) < 1e-8 * change


def test_gyration_frequency_matches_oracle(O, disk_30_5):
    """Release the oracle-relaxed vortex from X = 2a, undamped RK4 at
    dtau = 0.04 (the paper's step) for one gyration period, core sampled every
    10 time units; Omega_G from each side's track and estimator."""
    model, relaxed = disk_30_5
    g = relaxed[4e-9]
    dtau, every, nsamp = 0.04, 250, 206                 # 206 x 10 = 2060 time units ~ one period
    xo, yo = [], []
    mo = g
    for _ in range(nsamp):
        mo = model.rk4(mo, every, dtau)
        st, xc, _ = model.vortex_core(mo)
        assert st == 0
        xo.append(xc[0]); yo.append(xc[1])
    om_orc = O.omega_from_track(np.array(xo), np.array(yo), every * dtau)
    tau_G = 2 * math.pi / abs(om_orc)
    print(f"oracle Omega_G = {om_orc:.6e} (tau_G = {tau_G:.1f})")
    assert om_orc < 0 and tau_G == pytest.approx(2020.0, rel=0.05)
    for prec in (nd.ND_FP64, nd.ND_FP32):
        h = Nanodisk([Disk(30e-9, 5e-9, alpha=0.0)], [1], prec)
        m = h.to_device([g])
        dt = dtau * h.units[0][3]
        xs, ys = [], []
        for _ in range(nsamp):
            h.rk4(m, every, dt)
            Xc, st = h.vortex_core(m)
            assert st[0] == 0
            xs.append(Xc[0, 0]); ys.append(Xc[0, 1])
        om = omega_from_core(xs, ys, every * dtau)
        print(f"prec {prec}: Omega_G = {om:.6e}, relative to the oracle {om / om_orc - 1:+.2e}")
        assert om == pytest.approx(om_orc, rel=1e-3)
        if prec == nd.ND_FP64:
            assert np.max(np.abs(np.array(xs) - xo)) < 1e-3 * 4e-9


def test_sweep_force_constants_match_oracle(O):
    """One disk per size class of the sweep: D = 30 (P = 64), D = 60 (P = 128,
    config 2's disk) and D = 66 (P = 256, the global path), relaxed together in
    one batched FP32 call; k_F against the oracle's FP64 relaxations."""
    geoms = [(30e-9, 5e-9), (60e-9, 10e-9), (66e-9, 10e-9)]
    res = geometry_sweep([g[0] for g in geoms], [g[1] for g in geoms], tol=1e-6)
    a = 2e-9
    for (R, L), r in zip(geoms, res):
        assert r["converged"]
        model = O.Model(R, L)
        U = []
        for X in (0.0, 2 * a):
            o = model.relax(model.init_vortex(X, 0.0), (X, 0.0), tol=1e-8, max_iter=40000)
            assert o["status"] == 0
            U.append(o["U"])
        kF_ref = O.kF_from_energies(U[0] * model.J, U[1] * model.J, 2 * a)
        print(f"R={R*1e9:.0f} nm L={L*1e9:.0f} nm: kF GPU {r['kF']:.6e}  oracle {kF_ref:.6e}  "
              f"rel {r['kF'] / kF_ref - 1:+.2e}")
        assert r["kF"] == pytest.approx(kF_ref, rel=1e-3)
