"""GPU constrained relaxation against the oracle: sweep by sweep (state and
Lagrange multipliers), converged energies, and the force constant k_F of
Eq. Ux from two relaxed positions."""
import numpy as np
import pytest

import paper_1207_2192_gb300 as nd
from paper_1207_2192_gb300 import Disk, Nanodisk

pytestmark = pytest.mark.gpu


def model_for(O, disk):
    return O.Model(disk.R, disk.L, disk.a, disk.Ms, disk.A, disk.gamma, disk.alpha, disk.hext, disk.polarity,
                   disk.chirality)


@pytest.mark.parametrize("prec,tol", [(nd.ND_FP64, 1e-11), (nd.ND_FP32, 2e-5)])
@pytest.mark.parametrize("R,L,nsweep", [(16e-9, 10e-9, 1), (16e-9, 10e-9, 6), (30e-9, 10e-9, 3)])
def test_relax_sweeps_match_oracle(O, prec, tol, R, L, nsweep):
    disk = Disk(R, L)
    h = Nanodisk([disk], [2], prec)
    model = model_for(O, disk)
    X = np.array([[2.5e-9, 1.0e-9], [0.0, 0.0]])
    grids = [model.init_vortex(0.0, 0.0), model.init_vortex(-1e-9, 2e-9)]
    m = h.to_device(grids)
    rc, U, lam, it = h.relax(m, X, tol=1e-300, max_iter=nsweep)
    assert rc == nd.ND_ERR_NOT_CONVERGED and np.all(it == nsweep)
    out = h.unpack(m)
    start = h.unpack(h.to_device(grids))     # the inputs as the GPU saw them
    for r in range(2):
        mm, lm = start[r], np.zeros(2)
        for _ in range(nsweep):
            mm, lm, _ = model.relax_sweep(mm, X[r], lm)
        assert np.max(np.abs(out[r] - mm)) < 10 * tol
        assert np.allclose(lam[r], lm, rtol=100 * tol, atol=100 * tol * max(1e-3, np.abs(lm).max()))
        assert U[r] == pytest.approx(model.energy(out[r]), rel=1e-12)


def test_relaxed_energies_and_kF_match_oracle(O):
    """Converged relaxations at X = 0 and X = 2a: FP64 GPU energies agree with
    the oracle's to 1e-9 relative; k_F (FP64 and FP32 relaxations, FP64
    energies) within 1e-3."""
    disk = Disk(30e-9, 10e-9)
    a = disk.a
    model = model_for(O, disk)
    Xs = np.array([[0.0, 0.0], [2 * a, 0.0]])
    ref = {}
    for X in Xs:
        r = model.relax(model.init_vortex(*X), X, tol=1e-9, max_iter=20000)
        assert r["status"] == 0
        ref[X[0]] = r["U"]
    kF_ref = O.kF_from_energies(ref[0.0] * model.J, ref[2 * a] * model.J, 2 * a)
    for prec, tol in ((nd.ND_FP64, 1e-9), (nd.ND_FP32, 1e-5)):
        h = Nanodisk([disk], [2], prec)
        m = h.empty_device()
        h.init_vortex(m, Xs)
        rc, U, lam, it = h.relax(m, Xs, tol=tol, max_iter=20000)
        assert rc == nd.ND_OK, it
        if prec == nd.ND_FP64:
            assert U[0] == pytest.approx(ref[0.0], rel=1e-9)
            assert U[1] == pytest.approx(ref[2 * a], rel=1e-9)
        kF = O.kF_from_energies(U[0] * model.J, U[1] * model.J, 2 * a)
        assert kF == pytest.approx(kF_ref, rel=1e-3)
        # the relaxed core sits at the constraint position
        Xc, st = h.vortex_core(m)
        assert np.all(st == 0) and abs(Xc[1, 0] - 2 * a) < 0.1 * a


@pytest.mark.parametrize("prec,tol,disks", [
    (nd.ND_FP32, 2e-5, [(66e-9, 10e-9)]),                  # P = 256: global path
    (nd.ND_FP64, 1e-11, [(40e-9, 10e-9)]),                 # P = 128 in FP64: global path
    (nd.ND_FP32, 2e-5, [(30e-9, 10e-9), (66e-9, 10e-9)]),  # one fused and one global size class
])
def test_global_path_relax_sweeps_match_oracle(O, prec, tol, disks):
    """The relaxation sweeps of the global path (sizes the on-chip kernel does
    not hold) against the oracle sweep by sweep, in a handle that may mix size
    classes."""
    nsweep = 3
    ds = [Disk(R, L) for R, L in disks]
    h = Nanodisk(ds, [2] * len(ds), prec)
    X = np.array([[2.5e-9, 1.0e-9], [0.0, -2e-9]] * len(ds))
    grids = []
    for d in ds:
        model = model_for(O, d)
        grids += [model.init_vortex(0.0, 0.0), model.init_vortex(-1e-9, 2e-9)]
    m = h.to_device(grids)
    rc, U, lam, it = h.relax(m, X, tol=1e-300, max_iter=nsweep)
    assert rc == nd.ND_ERR_NOT_CONVERGED and np.all(it == nsweep)
    out = h.unpack(m)
    start = h.unpack(h.to_device(grids))
    for r in range(h.B):
        model = model_for(O, ds[h.rep_disk[r]])
        mm, lm = start[r], np.zeros(2)
        for _ in range(nsweep):
            mm, lm, _ = model.relax_sweep(mm, X[r], lm)
        assert np.max(np.abs(out[r] - mm)) < 10 * tol
        assert np.allclose(lam[r], lm, rtol=100 * tol, atol=100 * tol * max(1e-3, np.abs(lm).max()))
        assert U[r] == pytest.approx(model.energy(out[r]), rel=1e-12)


def test_global_path_relax_converges_to_oracle_energy(O):
    """A converged FP64 relaxation on the global path (P = 128 in FP64) ends at
    the oracle's energy and multipliers, and stops early: every replica reports
    its own sweep count below max_iter."""
    disk = Disk(40e-9, 10e-9)
    model = model_for(O, disk)
    X = np.array([3e-9, 0.0])
    ref = model.relax(model.init_vortex(*X), X, tol=1e-9, max_iter=20000)
    assert ref["status"] == 0
    h = Nanodisk([disk], [1], nd.ND_FP64)
    m = h.empty_device()
    h.init_vortex(m, X.reshape(1, 2))
    rc, U, lam, it = h.relax(m, X.reshape(1, 2), tol=1e-9, max_iter=20000)
    assert rc == nd.ND_OK
    assert 0 < it[0] < 20000 and abs(int(it[0]) - ref["iters"]) <= 1
    assert U[0] == pytest.approx(ref["U"], rel=1e-9)
    assert np.allclose(lam[0], ref["lam"], rtol=1e-5, atol=1e-8)
