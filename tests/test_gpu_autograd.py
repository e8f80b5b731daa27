"""The autograd energy: dE/dm against central finite differences (FP64,
config-2 disk, 50 random cells, step 1e-6) and against the oracle's field;
dE/dL against finite differences of the oracle energy in L; dk_F/dL by the
envelope theorem against finite differences of k_F over L; the constrained
relaxation driven by the autograd gradient against the library's and the
oracle's sweeps; dk_F/d(L/R) as the backward of the force constant over the
uneven 64-disk batch against finite differences."""
import numpy as np
import pytest
import torch

import ndsynth
import paper_1207_2192_gb300 as nd
from paper_1207_2192_gb300 import Disk, Nanodisk
from paper_1207_2192_gb300.autograd import energy
from paper_1207_2192_gb300.physics import kF_map

pytestmark = pytest.mark.gpu


def test_energy_gradient_matches_finite_differences_and_oracle(O):
    disk = Disk(60e-9, 10e-9, hext=(1e4, 0.0, 5e3))
    h = Nanodisk([disk], [1], nd.ND_FP64)
    model = O.Model(disk.R, disk.L, hext=disk.hext)
    g = model.init_vortex(4e-9, 0.0)
    g = ndsynth.perturbed(g, 0.05, seed=5) * model.mask
    m = h.to_device([g]).requires_grad_(True)
    L = torch.tensor(disk.L, dtype=torch.float64, requires_grad=True)
    E = energy(m, L, h)
    E.sum().backward()
    J = h.units[0][4]
    grad = h.unpack(m.grad)[0]
    # the oracle gradient: dE/dm = -J b
    assert np.linalg.norm((grad + J * model.field(g)) * model.mask) <= 1e-11 * np.linalg.norm(J * model.field(g))
    # central differences on 50 random cells of the disk, all three components
    inside = np.flatnonzero(model.mask.ravel())
    cells = inside[ndsynth.sample_indices(len(inside), 50, seed=0)]
    base = h.pack([g])
    L0 = h.layout[0]
    # the energy is a quadratic form, so central differences have no truncation
    # error; what remains is FP64 rounding of |E| (~5e3 J units) over the step,
    # about 1e-12/1e-6 = 1e-6 of the typical gradient component
    scale = np.abs(grad).max()
    for c in cells:
        j, i = divmod(int(c), model.D)
        for k in range(3):
            idx = L0["offset"] + k * L0["D"] * L0["Dpad"] + j * L0["Dpad"] + i
            hstep = 1e-6
            p, q = base.copy(), base.copy()
            p[idx] += hstep
            q[idx] -= hstep
            Ep = nd.nd_energy(h.h, torch.from_numpy(p).cuda(), 1)[0] * J
            Eq = nd.nd_energy(h.h, torch.from_numpy(q).cuda(), 1)[0] * J
            fd = (Ep - Eq) / (2 * hstep)
            assert abs(fd - grad[k, j, i]) <= 2e-6 * scale


def test_dE_dL_matches_finite_differences_of_the_oracle(O):
    disk = Disk(30e-9, 6e-9)
    h = Nanodisk([disk], [2], nd.ND_FP64)
    model = O.Model(disk.R, disk.L)
    grids = [model.init_vortex(2e-9, 0.0), ndsynth.random_unit_vectors(model.D, seed=3) * model.mask]
    m = h.to_device(grids)
    E, dEdL = nd.nd_energy(h.h, m, 2, with_dL=True)
    exact = h.unpack(m)
    dL = 1e-4 * disk.L
    for r in range(2):
        mp, mm = O.Model(disk.R, disk.L + dL), O.Model(disk.R, disk.L - dL)
        fd = (mp.energy(exact[r]) * mp.J - mm.energy(exact[r]) * mm.J) / (2 * dL)
        assert dEdL[r] == pytest.approx(fd, rel=1e-6)
    # autograd path for L
    L = torch.tensor(disk.L, dtype=torch.float64, requires_grad=True)
    energy(m, L, h).sum().backward()
    assert L.grad.item() == pytest.approx(dEdL.sum(), rel=1e-12)


def test_dkF_dL_envelope_matches_finite_differences():
    R, L, a = 30e-9, 10e-9, 2e-9
    xs = np.array([0.0, 2 * a])
    res = {}
    for Lv in (L - 0.2e-9, L, L + 0.2e-9):
        h = Nanodisk([Disk(R, Lv)], [2], nd.ND_FP64)
        res[Lv] = kF_map(h, xs, tol=1e-10, max_iter=60000)
        assert res[Lv]["converged"]
    fd = (res[L + 0.2e-9]["kF_2pt"] - res[L - 0.2e-9]["kF_2pt"]) / 0.4e-9
    assert res[L]["dkF_dL"] == pytest.approx(fd, rel=2e-3)
    assert res[L]["kF_2pt"] > 0 and res[L]["dkF_dL"] > 0    # k_F grows with thickness (Sec. IV.B)


def test_energy_gradient_drives_the_constrained_relaxation(O):
    """relax_by_energy_gradient: every sweep takes its field from the autograd
    gradient of the energy (nd_relax_sweep_grad).  Sweep by sweep it is the
    library's own relaxation and the oracle's; run to convergence it reaches
    the same energy; an extra torch energy term (a uniaxial anisotropy) enters
    the relaxation through the same gradient."""
    from paper_1207_2192_gb300.autograd import relax_by_energy_gradient
    disk = Disk(16e-9, 10e-9)
    model = O.Model(disk.R, disk.L)
    X = np.array([[2.5e-9, 1.0e-9], [0.0, 0.0]])
    grids = [model.init_vortex(0.0, 0.0), model.init_vortex(-1e-9, 2e-9)]
    nsweep = 6
    ha = Nanodisk([disk], [2], nd.ND_FP64)
    ma = ha.to_device(grids)
    out = relax_by_energy_gradient(ha, ma, X, tol=1e-300, max_iter=nsweep)
    assert not out["converged"] and out["iters"] == nsweep
    hb = Nanodisk([disk], [2], nd.ND_FP64)
    mb = hb.to_device(grids)
    rc, U, lam, it = hb.relax(mb, X, tol=1e-300, max_iter=nsweep)
    assert np.max(np.abs((ma - mb).cpu().numpy())) < 1e-11
    assert np.allclose(out["lam"], lam, rtol=1e-9, atol=1e-12)
    got = ha.unpack(ma)
    for r in range(2):
        mm, lm = grids[r], np.zeros(2)
        for _ in range(nsweep):
            mm, lm, _ = model.relax_sweep(mm, X[r], lm)
        assert np.max(np.abs(got[r] - mm)) < 1e-10
        assert np.allclose(out["lam"][r], lm, rtol=1e-8, atol=1e-10)
    # to convergence (the R = 30 nm disk, cores at X = 2a and 0): the same
    # energy as the library's relaxation
    disk = Disk(30e-9, 10e-9)
    model = O.Model(disk.R, disk.L)
    X = np.array([[4e-9, 0.0], [0.0, 0.0]])
    grids = [model.init_vortex(*X[0]), model.init_vortex(*X[1])]
    ha, hb = Nanodisk([disk], [2], nd.ND_FP64), Nanodisk([disk], [2], nd.ND_FP64)
    ma, mb = ha.to_device(grids), hb.to_device(grids)
    out = relax_by_energy_gradient(ha, ma, X, tol=1e-9, max_iter=20000)
    rc, U, lam, it = hb.relax(mb, X, tol=1e-9, max_iter=20000)
    print(f"gradient-driven: converged {out['converged']} after {out['iters']} sweeps, resid {out['resid']}; "
          f"library: rc {rc}, sweeps {it}")
    assert out["converged"] and rc == nd.ND_OK
    assert abs(out["iters"] - int(it.max())) <= 1
    assert np.allclose(ha.energy(ma), U, rtol=1e-9)
    # an anisotropy -K sum m_z^2 (joules) added in torch pulls the state out of
    # plane; the relaxation still converges under the constraint
    mc = ha.to_device(grids)
    K = 0.02 * ha.units[0][4]

    def anisotropy(m):
        e = 0.0
        for L0 in ha.layout:
            n = L0["D"] * L0["Dpad"]
            z = m[L0["offset"] + 2 * n:L0["offset"] + 3 * n]
            e = e - K * (z * z).sum()
        return e

    out_k = relax_by_energy_gradient(ha, mc, X, tol=1e-8, max_iter=20000, extra_energy=anisotropy)
    print(f"with the anisotropy: converged {out_k['converged']} after {out_k['iters']} sweeps")
    assert out_k["converged"]
    gz = [g[2][model.mask.astype(bool)] for g in ha.unpack(mc)]
    g0 = [g[2][model.mask.astype(bool)] for g in ha.unpack(ma)]
    assert all((a ** 2).sum() > (b ** 2).sum() for a, b in zip(gz, g0))
    for r in range(2):
        assert np.max(np.abs(model.constraint(ha.unpack(mc)[r], X[r]))) < 1e-6


def test_dkF_d_aspect_backward_over_the_uneven_batch():
    """Config 4's 64 disks (R ~ U(20, 100) nm, L/R ~ U(0.05, 0.2)), every size
    class in one batched relaxation: k_F as a function of L/R with
    dk_F/d(L/R) from the backward pass, against central differences of the
    forward (aspect ratios changed by 2%, the radii and masks fixed)."""
    from paper_1207_2192_gb300.autograd import force_constants
    R, L, _ = ndsynth.uneven_disks(64, seed=0)
    asp = torch.tensor(L / R, dtype=torch.float64, requires_grad=True)
    kF = force_constants(asp, R)
    kF.sum().backward()
    grad = asp.grad.numpy()
    eps = 0.02
    kp = force_constants(asp.detach() * (1 + eps), R).numpy()
    km = force_constants(asp.detach() * (1 - eps), R).numpy()
    fd = (kp - km) / (2 * eps * asp.detach().numpy())
    k0 = kF.detach().numpy()
    ok = (k0 > 0) & (kp > 0) & (km > 0)
    print(f"{ok.sum()} of 64 disks hold a vortex at all three aspect ratios")
    assert ok.sum() >= 48
    relerr = np.abs(grad[ok] - fd[ok]) / np.abs(fd[ok])
    print(f"dkF/d(L/R): backward vs central differences, median rel. diff {np.median(relerr):.2e}, max {relerr.max():.2e}")
    assert np.median(relerr) < 0.01
    assert np.all(relerr < 0.05)
    assert np.all(grad[ok] > 0)                     # thicker disks are stiffer (Sec. IV.B)
