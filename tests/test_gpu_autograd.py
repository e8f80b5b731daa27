"""The autograd energy: dE/dm against central finite differences (FP64,
config-2 disk, 50 random cells, step 1e-6) and against the oracle's field;
dE/dL against finite differences of the oracle energy in L; dk_F/dL by the
envelope theorem against finite differences of k_F over L."""
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
