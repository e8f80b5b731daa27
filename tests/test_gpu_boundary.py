"""The boundary calls that change a handle's physics after creation, through
the C ABI: nd_set_green_tensor (Sec. II.B, the spectral kernel from a user
table or rebuilt from the closed forms) and nd_set_damping (Sec. III.A,
per-replica alpha), against the FP64 oracle built with the same table or
damping."""
import numpy as np
import pytest

import ndsynth
import paper_1207_2192_gb300 as nd
from paper_1207_2192_gb300 import Disk, Nanodisk

pytestmark = pytest.mark.gpu


def rel(a, b, mask):
    return np.linalg.norm((np.asarray(a) - np.asarray(b)) * mask) / np.linalg.norm(np.asarray(b) * mask)


# (R, L): on-chip FP64 class (P = 64) and the global path (P = 256)
@pytest.mark.parametrize("R,L", [(30e-9, 5e-9), (70e-9, 12e-9)])
def test_set_green_tensor_rebuild_and_closed_form_table(O, R, L):
    disk = Disk(R, L, alpha=0.02, hext=(0.0, 1.2e4, -0.8e4))
    h = Nanodisk([disk], [2], nd.ND_FP64)
    model = O.Model(R, L, hext=disk.hext)
    grids = [ndsynth.random_unit_vectors(model.D, seed=s) * model.mask for s in (41, 42)]
    m = h.to_device(grids)
    b0 = h.field(m).clone()
    # (i) Gq = NULL after a damping change: the rebuilt kernel is the same, bit for bit
    h.set_damping([0.3, 0.07])
    h.set_green_tensor(0, None)
    assert bool((h.field(m) == b0).all())
    # (ii) the oracle's own quarter table reproduces the default field
    h.set_green_tensor(0, model.quarter_table())
    b = h.unpack(h.field(m))
    for g, bg in zip(grids, b):
        assert rel(bg, model.field(g), model.mask) < 1e-11


@pytest.mark.parametrize("prec,tol", [(nd.ND_FP64, 1e-11), (nd.ND_FP32, 1e-5)])
@pytest.mark.parametrize("R,L", [(30e-9, 5e-9), (70e-9, 12e-9)])
def test_set_green_tensor_user_table_matches_oracle_with_that_table(O, prec, tol, R, L):
    """(iii) a modified tensor -- G_zz halved, G_xy scaled by 1.5 and a perturbed
    self term -- against the oracle model given the same table."""
    disk = Disk(R, L, hext=(2e4, 0.0, 1e4))
    h = Nanodisk([disk], [1], prec)
    model = O.Model(R, L, hext=disk.hext)
    q = model.quarter_table()
    q[3] *= 0.5
    q[2] *= 1.5
    q[0, 0, 0] *= 1.1
    model.set_green(q)
    h.set_green_tensor(0, q)
    g = ndsynth.random_unit_vectors(model.D, seed=43) * model.mask
    b = h.unpack(h.field(h.to_device([g])))[0]
    ref = model.field(g)
    assert rel(b, ref, model.mask) < tol
    # and it differs from the default field by far more than the tolerance
    assert rel(ref, O.Model(R, L, hext=disk.hext).field(g), model.mask) > 1e-3


def test_set_damping_per_replica_matches_oracle(O):
    disk = Disk(20e-9, 5e-9, alpha=0.02)
    h = Nanodisk([disk], [3], nd.ND_FP64)
    model = O.Model(disk.R, disk.L)
    g = model.init_vortex(2e-9, 1e-9)
    alphas = [0.0, 0.05, 0.3]
    h.set_damping(alphas)
    m = h.to_device([g, g, g])
    # (tolerance: relative to the change over the run, 20x the FP64 field
    # tolerance, as for the other short trajectories)
    dt = 2e-14
    h.rk4(m, 6, dt)
    out = h.unpack(m)
    for r, a in enumerate(alphas):
        model.set_alpha(a)
        ref = model.rk4(g, 6, model.dtau(dt))
        assert rel(out[r] - g, ref - g, model.mask) < 2e-10, a
    # Heun at T > 0 uses the per-replica alpha in the noise amplitude too
    m = h.to_device([g, g, g])
    h.heun(m, 4, dt, [300.0] * 3, [5, 6, 7], step0=2)
    out = h.unpack(m)
    Ts = O.scaled_temperature(300.0, disk.A, disk.L)
    for r, a in enumerate(alphas):
        model.set_alpha(a)
        ref = model.heun(g, 4, model.dtau(dt), Ts, 5 + r, 2)
        assert rel(out[r] - g, ref - g, model.mask) < 2e-10, a
