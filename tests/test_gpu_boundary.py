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


def test_boundary_rejects_bad_arguments_and_keeps_state():
    """The error behaviour the header states: bad arguments return
    ND_ERR_ARG with a message and leave the state untouched; zero steps are a
    no-op; the handle stays usable afterwards."""
    import torch
    with pytest.raises(nd.NDError) as e:
        nd.nd_create_disk([Disk(-1e-9, 5e-9).desc()])
    assert e.value.code == nd.ND_ERR_ARG
    with pytest.raises(nd.NDError):
        nd.nd_create_disk([])
    with pytest.raises(nd.NDError):
        nd.nd_create_disk([Disk(20e-9, 5e-9).desc()], precision=7)
    disk = Disk(20e-9, 5e-9, alpha=0.02)
    h = Nanodisk([disk], [2], nd.ND_FP32)
    m = h.empty_device()
    h.init_vortex(m, np.zeros((2, 2)))
    before = m.clone()
    T, s = np.full(2, 300.0), np.arange(2, dtype=np.uint64)
    for bad in (lambda: nd.nd_step_rk4(h.h, m, -1, 1e-14),
                lambda: nd.nd_step_rk4(h.h, m, 1, 0.0),
                lambda: nd.nd_step_heun(h.h, m, 1, -1e-14, T, s),
                lambda: nd.nd_step_heun(h.h, m, 1, 1e-14, np.array([300.0, -1.0]), s),
                lambda: nd.nd_step_heun(h.h, m, -2, 1e-14, T, s)):
        with pytest.raises(nd.NDError) as e:
            bad()
        assert e.value.code == nd.ND_ERR_ARG and nd.nd_last_error()
    nd.nd_step_rk4(h.h, m, 0, 1e-14)
    nd.nd_step_heun(h.h, m, 0, 1e-14, T, s)
    torch.cuda.synchronize()
    assert torch.equal(m, before)
    assert nd.nd_check_status(h.h) == nd.ND_OK
    h.heun(m, 2, 1e-14, T, s)
    torch.cuda.synchronize()
    assert not torch.equal(m, before)
