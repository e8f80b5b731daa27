"""Single-disk stepping on a thread-block cluster (plan 200: 8 CTAs, plan 201:
16 CTAs for P >= 32): each replica is spread over the cluster's CTAs, whose
shared memories hold its rows and exchange columns through distributed shared
memory.  The per-element arithmetic is that of the
one-CTA kernel, so trajectories match it, and they match the oracle's RK4 and
stochastic Heun steps (Sec. II.C) to the field tolerance."""
import numpy as np
import pytest
import torch

import paper_1207_2192_gb300 as nd
from paper_1207_2192_gb300 import Disk, Nanodisk

pytestmark = pytest.mark.gpu

PLAN_CLUSTER = 200
PLANS = [200, 201]
DISKS = [Disk(6e-9, 3e-9, alpha=0.02), Disk(13e-9, 3e-9, alpha=0.02), Disk(24e-9, 5e-9, alpha=0.02),
         Disk(50e-9, 10e-9, alpha=0.02)]                    # P = 16, 32, 64, 128


def cluster_handle(disks, reps, method, prec=nd.ND_FP32, plan=PLAN_CLUSTER):
    """A handle whose classes step on the cluster plan (the 16-CTA plan where
    the class's P has one, else the 8-CTA plan)."""
    h = Nanodisk(disks, reps, prec)
    ci = 0
    while nd.nd_plan_info(h.h, ci) is not None:
        if nd.nd_set_plan(h.h, ci, method, plan, check=False) != nd.ND_OK:
            nd.nd_set_plan(h.h, ci, method, PLAN_CLUSTER)
        ci += 1
    return h


def run(h, method, n, X0=None):
    m = h.empty_device()
    h.init_vortex(m, np.zeros((h.B, 2)) if X0 is None else X0)
    if method == nd.ND_METHOD_HEUN:
        h.heun(m, n, 1e-14, np.full(h.B, 300.0), np.arange(h.B, dtype=np.uint64) + 11)
    else:
        h.rk4(m, n, 1e-14)
    torch.cuda.synchronize()
    return m


@pytest.mark.parametrize("plan", PLANS)
@pytest.mark.parametrize("method", [nd.ND_METHOD_HEUN, nd.ND_METHOD_RK4])
def test_cluster_plan_matches_one_cta_kernel(method, plan):
    reps = [3, 1, 2, 1]
    X0 = np.array([[1e-9 * (i % 3), -0.5e-9 * (i % 2)] for i in range(sum(reps))])
    ref = run(Nanodisk(DISKS, reps, nd.ND_FP32), method, 4, X0)
    h = cluster_handle(DISKS, reps, method, plan=plan)
    info = [nd.nd_plan_info(h.h, ci) for ci in range(4)]
    key = "plan_heun" if method == nd.ND_METHOD_HEUN else "plan_rk4"
    want = [PLAN_CLUSTER] + [plan] * 3                      # P = 16 has only the 8-CTA plan
    assert [i[key] for i in info] == want
    nct = {200: 8, 201: 16}
    assert [i["threads_heun" if method == nd.ND_METHOD_HEUN else "threads_rk4"] for i in info] == \
        [256 * nct[p] for p in want]
    out = run(h, method, 4, X0)
    diff = (out - ref).abs().max().item()
    assert diff <= 1e-6, diff
    assert nd.nd_check_status(h.h) == nd.ND_OK


TOL = {nd.ND_FP32: 1e-5, nd.ND_FP64: 1e-11}      # relative field error of each precision


def traj_ok(out, ref, start, model, prec):
    """Trajectory error against 20x the field tolerance times the change over
    the run, plus the rounding of the stored state."""
    change = np.linalg.norm((ref - start) * model.mask)
    floor = (1e-7 if prec == nd.ND_FP32 else 1e-15) * np.sqrt(3 * model.C)
    return np.linalg.norm((out - ref) * model.mask) <= 20 * TOL[prec] * change + floor


@pytest.mark.parametrize("plan", PLANS)
@pytest.mark.parametrize("prec", [nd.ND_FP32, nd.ND_FP64])
@pytest.mark.parametrize("R,L", [(13e-9, 3e-9), (24e-9, 5e-9), (50e-9, 10e-9)])
def test_cluster_plan_matches_oracle(O, R, L, prec, plan):
    disk = Disk(R, L, alpha=0.02, hext=(2e3, -1e3, 5e2))
    model = O.Model(R, L, alpha=disk.alpha, hext=disk.hext)
    g = model.init_vortex(2e-9 if R > 20e-9 else 0.5e-9, -1e-9 if R > 20e-9 else 0.0)
    dt = 1e-14
    h = cluster_handle([disk], [1], nd.ND_METHOD_RK4, prec, plan)
    assert nd.nd_plan_info(h.h, 0)["plan_rk4"] == plan
    start = h.unpack(h.to_device([g]))[0]
    m = h.to_device([g])
    h.rk4(m, 3, dt)
    ref = model.rk4(start, 3, model.dtau(dt))
    assert traj_ok(h.unpack(m)[0], ref, start, model, prec)
    h = cluster_handle([disk], [2], nd.ND_METHOD_HEUN, prec, plan)
    m = h.to_device([g, g])
    h.heun(m, 3, dt, [300.0, 300.0], [21, 22], step0=5)
    Ts = O.scaled_temperature(300.0, disk.A, disk.L)
    for r, out in enumerate(h.unpack(m)):
        ref = model.heun(start, 3, model.dtau(dt), Ts, 21 + r, 5)
        assert traj_ok(out, ref, start, model, prec)


@pytest.mark.parametrize("plan", PLANS)
def test_cluster_plan_with_mask_and_field_schedule(O, plan):
    """An elliptical mask and a per-step field schedule on the cluster plan,
    against the oracle with the same mask and schedule."""
    disk = Disk(40e-9, 8e-9, alpha=0.05)
    model = O.Model(disk.R, disk.L, alpha=disk.alpha)
    D = model.D
    yy, xx = np.mgrid[0:D, 0:D]
    c = 0.5 * (D - 1)
    mask = (((xx - c) / (0.5 * D)) ** 2 + ((yy - c) / (0.35 * D)) ** 2 <= 1.0).astype(np.uint8)
    sched = np.array([[1e4 * np.sin(0.3 * k), 5e3, -2e3] for k in range(6)])
    h = cluster_handle([disk], [1], nd.ND_METHOD_RK4, plan=plan)
    h.set_mask(0, mask)
    h.set_field_schedule(0, sched)
    model.set_mask(mask)
    model.set_schedule(sched)
    g = model.init_vortex(1e-9, 1e-9)
    start = h.unpack(h.to_device([g]))[0]
    m = h.to_device([g])
    h.rk4(m, 4, 1e-14)
    ref = model.rk4(start, 4, model.dtau(1e-14))
    assert traj_ok(h.unpack(m)[0], ref, start, model, nd.ND_FP32)


def test_cluster_plan_is_offered_by_autotune():
    h = Nanodisk([Disk(50e-9, 10e-9, alpha=0.02)], [1], nd.ND_FP32)
    assert nd.nd_set_plan(h.h, 0, nd.ND_METHOD_HEUN, PLAN_CLUSTER, check=False) == nd.ND_OK
    big = Nanodisk([Disk(200e-9, 10e-9)], [1], nd.ND_FP32)            # P = 512: no cluster plan
    for plan in PLANS:
        assert nd.nd_set_plan(big.h, 0, nd.ND_METHOD_HEUN, plan, check=False) == nd.ND_ERR_ARG
    tiny = Nanodisk([Disk(6e-9, 3e-9)], [1], nd.ND_FP32)               # P = 16: 8 CTAs only
    assert nd.nd_set_plan(tiny.h, 0, nd.ND_METHOD_HEUN, 201, check=False) == nd.ND_ERR_ARG
    nd.nd_autotune(h.h, nd.ND_METHOD_HEUN, 1e-14, 5)
    assert nd.nd_plan_info(h.h, 0)["plan_heun"] in (0, 1, 2, 100, 200, 201)


@pytest.mark.parametrize("R,grid3x,P", [(70e-9, False, 256), (80e-9, True, 192)])
@pytest.mark.parametrize("method", [nd.ND_METHOD_HEUN, nd.ND_METHOD_RK4])
def test_large_grid_cluster_plan_matches_global_path_and_oracle(O, method, R, grid3x, P):
    """P = 256 (D = 70) and P = 192 (D = 80, the radix-3 grid): the spectrum
    of one replica is too large for one CTA's shared memory but fits in a
    16-CTA cluster's; against the global path (plan 100) and the oracle."""
    disk = Disk(R, 10e-9, alpha=0.02, hext=(1e3, 0.0, -2e3))
    h = Nanodisk([disk], [2], nd.ND_FP32, grid3x=grid3x)
    assert h.layout[0]["P"] == P
    assert nd.nd_set_plan(h.h, 0, method, 200, check=False) == nd.ND_ERR_ARG      # 8 CTAs: no such plan
    nd.nd_set_plan(h.h, 0, method, 201)
    nt = 512 if P >= 256 else 256
    assert nd.nd_plan_info(h.h, 0)["threads_heun" if method == nd.ND_METHOD_HEUN else "threads_rk4"] == 16 * nt
    hg = Nanodisk([disk], [2], nd.ND_FP32, grid3x=grid3x)
    nd.nd_set_plan(hg.h, 0, method, 100)
    X0 = np.array([[3e-9, 1e-9], [-2e-9, 0.0]])
    out, ref = run(h, method, 3, X0), run(hg, method, 3, X0)
    assert (out - ref).abs().max().item() <= 1e-6
    model = O.Model(disk.R, disk.L, alpha=disk.alpha, hext=disk.hext)
    start = h.unpack(h.to_device([model.init_vortex(3e-9, 1e-9)]))[0]
    m = h.to_device([start, start])
    if method == nd.ND_METHOD_RK4:
        h.rk4(m, 2, 1e-14)
        refs = [model.rk4(start, 2, model.dtau(1e-14))] * 2
    else:
        h.heun(m, 2, 1e-14, [300.0, 300.0], [5, 6], step0=3)
        Ts = O.scaled_temperature(300.0, disk.A, disk.L)
        refs = [model.heun(start, 2, model.dtau(1e-14), Ts, s, 3) for s in (5, 6)]
    for o, r in zip(h.unpack(m), refs):
        assert traj_ok(o, r, start, model, nd.ND_FP32)
