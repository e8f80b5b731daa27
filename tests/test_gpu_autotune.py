"""The stepping plans (fused-kernel thread-count variants, global path) give
bit-identical trajectories (to rounding where the global path transforms the
rows differently), and the autotuner picks one of the valid plans per size
class."""
import numpy as np
import pytest
import torch

import paper_1207_2192_gb300 as nd
from paper_1207_2192_gb300 import Disk, Nanodisk

pytestmark = pytest.mark.gpu

DISKS = [Disk(6e-9, 3e-9, alpha=0.02), Disk(13e-9, 3e-9, alpha=0.02), Disk(24e-9, 5e-9, alpha=0.02),
         Disk(50e-9, 10e-9, alpha=0.02)]                    # P = 16, 32, 64, 128
REPS = [3, 2, 2, 2]


def classes(h):
    out, i = [], 0
    while True:
        info = nd.nd_plan_info(h.h, i)
        if info is None:
            return out
        out.append(info)
        i += 1


@pytest.mark.parametrize("method", [nd.ND_METHOD_HEUN, nd.ND_METHOD_RK4])
def test_every_plan_gives_the_same_trajectory(method):
    ref_h = Nanodisk(DISKS, REPS, nd.ND_FP32)
    B = ref_h.B
    X0 = np.zeros((B, 2))
    T, seeds, dt = np.full(B, 300.0), np.arange(B, dtype=np.uint64), 1e-14

    def run(h):
        m = h.empty_device()
        h.init_vortex(m, X0)
        if method == nd.ND_METHOD_HEUN:
            h.heun(m, 3, dt, T, seeds)
        else:
            h.rk4(m, 3, dt)
        torch.cuda.synchronize()
        return m

    ref = run(ref_h)
    cls = classes(ref_h)
    assert [c["P"] for c in cls] == [16, 32, 64, 128]
    tried = 0
    for ci in range(len(cls)):
        for plan in (0, 1, 2, 100):
            h = Nanodisk(DISKS, REPS, nd.ND_FP32)
            if nd.nd_set_plan(h.h, ci, method, plan, check=False) != nd.ND_OK:
                continue
            tried += 1
            out = run(h)
            if plan == 100 and cls[ci]["P"] == 128:
                # on chip the P = 128 rows are half-length real transforms, on the
                # global path complex row pairs: equal to rounding, not bit for bit
                assert (out - ref).abs().max().item() <= 1e-6, (ci, plan)
            else:
                assert torch.equal(out, ref), (ci, plan)
    assert tried >= 10


def test_autotune_picks_valid_plans():
    h = Nanodisk(DISKS, REPS, nd.ND_FP32)
    nd.nd_autotune(h.h, nd.ND_METHOD_HEUN, 1e-14, 5)
    for c in classes(h):
        assert c["plan_heun"] in (0, 1, 2, 100, 200, 201)
        assert c["plan_rk4"] == -1
        assert (c["threads_heun"] > 0) == (c["plan_heun"] != 100)
    m = h.empty_device()
    h.init_vortex(m, np.zeros((h.B, 2)))
    h.heun(m, 2, 1e-14, np.full(h.B, 300.0), np.arange(h.B, dtype=np.uint64))
    assert nd.nd_check_status(h.h) == nd.ND_OK


def test_group_autotune_keeps_valid_plans_for_handles_that_share_the_gpu():
    """nd_autotune_group times the classes of several handles stepping side by
    side; every class ends on a valid plan and the handles still step."""
    ha = Nanodisk([Disk(13e-9, 3e-9), Disk(50e-9, 10e-9)], [1, 2], nd.ND_FP32)
    hb = Nanodisk([Disk(24e-9, 5e-9, alpha=0.02), Disk(70e-9, 10e-9, alpha=0.02)], [3, 2], nd.ND_FP32)
    nd.nd_autotune_group([ha.h, hb.h], [nd.ND_METHOD_RK4, nd.ND_METHOD_HEUN], 1e-14, 4)
    for h, key in ((ha, "plan_rk4"), (hb, "plan_heun")):
        for c in classes(h):
            assert c[key] in (0, 1, 2, 100, 200, 201)
    ma, mb = ha.empty_device(), hb.empty_device()
    ha.init_vortex(ma, np.zeros((ha.B, 2)))
    hb.init_vortex(mb, np.zeros((hb.B, 2)))
    ha.rk4(ma, 2, 1e-14)
    hb.heun(mb, 2, 1e-14, np.full(hb.B, 300.0), np.arange(hb.B, dtype=np.uint64))
    torch.cuda.synchronize()
    assert nd.nd_check_status(ha.h) == nd.ND_OK and nd.nd_check_status(hb.h) == nd.ND_OK
    with pytest.raises(nd.NDError):
        nd.nd_autotune_group([ha.h, ha.h], [nd.ND_METHOD_RK4, nd.ND_METHOD_RK4], 1e-14, 2)
    with pytest.raises(nd.NDError):
        nd.nd_autotune_group([], [], 1e-14, 2)
