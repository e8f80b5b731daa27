"""The time-sliced stepping schedule (more replicas than resident CTAs, so
replicas change CTA between steps) gives bit-identical trajectories to the
one-CTA-per-replica launch, for Heun and RK4."""
import numpy as np
import pytest
import torch

import paper_1207_2192_gb300 as nd
from paper_1207_2192_gb300 import Disk, Nanodisk

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", ["heun", "rk4"])
def test_time_sliced_schedule_is_bit_identical(mode):
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    disk = Disk(50e-9, 10e-9, alpha=0.01)
    B = n_sm + 104 if n_sm >= 104 else 2 * n_sm       # above one CTA per SM for the P = 128 on-chip kernel
    half = B // 2
    X0 = np.stack([np.linspace(-6e-9, 6e-9, B), np.zeros(B)], 1)
    big = Nanodisk([disk], [B], nd.ND_FP32)
    m = big.empty_device()
    big.init_vortex(m, X0)
    parts = [Nanodisk([disk], [half], nd.ND_FP32), Nanodisk([disk], [B - half], nd.ND_FP32)]
    T = np.full(B, 300.0)
    seeds = np.arange(B, dtype=np.uint64) * 7 + 1
    steps, dt = 7, 1e-14
    ms = [p.empty_device() for p in parts]
    parts[0].init_vortex(ms[0], X0[:half])
    parts[1].init_vortex(ms[1], X0[half:])
    if mode == "heun":
        big.heun(m, steps, dt, T, seeds, step0=3)
        parts[0].heun(ms[0], steps, dt, T[:half], seeds[:half], step0=3)
        parts[1].heun(ms[1], steps, dt, T[half:], seeds[half:], step0=3)
    else:
        big.rk4(m, steps, dt)
        parts[0].rk4(ms[0], steps, dt)
        parts[1].rk4(ms[1], steps, dt)
    assert nd.nd_check_status(big.h) == nd.ND_OK
    n0 = ms[0].numel()
    assert torch.equal(m[:n0], ms[0]) and torch.equal(m[n0:], ms[1])
    assert not torch.equal(m[:n0], parts[0].to_device(parts[0].unpack(ms[0])) * 0)


def test_expired_handover_wait_reports_timeout_and_leaves_context_usable():
    """A segment whose hand-over flag is never set gives up after its bounded
    wait: the status word reports ND_ERR_TIMEOUT, no state is touched, and the
    same handle steps normally afterwards."""
    import time
    h = Nanodisk([Disk(50e-9, 10e-9, alpha=0.01)], [3], nd.ND_FP32)
    m = h.empty_device()
    h.init_vortex(m, np.zeros((3, 2)))
    before = m.clone()
    assert nd.nd_check_status(h.h) == nd.ND_OK
    t0 = time.perf_counter()
    nd.nd_selftest_handover_timeout(h.h)
    waited = time.perf_counter() - t0
    assert nd.nd_check_status(h.h) == nd.ND_ERR_TIMEOUT
    assert nd.nd_check_status(h.h) == nd.ND_OK          # reading the word clears it
    assert 0.05 < waited < 30.0
    assert torch.equal(m, before)
    h.heun(m, 3, 1e-14, np.full(3, 300.0), np.arange(3, dtype=np.uint64))
    torch.cuda.synchronize()
    assert nd.nd_check_status(h.h) == nd.ND_OK
    assert not torch.equal(m, before) and torch.isfinite(m).all()


def test_non_finite_state_sets_the_nan_status():
    """A NaN in a disk cell propagates through a step and the status word
    reports ND_ERR_NAN; a NaN outside the disk is ignored."""
    disk = Disk(30e-9, 10e-9, alpha=0.01)
    h = Nanodisk([disk], [2], nd.ND_FP32)
    mask = h.mask(0).astype(bool)
    D = h.layout[0]["D"]
    g = [np.zeros((3, D, D)) for _ in range(2)]
    for k in range(2):
        g[k][2][mask] = 1.0
    outside = np.argwhere(~mask)[0]
    g[0][0, outside[0], outside[1]] = np.nan            # ignored: not a disk cell
    m = h.to_device(g)
    h.rk4(m, 1, 1e-14)
    assert nd.nd_check_status(h.h) == nd.ND_OK
    inside = np.argwhere(mask)[len(np.argwhere(mask)) // 2]
    g[1][1, inside[0], inside[1]] = np.nan
    m = h.to_device(g)
    h.rk4(m, 1, 1e-14)
    assert nd.nd_check_status(h.h) == nd.ND_ERR_NAN
    assert nd.nd_check_status(h.h) == nd.ND_OK
