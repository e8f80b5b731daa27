"""Graph-captured stepping: replays are bit-identical to direct calls with
the noise-step counter advanced, for Heun and RK4, for a batch above one
replica per SM (time-sliced schedule) and for an uneven multi-disk handle."""
import numpy as np
import pytest
import torch

import paper_1207_2192_gb300 as nd
from paper_1207_2192_gb300 import Disk, Nanodisk

pytestmark = pytest.mark.gpu


def _handles(kind):
    if kind == "batched":
        n_sm = torch.cuda.get_device_properties(0).multi_processor_count
        disks, reps = [Disk(50e-9, 10e-9, alpha=0.01)], [n_sm + 20]
    else:
        disks = [Disk(9e-9, 2e-9, alpha=0.02), Disk(21e-9, 3e-9, alpha=0.02), Disk(70e-9, 12e-9, alpha=0.02)]
        reps = [3, 2, 2]
    return Nanodisk(disks, reps, nd.ND_FP32), Nanodisk(disks, reps, nd.ND_FP32)


@pytest.mark.parametrize("kind", ["batched", "uneven"])
@pytest.mark.parametrize("method", [nd.ND_METHOD_HEUN, nd.ND_METHOD_RK4])
def test_graph_replays_match_direct_calls(kind, method):
    a, b = _handles(kind)
    B = a.B
    ma, mb = a.empty_device(), b.empty_device()
    X0 = np.stack([np.linspace(-3e-9, 3e-9, B), np.zeros(B)], 1)
    a.init_vortex(ma, X0)
    b.init_vortex(mb, X0)
    T, seeds, dt, n = np.full(B, 300.0), np.arange(B, dtype=np.uint64) + 5, 1e-14, 4
    g = nd.nd_graph_create(a.h, ma, method, n, dt, T, seeds, step0=2)
    try:
        assert nd.nd_graph_nodes(g) >= 2
        for k in range(3):
            nd.nd_graph_launch(g)
            if method == nd.ND_METHOD_HEUN:
                b.heun(mb, n, dt, T, seeds, step0=2 + n * k)
            else:
                b.rk4(mb, n, dt)
            torch.cuda.synchronize()
            assert torch.equal(ma, mb), k
    finally:
        nd.nd_graph_destroy(g)
    assert nd.nd_check_status(a.h) == nd.ND_OK


def test_graph_with_statistics_sample():
    a, b = _handles("uneven")
    B = a.B
    ma, mb = a.empty_device(), b.empty_device()
    X0 = np.zeros((B, 2))
    a.init_vortex(ma, X0)
    b.init_vortex(mb, X0)
    for h in (a, b):
        nd.nd_stats_reset(h.h, 10e-9, 50, 500.0, 50)
    T, seeds, dt, n = np.full(B, 200.0), np.arange(B, dtype=np.uint64), 1e-14, 6
    g = nd.nd_graph_create(a.h, ma, nd.ND_METHOD_HEUN, n, dt, T, seeds, step0=0, stats_sample=True)
    try:
        for k in range(4):
            nd.nd_graph_launch(g)
            b.heun(mb, n, dt, T, seeds, step0=n * k)
            nd.nd_stats_sample(b.h, mb, n * dt)
    finally:
        nd.nd_graph_destroy(g)
    sa = nd.nd_stats_read(a.h, B, 50, 50)
    sb = nd.nd_stats_read(b.h, B, 50, 50)
    assert torch.equal(ma, mb)
    for x, y in zip(sa, sb):
        assert np.array_equal(x, y)
