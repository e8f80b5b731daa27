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


def _uneven_groups():
    import ndsynth
    R, L, T = ndsynth.uneven_disks(64, seed=1)
    return R, L, T, {"rk4": list(range(8)), "heun": list(range(8, 64))}


def test_size_classes_side_by_side_match_one_class_per_handle():
    """The classes of a multi-class handle step on forked streams; every
    replica ends bit for bit where a handle holding only its class puts it."""
    R, L, T, groups = _uneven_groups()
    idx = groups["heun"]
    disks = [Disk(R[i], L[i], alpha=0.01) for i in idx]
    h = Nanodisk(disks, None, nd.ND_FP32)
    Ps = [h.layout[r]["P"] for r in range(h.B)]
    assert len(set(Ps)) >= 3
    X0 = np.stack([0.1 * R[idx], np.zeros(len(idx))], 1)
    m = h.empty_device()
    h.init_vortex(m, X0)
    h.heun(m, 3, 1e-14, T[idx], np.arange(len(idx), dtype=np.uint64), step0=2)
    out = h.unpack(m)
    for P in sorted(set(Ps)):
        sel = [r for r in range(h.B) if Ps[r] == P]
        hc = Nanodisk([disks[r] for r in sel], None, nd.ND_FP32)
        mc = hc.empty_device()
        hc.init_vortex(mc, X0[sel])
        hc.heun(mc, 3, 1e-14, T[idx][sel], np.array(sel, dtype=np.uint64), step0=2)
        for k, o in enumerate(hc.unpack(mc)):
            assert np.array_equal(o, out[sel[k]]), (P, sel[k])


def test_joined_graph_replays_both_handles_as_their_own_graphs_do():
    """The uneven batch as one graph launch: the RK4 graph of the T = 0 disks
    and the Heun graph of the others joined side by side replay exactly as
    the two graphs launched one after the other."""
    R, L, T, groups = _uneven_groups()
    runs = {}
    for joined in (False, True):
        hs, ms, gs = {}, {}, {}
        for name, idx in groups.items():
            h = Nanodisk([Disk(R[i], L[i], alpha=0.01) for i in idx], None, nd.ND_FP32)
            m = h.empty_device()
            h.init_vortex(m, np.stack([0.1 * R[idx], np.zeros(len(idx))], 1))
            method = nd.ND_METHOD_RK4 if name == "rk4" else nd.ND_METHOD_HEUN
            Tk = T[idx] if name == "heun" else None
            sd = np.arange(len(idx), dtype=np.uint64) + 3 if name == "heun" else None
            gs[name] = nd.nd_graph_create(h.h, m, method, 4, 1e-14, Tk, sd, step0=0)
            hs[name], ms[name] = h, m
        if joined:
            g = nd.nd_graph_join([gs["rk4"], gs["heun"]])
            assert nd.nd_graph_nodes(g) == nd.nd_graph_nodes(gs["rk4"]) + nd.nd_graph_nodes(gs["heun"])
            for _ in range(3):
                nd.nd_graph_launch(g)
            nd.nd_graph_destroy(g)
        else:
            for _ in range(3):
                nd.nd_graph_launch(gs["rk4"])
                nd.nd_graph_launch(gs["heun"])
        torch.cuda.synchronize()
        runs[joined] = {name: hs[name].unpack(ms[name]) for name in groups}
        for name in groups:
            assert nd.nd_check_status(hs[name].h) == nd.ND_OK
            nd.nd_graph_destroy(gs[name])
    for name in groups:
        for r, (a, b) in enumerate(zip(runs[False][name], runs[True][name])):
            assert np.array_equal(a, b), (name, r)
    with pytest.raises(nd.NDError):
        nd.nd_graph_join([])
