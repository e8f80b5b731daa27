"""Parity at the full sizes of the benchmark configurations, in the launch
configuration the benchmark times.

* Large disk (R = 500 nm, P = 1024, global path) and R = 200 nm (P = 512):
  the field on sampled cells against the oracle's direct sum at those cells;
  full-state Heun trajectories (every cell: two steps at P = 512, one at
  P = 1024) against the oracle's; FP64 fields at P = 512 (every cell) and
  P = 1024 (sampled cells).
* Batched Heun, 256 replicas of R = 50 nm (time-sliced schedule over the
  SMs): sampled replicas against the oracle's Heun trajectory.
"""
import numpy as np
import torch
import pytest

import ndsynth
import paper_1207_2192_gb300 as nd
from paper_1207_2192_gb300 import Disk, Nanodisk

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("R,L", [(200e-9, 20e-9), (500e-9, 20e-9)])
def test_large_disk_field_on_sampled_cells(O, R, L):
    disk = Disk(R, L, hext=(0.0, 2e4, 0.0))
    h = Nanodisk([disk], [2], nd.ND_FP32)
    model = O.Model(R, L, hext=disk.hext)
    grids = [ndsynth.random_unit_vectors(model.D, seed=21) * model.mask, model.init_vortex(12e-9, -4e-9)]
    b = h.unpack(h.field(h.to_device(grids)))
    inside = np.flatnonzero(model.mask.ravel())
    cells = inside[ndsynth.sample_indices(len(inside), 24, seed=2)]
    # include the rim, where the field is largest and least smooth
    cells = np.concatenate([cells, inside[:4], inside[-4:]])
    for r in range(2):
        ref = model.field_at(grids[r], cells)
        got = np.stack([b[r][:, c // model.D, c % model.D] for c in cells])
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 1e-5 * scale


def test_batched_heun_full_size_on_sampled_replicas(O):
    disk = Disk(50e-9, 10e-9, alpha=0.01)
    B = 256
    h = Nanodisk([disk], [B], nd.ND_FP32)
    model = O.Model(disk.R, disk.L, alpha=disk.alpha)
    X0 = np.stack([np.linspace(-5e-9, 5e-9, B), np.zeros(B)], 1)
    m = h.empty_device()
    h.init_vortex(m, X0)
    start = h.unpack(m)
    T, seeds, dt, steps = np.full(B, 300.0), np.arange(B, dtype=np.uint64), 1e-14, 3
    h.heun(m, steps, dt, T, seeds, step0=0)
    assert nd.nd_check_status(h.h) == nd.ND_OK
    out = h.unpack(m)
    Ts = O.scaled_temperature(300.0, disk.A, disk.L)
    for r in (0, 97, 151, 152, 255):
        ref = model.heun(start[r], steps, model.dtau(dt), Ts, int(seeds[r]), 0)
        assert np.max(np.abs(out[r] - ref)) < 1e-4
        assert np.linalg.norm((out[r] - ref) * model.mask) <= 2e-4 * np.linalg.norm((ref - start[r]) * model.mask) + 1e-6


def test_large_disk_heun_properties():
    """P = 1024 Heun: unit norm kept, resumable bit for bit, noise matters."""
    disk = Disk(500e-9, 20e-9, alpha=0.01)
    h = Nanodisk([disk], [2], nd.ND_FP32)
    m = h.empty_device()
    h.init_vortex(m, np.zeros((2, 2)))
    a, b = m.clone(), m.clone()
    h.heun(a, 4, 1e-14, [300.0, 300.0], [1, 2], step0=0)
    h.heun(b, 1, 1e-14, [300.0, 300.0], [1, 2], step0=0)
    h.heun(b, 3, 1e-14, [300.0, 300.0], [1, 2], step0=1)
    assert bool((a == b).all())
    g = h.unpack(a)
    mask = h.mask(0).astype(bool)
    for r in range(2):
        n = np.sqrt((g[r] ** 2).sum(0))[mask]
        assert np.max(np.abs(n - 1)) < 1e-5
    assert not np.allclose(g[0], g[1])


def test_uneven_batch_full_size_with_graphs_and_autotuned_plans(O):
    """The uneven batch: 64 disks with R ~ U(20, 100) nm, L/R ~ U(0.05, 0.2)
    and T ~ U(0, 400) K, disks 0-7 at T = 0 stepping with RK4 and the rest
    with Heun, size classes P = 64, 128 and 256 (on-chip, cluster and global
    paths), in the launch configuration the bench times: both handles tuned
    together (nd_autotune_group), each handle's steps captured in a CUDA
    graph and the two graphs joined into one launch.  Sampled disks of every
    size class match their oracle trajectory."""
    R, L, T = ndsynth.uneven_disks(64, seed=0)
    alpha, dt, steps = 0.01, 1e-14, 2
    groups = {"rk4": list(range(8)), "heun": list(range(8, 64))}
    hs, ms, starts, gs = {}, {}, {}, {}
    for name, idx in groups.items():
        hs[name] = Nanodisk([Disk(R[i], L[i], alpha=alpha) for i in idx], None, nd.ND_FP32)
    nd.nd_autotune_group([hs["rk4"].h, hs["heun"].h], [nd.ND_METHOD_RK4, nd.ND_METHOD_HEUN], dt, 4)
    for name, idx in groups.items():
        h = hs[name]
        method = nd.ND_METHOD_RK4 if name == "rk4" else nd.ND_METHOD_HEUN
        m = h.empty_device()
        h.init_vortex(m, np.stack([0.1 * R[idx], np.zeros(len(idx))], 1))
        starts[name] = h.unpack(m)
        Tk = T[idx] if name == "heun" else None
        seeds = np.arange(len(idx), dtype=np.uint64) + 100 if name == "heun" else None
        gs[name] = nd.nd_graph_create(h.h, m, method, steps, dt, Tk, seeds, step0=0)
        ms[name] = m
    joined = nd.nd_graph_join([gs["rk4"], gs["heun"]])
    nd.nd_graph_launch(joined)
    torch.cuda.synchronize()
    nd.nd_graph_destroy(joined)
    for g in gs.values():
        nd.nd_graph_destroy(g)
    Ps = {name: sorted({hs[name].layout[r]["P"] for r in range(hs[name].B)}) for name in groups}
    assert Ps["heun"][0] <= 64 and Ps["heun"][-1] == 256
    for name, idx in groups.items():
        h = hs[name]
        assert nd.nd_check_status(h.h) == nd.ND_OK
        out = h.unpack(ms[name])
        Pk = [h.layout[r]["P"] for r in range(h.B)]
        # one replica of every size class, plus the largest disk
        pick = sorted({Pk.index(p) for p in set(Pk)} | {int(np.argmax(R[idx]))})
        for r in pick:
            i = idx[r]
            model = O.Model(R[i], L[i], alpha=alpha)
            if name == "rk4":
                ref = model.rk4(starts[name][r], steps, model.dtau(dt))
            else:
                Ts = O.scaled_temperature(T[i], model.A, model.L)
                ref = model.heun(starts[name][r], steps, model.dtau(dt), Ts, 100 + r, 0)
            assert np.max(np.abs(out[r] - ref)) < 1e-4, (name, r, Pk[r])
            # relative to the change over the run, plus the FP32 rounding of the
            # stored state itself (~1e-7 per component, rms over 3C components)
            change = np.linalg.norm((ref - starts[name][r]) * model.mask)
            floor = 1e-7 * np.sqrt(3 * model.C)
            assert np.linalg.norm((out[r] - ref) * model.mask) <= 2e-4 * change + floor, (name, r, Pk[r])


def _heun_full_state(O, R, L, steps, B):
    """Full-state Heun parity on the global path: every cell of every replica
    after `steps` steps against the oracle's trajectory from the same state and
    Philox stream.  Tolerance: the FP32 field error (1e-5 relative) times the
    change over the run, plus the FP32 rounding of the stored state."""
    disk = Disk(R, L, alpha=0.01, hext=(0.0, 0.0, 1e4))
    h = Nanodisk([disk], [B], nd.ND_FP32)
    model = O.Model(R, L, alpha=disk.alpha, hext=disk.hext)
    X0 = np.stack([np.linspace(-6e-9, 6e-9, B), np.linspace(3e-9, -2e-9, B)], 1)
    m = h.empty_device()
    h.init_vortex(m, X0)
    start = h.unpack(m)
    T, seeds, dt = np.full(B, 300.0), np.arange(B, dtype=np.uint64) + 40, 1e-14
    h.heun(m, steps, dt, T, seeds, step0=5)
    assert nd.nd_check_status(h.h) == nd.ND_OK
    out = h.unpack(m)
    Ts = O.scaled_temperature(300.0, disk.A, disk.L)
    for r in range(B):
        ref = model.heun(start[r], steps, model.dtau(dt), Ts, int(seeds[r]), 5)
        change = np.linalg.norm((ref - start[r]) * model.mask)
        err = np.linalg.norm((out[r] - ref) * model.mask)
        print(f"R={R*1e9:.0f} nm replica {r}: |error| / |change| = {err / change:.2e}, max abs {np.max(np.abs(out[r] - ref)):.2e}")
        assert np.max(np.abs(out[r] - ref)) < 2e-5
        assert err <= 5e-5 * change + 1e-7 * np.sqrt(3 * model.C)


def test_p512_heun_full_state_matches_oracle(O):
    _heun_full_state(O, 200e-9, 20e-9, steps=2, B=2)


def test_p1024_heun_full_state_matches_oracle(O):
    """One step of the large-disk workload's disk (R = 500 nm, 196,364 cells):
    about 8e10 direct-sum pair terms on the host."""
    _heun_full_state(O, 500e-9, 20e-9, steps=1, B=1)


@pytest.mark.parametrize("R,L,sampled", [(150e-9, 20e-9, False), (500e-9, 20e-9, True)])
def test_fp64_global_path_field_large_grids(O, R, L, sampled):
    """FP64 on the global path at P = 512 (every cell) and P = 1024 (sampled
    cells): relative error 1e-11."""
    disk = Disk(R, L, hext=(1e4, 0.0, -2e4))
    h = Nanodisk([disk], [1], nd.ND_FP64)
    assert h.layout[0]["P"] == (512 if R < 256e-9 else 1024)
    model = O.Model(R, L, hext=disk.hext)
    g = ndsynth.random_unit_vectors(model.D, seed=77) * model.mask
    b = h.unpack(h.field(h.to_device([g])))[0]
    if not sampled:
        ref = model.field(g)
        err = np.linalg.norm((b - ref) * model.mask) / np.linalg.norm(ref * model.mask)
        assert err < 1e-11
    else:
        inside = np.flatnonzero(model.mask.ravel())
        cells = np.concatenate([inside[ndsynth.sample_indices(len(inside), 24, seed=9)], inside[:4], inside[-4:]])
        ref = model.field_at(g, cells)
        got = np.stack([b[:, c // model.D, c % model.D] for c in cells])
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-11
