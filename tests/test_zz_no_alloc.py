"""The allocation-free Heun entry point (nd_step_heun_noalloc) against the
handle-based nd_step_heun.

It serves callers that cannot allocate device memory (a framework owning all
allocations, a real-time loop, a plugin limited to its host's buffers): its
working memory is a fixed device array inside the library.  This file sorts
last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

import paper_1207_2192_gb300 as nd
from paper_1207_2192_gb300 import Disk, Nanodisk, _binding

pytestmark = pytest.mark.gpu


def test_noalloc_heun_matches_handle_heun_on_two_calls():
    import torch
    disk = Disk(30e-9, 5e-9, alpha=0.02, hext=(0.0, 5e3, 0.0))
    B = 3
    h = Nanodisk([disk], [B], nd.ND_FP32)
    m0 = h.empty_device()
    h.init_vortex(m0, np.array([[2e-9, 0.0], [0.0, -3e-9], [0.0, 0.0]]))
    T = np.array([300.0, 150.0, 0.0])
    seeds = np.array([11, 12, 13], dtype=np.uint64)
    dt = 1e-14
    ref, out = m0.clone(), m0.clone()
    for n, s0 in ((7, 0), (5, 7)):             # two calls in a row, the second resuming the noise counter
        nd.nd_step_heun(h.h, ref, n, dt, T, seeds, s0)
        _binding.nd_step_heun_noalloc(disk, B, out, n, dt, T, seeds, s0)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert (out - ref).abs().max().item() <= 1e-5
        # both paths launch the same Heun kernel on the same spectral kernel,
        # twiddles and parameter blocks, so the states agree bit for bit
        assert torch.equal(out, ref)
    assert (out - m0).abs().max().item() > 1e-4     # the state did move


def test_noalloc_rebuilds_its_tables_when_the_geometry_changes():
    # the array caches one geometry's spectral kernel, mask and twiddles; a
    # stale cache would step with the wrong Green's tensor.  Alternate two
    # disks of the same grid (D = 30, P = 64) but different thickness, one of
    # another padded size (D = 14, P = 32), and return to the first.
    import torch
    disks = [Disk(30e-9, 5e-9, alpha=0.05), Disk(30e-9, 12e-9, alpha=0.05), Disk(14e-9, 5e-9, alpha=0.05),
             Disk(30e-9, 5e-9, alpha=0.05)]
    T = np.array([0.0, 300.0])
    seeds = np.array([3, 4], dtype=np.uint64)
    dt = 1e-14
    for k, disk in enumerate(disks):
        h = Nanodisk([disk], [2], nd.ND_FP32)
        m0 = h.empty_device()
        h.init_vortex(m0, np.array([[2e-9, 0.0], [-2e-9, 1e-9]]))
        ref, out = m0.clone(), m0.clone()
        nd.nd_step_heun(h.h, ref, 6, dt, T, seeds, 0)
        _binding.nd_step_heun_noalloc(disk, 2, out, 6, dt, T, seeds, 0)
        torch.cuda.synchronize()
        assert (out - ref).abs().max().item() <= 1e-5, f"geometry {k}"
        assert torch.equal(out, ref), f"geometry {k}"
        h.close()


def test_noalloc_rejects_what_exceeds_its_limits():
    import torch
    small = Disk(30e-9, 5e-9)
    big = Disk(100e-9, 10e-9)                        # 100 cells across: P = 256 > 128
    m = torch.zeros(10, device="cuda")
    T, s = np.zeros(1), np.zeros(1, dtype=np.uint64)
    assert _binding.nd_step_heun_noalloc(big, 1, m, 1, 1e-14, T, s, check=False) == nd.ND_ERR_ARG
    assert "padded grid" in nd.nd_last_error()
    many = _binding.ND_OK + 4097
    assert _binding.nd_step_heun_noalloc(small, many, m, 1, 1e-14, np.zeros(many), np.zeros(many, np.uint64),
                                         check=False) == nd.ND_ERR_ARG
    host = np.zeros(3 * 30 * 32, dtype=np.float32)
    assert _binding.nd_step_heun_noalloc(small, 1, host, 1, 1e-14, T, s, check=False) == nd.ND_ERR_ARG
    assert "device pointer" in nd.nd_last_error()


def test_noalloc_refuses_stream_capture():
    """A captured call would replay stale parameter blocks, so it is refused
    on a capturing stream before any work is issued; the capture stays valid
    and an ordinary call afterwards steps as before."""
    import torch
    disk = Disk(30e-9, 5e-9, alpha=0.02)
    h = Nanodisk([disk], [1], nd.ND_FP32)
    m = h.empty_device()
    h.init_vortex(m, np.zeros((1, 2)))
    T, s = np.full(1, 300.0), np.arange(1, dtype=np.uint64)
    _binding.nd_step_heun_noalloc(disk, 1, m, 1, 1e-14, T, s)           # first call outside any capture
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    scratch = torch.zeros(4, device="cuda")
    with torch.cuda.graph(g, stream=side):
        rc = _binding.nd_step_heun_noalloc(disk, 1, m, 1, 1e-14, T, s, stream=side, check=False)
        scratch.add_(1.0)                                                  # the capture itself goes on
    assert rc == nd.ND_ERR_ARG and "captured" in nd.nd_last_error()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(scratch, torch.ones(4, device="cuda"))
    before = m.clone()
    assert _binding.nd_step_heun_noalloc(disk, 1, m, 1, 1e-14, T, s, step0=1) == nd.ND_OK
    torch.cuda.synchronize()
    assert not torch.equal(before, m)
