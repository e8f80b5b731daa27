"""Device-resident core statistics against a host-side accumulation of the
per-sample core positions (nd_vortex_core) over the same Heun run."""
import numpy as np
import pytest

import paper_1207_2192_gb300 as nd
from paper_1207_2192_gb300 import Disk, Nanodisk

pytestmark = pytest.mark.gpu


def test_stats_match_host_accumulation():
    disk = Disk(20e-9, 10e-9, alpha=0.05)
    B = 4
    h = Nanodisk([disk], [B], nd.ND_FP32)
    m = h.empty_device()
    h.init_vortex(m, np.array([[2e-9, 0.0], [0.0, 2e-9], [-1e-9, 1e-9], [0.0, 0.0]]))
    rb, vb, rmax, vmax = 40, 30, 8e-9, 300.0
    nd.nd_stats_reset(h.h, rmax, rb, vmax, vb)
    dt, nsub = 1e-14, 20
    T, seeds = np.full(B, 300.0), np.arange(B, dtype=np.uint64)
    n = np.zeros(B); sx = np.zeros(B); sy = np.zeros(B); sr2 = np.zeros(B); nv = np.zeros(B); sv2 = np.zeros(B)
    hr = np.zeros((B, rb), np.uint64); hv = np.zeros((B, vb), np.uint64)
    prev = [None] * B
    step = 0
    for k in range(30):
        h.heun(m, nsub, dt, T, seeds, step0=step)
        step += nsub
        nd.nd_stats_sample(h.h, m, nsub * dt)
        Xc, st = h.vortex_core(m)
        for r in range(B):
            if st[r] != 0:
                prev[r] = None
                continue
            x, y = Xc[r]
            rr = np.sqrt(x * x + y * y)
            n[r] += 1; sx[r] += x; sy[r] += y; sr2[r] += x * x + y * y
            b = int(np.floor(rr / rmax * rb))
            if 0 <= b < rb:
                hr[r, b] += 1
            if prev[r] is not None:
                v = np.hypot(x - prev[r][0], y - prev[r][1]) / (nsub * dt)
                nv[r] += 1; sv2[r] += v * v
                bv = int(np.floor(v / vmax * vb))
                if 0 <= bv < vb:
                    hv[r, bv] += 1
            prev[r] = (x, y)
    mom, ghr, ghv = nd.nd_stats_read(h.h, B, rb, vb)
    assert np.array_equal(mom[:, 0], n) and np.array_equal(mom[:, 4], nv)
    assert np.allclose(mom[:, 1], sx, rtol=1e-12, atol=1e-24)
    assert np.allclose(mom[:, 2], sy, rtol=1e-12, atol=1e-24)
    assert np.allclose(mom[:, 3], sr2, rtol=1e-12, atol=1e-36)
    assert np.allclose(mom[:, 5], sv2, rtol=1e-10)
    assert np.abs(ghr.astype(np.int64) - hr.astype(np.int64)).sum() <= 2     # bin edges may differ by one ulp
    assert np.abs(ghv.astype(np.int64) - hv.astype(np.int64)).sum() <= 2
    assert ghr.sum() > 0 and ghv.sum() > 0


def test_stats_checkpoint_resume_is_exact():
    """A run split in two, with the state, the noise counter and the
    statistics record carried over to a fresh handle, accumulates exactly as
    the uninterrupted run: moments, speed chain and both histograms."""
    disk = Disk(20e-9, 10e-9, alpha=0.05)
    B, rb, vb, rmax, vmax = 3, 25, 20, 8e-9, 300.0
    T, seeds, dt, nsub = np.full(B, 300.0), np.arange(B, dtype=np.uint64) + 7, 1e-14, 20
    X0 = np.array([[2e-9, 0.0], [0.0, -1e-9], [1e-9, 1e-9]])

    def run(h, m, k0, k1):
        for k in range(k0, k1):
            h.heun(m, nsub, dt, T, seeds, step0=k * nsub)
            nd.nd_stats_sample(h.h, m, nsub * dt)

    ha = Nanodisk([disk], [B], nd.ND_FP32)
    ma = ha.empty_device()
    ha.init_vortex(ma, X0)
    nd.nd_stats_reset(ha.h, rmax, rb, vmax, vb)
    run(ha, ma, 0, 24)
    whole = nd.nd_stats_read(ha.h, B, rb, vb)

    hb = Nanodisk([disk], [B], nd.ND_FP32)
    mb = hb.empty_device()
    hb.init_vortex(mb, X0)
    nd.nd_stats_reset(hb.h, rmax, rb, vmax, vb)
    run(hb, mb, 0, 10)
    record, state = nd.nd_stats_save(hb.h), mb.clone()
    del hb

    hc = Nanodisk([disk], [B], nd.ND_FP32)
    nd.nd_stats_load(hc.h, record)
    run(hc, state, 10, 24)
    resumed = nd.nd_stats_read(hc.h, B, rb, vb)
    for a, b in zip(whole, resumed):
        assert np.array_equal(a, b)
    assert whole[0][:, 4].min() > 0                         # the speed chain crossed the split
    # records of another replica count or a damaged tag are refused
    hd = Nanodisk([disk], [B + 1], nd.ND_FP32)
    with pytest.raises(nd.NDError):
        nd.nd_stats_load(hd.h, record)
    with pytest.raises(nd.NDError):
        nd.nd_stats_load(hc.h, b"x" + record[1:])
