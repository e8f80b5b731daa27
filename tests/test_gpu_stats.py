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
