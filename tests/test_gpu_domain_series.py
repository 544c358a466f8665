"""The domain-size series of Sec. 5.1 / Fig. 19 through the batched path:
the Lamb-Oseen setup at a fixed lattice spacing (sigma = 0.02, h = 0.8 sigma,
nu t = 0.002) on 63^2, 88^2 and 138^2 particles, at level l = 4 with p = 13
and p = 19, six instances in one batched evaluation.

The domain grows with the particle count, so the leaves widen (3.2, 4.4 and
6.9 sigma) and the kernel-substitution error of Sec. 4.1 -- far-field pairs
taken with the singular kernel -- falls: the paper's reading of Fig. 19,
whose values were lost in extraction.  Bars: every instance within 1e-6 of
the oracle FMM (FP32 batch path); against the FP64 direct sum the smallest
domain's kernel error dominates (the strict fall across all three, down to
1e-9, is pinned on the FP64 oracle in test_oracle_pins.py: FP32 rounding
sits near 1e-7), the wider domains meet 1e-6 at p = 19, errors lie within
the Eq. 29 estimate where leaves are narrower than 5 sigma, and on the
widest domain the truncation order shows.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

SIDES = (63, 88, 138)
ORDERS = (13, 19)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0809_1810_gb300 import build

    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def test_domain_size_series_in_one_batch():
    from paper_0809_1810_gb300 import BatchPlan

    ws = [W.lamb_oseen_fixed_spacing(s, p=p, L=4, dtype=np.float32)
          for p in ORDERS for s in SIDES]
    xy = torch.tensor(np.concatenate([np.stack([w.x, w.y], 1) for w in ws]), device="cuda")
    g = torch.tensor(np.concatenate([w.gamma for w in ws]), device="cuda")
    specs = [{"n": w.n, "p": w.p, "L": w.L, "sigma": w.sigma, "root": w.root} for w in ws]
    with BatchPlan(specs) as bp:
        uv = bp.velocity(xy, g)
        bp.check()
        every = torch.arange(bp.n_total, device="cuda")
        ref = bp.direct_sampled(xy, g, every, kernel=0)
        stats = bp.error_stats(xy, uv, every, ref).cpu().numpy()
        uv = uv.double().cpu().numpy()
        off = bp.offsets
    err = stats[:, 0] / stats[:, 1]
    rows = []
    for k, w in enumerate(ws):
        o = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.p, w.L, w.root)
        got = uv[off[k]:off[k + 1]]
        assert np.abs(got - o).max() / np.abs(o).max() <= 1e-6, (w.name, w.p)
        leaf = w.root[2] / 2 ** w.L
        # Eq. 29 at a = the leaf width, relative to the largest speed
        est = (math.exp(-leaf * leaf / (2 * w.sigma ** 2)) * np.abs(w.gamma).sum()
               / (2 * math.pi * leaf) / stats[k, 1])
        rows.append((w.n, w.p, leaf / w.sigma, err[k], est))
    print()
    for r in rows:
        print("N %6d p %2d leaf/sigma %.2f  max err %.2e  Eq. 29 estimate %.2e" % r)
    hi = [r for r in rows if r[1] == 19]
    assert hi[0][3] > 1e-4 and hi[0][3] > 100 * max(hi[1][3], hi[2][3]), hi
    assert hi[1][3] <= 1e-6 and hi[2][3] <= 1e-6, hi
    for r in rows:
        if r[2] < 5:  # where the kernel error dominates, Eq. 29 bounds it
            assert r[3] <= r[4], r
    # where the leaves are wide the truncation order shows: p = 13 above p = 19
    lo = [r for r in rows if r[1] == 13]
    assert lo[2][3] > hi[2][3], (lo[2], hi[2])
