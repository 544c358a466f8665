"""The convection step of Eq. 5 on the GPU (fmm2d_convect, Plan.convect):
forward Euler and Heun on the plan's FMM velocities, positions updated in
place.

Bars: one step of 20,000 particles against the oracle's step on the oracle
FMM at the same (p, L) -- 1e-10 of the largest displacement in FP64; in FP32
and FP32_TC 1e-6 of it plus two FP32 units of the coordinates (the new
positions are rounded to FP32).  A co-rotating pair of vortices, stepped on
the GPU, stays on its exact circle with errors falling at the integrator's
order.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0809_1810_gb300 import build

    build.build()
    oracle.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_tc"])
def test_one_step_matches_the_oracle(prec, order):
    from paper_0809_1810_gb300 import Plan

    dt_t, npdt = (torch.float64, np.float64) if prec == "fp64" else (torch.float32, np.float32)
    w = W.uniform_random(20000, 81, 2.0 / 141, sigma_over_h=1.5, p=16, L=5, dtype=npdt)
    w.x, w.y = (0.9 * w.x).astype(npdt), (0.9 * w.y).astype(npdt)  # room to move in the box
    xy = torch.tensor(np.stack([w.x, w.y], 1), dtype=dt_t, device="cuda")
    g = torch.tensor(w.gamma, dtype=dt_t, device="cuda")
    with Plan(w.p, w.L, w.sigma, prec, root=w.root, max_n=w.n) as plan:
        u0 = plan.velocity(xy, g, check=True).double().cpu().numpy()
        dt = 0.02 / np.abs(u0).max()  # the fastest particle moves 0.02
        plan.convect(xy, g, dt, order=order, check=True)
        new = xy.double().cpu().numpy()

    def vel(x, y):
        return oracle.fmm(x, y, w.gamma, w.sigma, w.p, w.L, w.root)

    ox, oy = oracle.convect(w.x, w.y, w.gamma, dt, vel, order=order)
    want = np.stack([ox, oy], 1)
    moved = np.abs(want - np.stack([w.x, w.y], 1).astype(np.float64)).max()
    assert moved > 0.01
    err = np.abs(new - want).max()
    bar = 1e-10 * moved if prec == "fp64" else 1e-6 * moved + 2 * 2.0 ** -23
    assert err <= bar, (err, bar, moved)


@pytest.mark.parametrize("order", [1, 2])
def test_co_rotating_pair_on_the_gpu(order):
    """Two equal vortices (sigma = 0.05, d = 0.1) turn about their midpoint at
    Omega = 2 Gamma (1 - exp(-d^2 / 2 sigma^2)) / (2 pi d^2); a quarter turn in
    20, 40 and 80 FP64 steps converges at the integrator's order."""
    from paper_0809_1810_gb300 import Plan

    sigma, d, g0 = 0.05, 0.1, 1.0
    omega = 2 * g0 * (1 - math.exp(-d * d / (2 * sigma * sigma))) / (2 * math.pi * d * d)
    errs = []
    for steps in (20, 40, 80):
        dt = 0.25 * 2 * math.pi / omega / steps
        xy = torch.tensor([[-d / 2, 0.0], [d / 2, 0.0]], dtype=torch.float64, device="cuda")
        g = torch.tensor([g0, g0], dtype=torch.float64, device="cuda")
        with Plan(4, 0, sigma, "fp64", root=(-1.0, -1.0, 2.0), max_n=2) as plan:
            for _ in range(steps):
                plan.convect(xy, g, dt, order=order)
            plan.check()
        th = omega * steps * dt
        want = np.array([[-d / 2 * math.cos(th), -d / 2 * math.sin(th)],
                         [d / 2 * math.cos(th), d / 2 * math.sin(th)]])
        errs.append(np.abs(xy.cpu().numpy() - want).max() / d)
    rates = [math.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert all(abs(r - order) < 0.15 for r in rates), (errs, rates)


def test_convect_rejects_bad_arguments():
    from paper_0809_1810_gb300 import FMMError, Plan

    w = W.uniform_random(500, 82, 0.09, p=6, L=3, dtype=np.float32)
    xy = torch.tensor(np.stack([w.x, w.y], 1), device="cuda")
    g = torch.tensor(w.gamma, device="cuda")
    with Plan(w.p, w.L, w.sigma, "fp32", root=w.root, max_n=w.n) as plan:
        with pytest.raises(FMMError):
            plan.convect(xy, g, 0.01, order=3)
        with pytest.raises(FMMError):
            plan.convect(xy, g, float("nan"))
        before = xy.clone()
        plan.convect(xy, g, 0.0, check=True)  # dt = 0 leaves the positions
        assert torch.equal(xy, before)
