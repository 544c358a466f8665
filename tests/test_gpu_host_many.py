"""Pipelined evaluations from host buffers (fmm2d_velocity_host_many): each of
several independent particle sets, copied in while the previous one is
evaluated and copied back while the next one is, must get exactly the
velocities a synchronous host-buffer call (and a device call) gives it."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plan_cls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0809_1810_gb300 import Plan, build

    build.build()
    torch.cuda.set_device(0)
    return Plan


def _sets(count, n, dt):
    out = []
    for k in range(count):
        # sigma = h: a cutoff of 5.26 sigma is 1.19 leaf widths at L = 5
        w = W.uniform_random(n, 300 + k, 2.0 / np.sqrt(n), sigma_over_h=1.0, p=12, L=5,
                             dtype=dt)
        xy = torch.tensor(np.stack([w.x, w.y], 1)).pin_memory()
        g = torch.tensor(w.gamma).pin_memory()
        out.append((w, xy, g))
    return out


@pytest.mark.parametrize("prec,cut", [("fp32_tc", 5.256521769756932), ("fp32", 0.0),
                                      ("fp64", 0.0)])
def test_pipelined_sets_equal_one_at_a_time(plan_cls, prec, cut):
    dt = np.float64 if prec == "fp64" else np.float32
    sets = _sets(5, 20000, dt)
    w0 = sets[0][0]
    with plan_cls(w0.p, w0.L, w0.sigma, prec, root=w0.root, max_n=20000,
                  cutoff=cut * w0.sigma) as plan:
        outs = [torch.empty_like(xy).pin_memory() for _, xy, _ in sets]
        plan.velocity_host_many([xy for _, xy, _ in sets], [g for _, _, g in sets], outs)
        for (w, xy, g), got in zip(sets, outs):
            one = torch.empty_like(xy).pin_memory()
            plan.velocity_host(xy, g, one)
            assert torch.equal(got, one)
            dev = plan.velocity(xy.cuda(), g.cuda(), check=True).cpu()
            assert torch.equal(got, dev)
        # again: the staging sets and the recorded graph are reused
        again = [torch.empty_like(o).pin_memory() for o in outs]
        plan.velocity_host_many([xy for _, xy, _ in sets], [g for _, _, g in sets], again)
        assert all(torch.equal(a, b) for a, b in zip(outs, again))


def test_pipelined_edge_counts(plan_cls):
    sets = _sets(1, 5000, np.float32)
    w, xy, g = sets[0]
    with plan_cls(w.p, w.L, w.sigma, "fp32", root=w.root, max_n=5000) as plan:
        plan.velocity_host_many([], [], [])  # no set: nothing to do
        out = torch.empty_like(xy).pin_memory()
        plan.velocity_host_many([xy], [g], [out])  # one set: no overlap, same result
        one = torch.empty_like(xy).pin_memory()
        plan.velocity_host(xy, g, one)
        assert torch.equal(out, one)
        with pytest.raises(ValueError):
            plan.velocity_host_many([xy], [g, g], [out])
