"""Failure detection on the GPU without a fault: the tensor-core M2L bounds
every wait on its pipeline barriers by a poll limit.  Here the limit is made
so short that the waits run out; the kernel must stop cleanly (the copies and
MMAs it already issued completed, its tensor memory freed), report
FMM2D_TIMEOUT through fmm2d_plan_check, and leave the context usable: the next
evaluation with the default limit reproduces the earlier result bit for bit."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plan_cls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0809_1810_gb300 import Plan

    torch.cuda.set_device(0)
    return Plan


@pytest.mark.parametrize("p,L", [(16, 5), (20, 6)])
def test_m2l_wait_limit_reports_timeout_and_recovers(plan_cls, p, L):
    from paper_0809_1810_gb300 import FMMError, _native

    w = W.uniform_random(30000, 40 + p, 2.0 / 173, sigma_over_h=1.0, p=p, L=L,
                         dtype=np.float32)
    xy = torch.tensor(np.stack([w.x, w.y], 1), device="cuda")
    g = torch.tensor(w.gamma, device="cuda")
    with plan_cls(w.p, w.L, w.sigma, "fp32_tc", root=w.root, max_n=w.n) as plan:
        before = plan.velocity(xy, g, check=True).clone()
        plan.set_spin_limit(1)  # one poll of about 32 ns: the waits run out
        plan.velocity(xy, g)
        with pytest.raises(FMMError) as err:
            plan.check()
        assert err.value.status == _native.TIMEOUT
        plan.set_spin_limit(0)  # the default limit again
        after = plan.velocity(xy, g, check=True)
        torch.cuda.synchronize()
        assert torch.equal(after, before)
