"""One evaluation split into partitions by contiguous Morton-key ranges of
leaves, the partitions run one after another on one GPU with exactly the
data the exchange plan moves: each partition forms the multipoles of its own
particles (fmm2d_multipoles), adds the partial multipoles the plan says the
others send for its interaction lists, and evaluates its own particles with
the halo particles of its neighbouring leaves from the summed multipoles
(fmm2d_velocity_from_multipoles).  The result must match the oracle FMM as
one evaluation does: 1e-12 in FP64, 1e-6 in the FP32 tensor-core form."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plan_cls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0809_1810_gb300 import Plan

    torch.cuda.set_device(0)
    oracle.build()
    return Plan


CASES = [
    # (workload, ranks, precision, cutoff in sigma)
    ("uniform", 2, "fp64", 0.0),
    ("uniform", 3, "fp64", 0.0),
    ("clustered", 2, "fp64", 0.0),
    ("uniform", 2, "fp32_tc", 0.0),
    ("clustered", 3, "fp32_tc", 0.0),
    ("uniform", 2, "fp32_tc", 4.6),
    ("uniform", 3, "fp64", 2.6),
]


@pytest.mark.parametrize("kind,ranks,prec,cut", CASES)
def test_split_matches_oracle_fmm(plan_cls, kind, ranks, prec, cut):
    from paper_0809_1810_gb300 import partition as PT

    npdt = np.float64 if prec == "fp64" else np.float32
    if kind == "uniform":
        w = W.uniform_random(24000, 61 + ranks, 2.0 / 155, sigma_over_h=1.5, p=14, L=5,
                             dtype=npdt)
    else:
        w = W.clustered_patches(30000, 62 + ranks, 8, 2.0 / 173, p=18, L=6, dtype=npdt)
    a = cut * w.sigma
    if a > 0 and w.L >= 2:
        assert a <= 2.0 * w.root[2] / 2 ** w.L
    dt = torch.float64 if prec == "fp64" else torch.float32
    xy = torch.tensor(np.stack([w.x, w.y], 1), dtype=dt, device="cuda")
    g = torch.tensor(w.gamma, dtype=dt, device="cuda")

    def factory(n):
        return plan_cls(w.p, w.L, w.sigma, prec, root=w.root, max_n=n, cutoff=a)

    uv, plan, bounds = PT.split_evaluate(factory, xy, g, w.L, w.root, ranks,
                                         reach=2 if a > 0 else 1)
    torch.cuda.synchronize()
    assert len(bounds) == ranks + 1 and all(b1 > b0 for b0, b1 in zip(bounds[:-1], bounds[1:]))
    # every pair of ranks exchanges something: the split is not trivial
    assert all(e["leaves"].size > 0 for (q, r), e in plan.items() if abs(q - r) == 1)
    ref = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.p, w.L, w.root, a=a)
    err = np.abs(uv.double().cpu().numpy() - ref).max() / np.abs(ref).max()
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert err < tol, err


def test_multipoles_of_parts_add_up(plan_cls):
    """Eq. 20 is linear in the particles: the multipoles of two halves of a
    set add up to those of the whole (FP64, to rounding)."""
    w = W.uniform_random(20000, 71, 2.0 / 141, sigma_over_h=1.0, p=12, L=5, dtype=np.float64)
    xy = torch.tensor(np.stack([w.x, w.y], 1), device="cuda")
    g = torch.tensor(w.gamma, device="cuda")
    with plan_cls(w.p, w.L, w.sigma, "fp64", root=w.root, max_n=w.n) as pl:
        reals = pl.multipole_reals()
        whole = pl.multipoles(xy, g).clone()
        a = pl.multipoles(xy[:7000].contiguous(), g[:7000].contiguous()).clone()
        b = pl.multipoles(xy[7000:].contiguous(), g[7000:].contiguous()).clone()
        torch.cuda.synchronize()
    assert reals == 2 * 16 * sum(4 ** lev for lev in range(2, w.L + 1)) == whole.numel()
    np.testing.assert_allclose((a + b).cpu().numpy(), whole.cpu().numpy(), rtol=0,
                               atol=1e-14 * whole.abs().max().item())
