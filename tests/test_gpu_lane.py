"""Sparse leaves in the FP32 near field: the per-target-lane pass.

In an evaluation with at most 32 particles per leaf on average, leaves of at
most 16 particles are evaluated one target per lane (each lane walking its
own target's local list, Sec. 3.3.1), the other leaves by the warp path.
Bars:
* FP32 and FP32_TC within 1e-6 of the oracle's FMM at the same (p, L, a)
  on both sides of both thresholds (leaf counts 16 / 17, mean occupancy 32 /
  just above), with and without the Sec. 4.1 cutoff, at every L the near
  field handles alone (0, 1) and with a far field;
* repeat evaluations bit-identical;
* the pass runs exactly when the evaluation is sparse (one more kernel per
  call);
* a batch of sparse instances equal to their single plans bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
FP32_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0809_1810_gb300 import build

    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _counts_instance(pattern, L, seed, soh, p):
    """Leaf (ix, iy) of level L holds pattern[(ix + 3 iy) % len] particles,
    uniform inside the leaf (a margin of 2% of a leaf from its sides, so that
    no coordinate rounds into a neighbour); circulations h^2 N(0, 1)."""
    x0, y0, Wd = W.ROOT
    nl = 1 << L
    s = Wd / nl
    rng = np.random.Generator(np.random.PCG64(seed))
    xs, ys = [], []
    for iy in range(nl):
        for ix in range(nl):
            c = pattern[(ix + 3 * iy) % len(pattern)]
            xs.append(x0 + (ix + rng.uniform(0.02, 0.98, c)) * s)
            ys.append(y0 + (iy + rng.uniform(0.02, 0.98, c)) * s)
    x = np.concatenate(xs)
    y = np.concatenate(ys)
    n = x.size
    h = Wd / np.sqrt(max(n, 1))
    gamma = h * h * rng.standard_normal(n)
    return W.Workload(f"counts_L{L}_n{n}", x.astype(np.float32), y.astype(np.float32),
                      gamma.astype(np.float32), soh * h, p, L, h)


def _velocity(w, prec, cutoff=0.0, repeats=1):
    from paper_0809_1810_gb300 import Plan

    xy = torch.tensor(np.stack([w.x, w.y], 1), device="cuda")
    g = torch.tensor(w.gamma, device="cuda")
    with Plan(w.p, w.L, w.sigma, prec, root=w.root, max_n=max(w.n, 1), cutoff=cutoff) as plan:
        outs = [plan.velocity(xy, g, check=True).clone() for _ in range(repeats)]
        kernels = plan.kernels_per_call()
    return outs, kernels


def _ref(w, cutoff=0.0):
    return oracle.fmm(w.x.astype(np.float64), w.y.astype(np.float64),
                      w.gamma.astype(np.float64), w.sigma, w.p, w.L, w.root, a=cutoff)


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


# leaves of 0, 1, 2, 15, 16 (lane pass) and 17, 18, 40 (warp path) particles,
# mean 13.6 per leaf
PATTERN = [0, 1, 2, 15, 16, 17, 18, 40]


@pytest.mark.parametrize("prec", ["fp32", "fp32_tc"])
@pytest.mark.parametrize("cut", [False, True])
def test_leaf_count_threshold_against_oracle(prec, cut):
    w = _counts_instance(PATTERN, 4, 11, 1.0, 14)
    # leaves of 2.5 sigma; a = 1.9 leaf widths = 4.75 sigma keeps the cutoff's
    # jump below the FP32 bar while the ring corrections stay visible
    leaf = w.root[2] / 2 ** w.L
    w.sigma = leaf / 2.5
    a = 1.9 * leaf if cut else 0.0
    (uv,), _ = _velocity(w, prec, a)
    err = _rel(uv.double().cpu().numpy(), _ref(w, a))
    assert err <= FP32_TOL, (prec, cut, err)


@pytest.mark.parametrize("prec", ["fp32", "fp32_tc"])
def test_mean_occupancy_threshold(prec):
    """n = 32 4^L takes the lane pass (one kernel more per call), n + 1 does
    not; both within the FP32 bar."""
    L = 4
    kernels = {}
    for n in (32 << (2 * L), (32 << (2 * L)) + 1):
        w = W.uniform_random(n, 7, 2.0 / np.sqrt(n), sigma_over_h=2.0, p=12, L=L,
                             dtype=np.float32)
        (uv,), kernels[n] = _velocity(w, prec)
        err = _rel(uv.double().cpu().numpy(), _ref(w))
        assert err <= FP32_TOL, (n, err)
    assert kernels[32 << (2 * L)] == kernels[(32 << (2 * L)) + 1] + 1, kernels


@pytest.mark.parametrize("L,n", [(0, 1), (0, 16), (0, 17), (1, 60), (1, 128)])
def test_near_field_only_levels(L, n):
    """L < 2: the near field is the whole sum (no far field), every particle
    in the lane pass where its leaf holds at most 16."""
    w = W.uniform_random(n, 30 + n, 2.0 / np.sqrt(n), sigma_over_h=1.5, p=8, L=L,
                         dtype=np.float32)
    (uv,), _ = _velocity(w, "fp32")
    ref = _ref(w)
    if np.abs(ref).max() == 0.0:
        assert np.abs(uv.cpu().numpy()).max() == 0.0
    else:
        assert _rel(uv.double().cpu().numpy(), ref) <= FP32_TOL


def test_repeat_evaluations_bit_identical():
    w = _counts_instance(PATTERN, 5, 12, 1.0, 16)
    leaf = w.root[2] / 2 ** w.L
    w.sigma = leaf / 2.2
    outs, _ = _velocity(w, "fp32_tc", 1.9 * leaf, repeats=4)
    assert all(torch.equal(outs[0], o) for o in outs[1:])


def test_clustered_sparse_instance():
    """Gaussian patches at a level fine enough that the mean occupancy is
    under 32: dense patch cores (warp path) beside sparse fringes (lane
    pass) whose local lists reach into the cores."""
    w = W.clustered_patches(12000, 9, npatch=5, h=2.0 / 110, sigma_over_h=1.0, p=16, L=5,
                            dtype=np.float32)
    assert w.n <= 32 << (2 * w.L)
    leaf = w.root[2] / 2 ** w.L
    a = 1.9 * leaf if 1.9 * leaf >= 4.4 * w.sigma else 0.0
    (uv,), _ = _velocity(w, "fp32_tc", a)
    assert _rel(uv.double().cpu().numpy(), _ref(w, a)) <= FP32_TOL


@pytest.mark.parametrize("prec", ["fp32", "fp32_tc"])
def test_sparse_batch_equals_single_plans(prec):
    from paper_0809_1810_gb300 import BatchPlan

    ws = [_counts_instance(PATTERN, 3, 20, 1.0, 6), _counts_instance(PATTERN, 4, 21, 1.0, 20),
          _counts_instance([3, 5, 0, 9], 5, 22, 1.0, 11),
          W.uniform_random(3000, 23, 2.0 / 55, sigma_over_h=1.5, p=10, L=4, dtype=np.float32)]
    cuts = []
    for k, w in enumerate(ws):
        leaf = w.root[2] / 2 ** w.L
        w.sigma = leaf / 2.3
        cuts.append(1.9 * leaf if k % 2 == 0 else 0.0)
    xy = torch.tensor(np.concatenate([np.stack([w.x, w.y], 1) for w in ws]), device="cuda")
    g = torch.tensor(np.concatenate([w.gamma for w in ws]), device="cuda")
    with BatchPlan([{"n": w.n, "p": w.p, "L": w.L, "sigma": w.sigma, "root": w.root,
                     "cutoff": c} for w, c in zip(ws, cuts)], precision=prec) as bp:
        uv = bp.velocity(xy, g)
        again = bp.velocity(xy, g)
        bp.check()
    assert torch.equal(uv, again)
    off = 0
    for w, c in zip(ws, cuts):
        (single,), _ = _velocity(w, prec, c)
        assert torch.equal(uv[off:off + w.n], single), (w.name, c)
        off += w.n
