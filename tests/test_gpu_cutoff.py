"""The cutoff a of Sec. 4.1 on the GPU (fmm2d_params.cutoff): pairs closer than
a keep the regularised kernel even when their leaves are not neighbours.

Bars as in test_gpu_parity: FP64 within 1e-12 of the oracle's cut FMM at the
same (p, L, a), FP32 and FP32_TC within 1e-6; the hybrid yardstick with the
cutoff within 1e-13 of the oracle's cut hybrid sum.  The benchmark's stated
configuration (2^20 uniform particles, p = 16, L = 7, leaves of 4 sigma)
misses 1e-6 against the direct sum under the plain 3x3 rule and meets it with
a = 5 sigma.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0809_1810_gb300 import build

    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _dev(w, dtype):
    xy = torch.tensor(np.stack([w.x, w.y], 1), dtype=dtype, device="cuda")
    g = torch.tensor(w.gamma, dtype=dtype, device="cuda")
    return xy, g


def _plan(w, prec, cutoff):
    from paper_0809_1810_gb300 import Plan

    return Plan(w.p, w.L, w.sigma, prec, root=w.root, max_n=max(w.n, 1), cutoff=cutoff)


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _rel_speed(uv, ref):
    return np.linalg.norm(uv - ref, axis=1).max() / np.linalg.norm(ref, axis=1).max()


def _leaf(w):
    return w.root[2] / 2 ** w.L


def _cases(specs, clustered):
    # specs: (n, p, L, sigma / h, a / leaf width)
    for n, p, L, soh, af in specs:
        yield (f"uniform_n{n}_p{p}_L{L}_a{af}",
               lambda dt, n=n, p=p, L=L, soh=soh: W.uniform_random(
                   n, n + p + 5, 2.0 / np.sqrt(n), sigma_over_h=soh, p=p, L=L, dtype=dt), af)
    soh, af = clustered
    yield (f"clustered_20000_a{af}",
           lambda dt: W.clustered_patches(20000, 4, npatch=6, h=2.0 / 140, sigma_over_h=soh,
                                          p=14, L=5, dtype=dt), af)


# FP64: leaf / sigma = 2.4, 1.4, 2.2, 0.7 and 1.5, a = 2.2 to 3.6 sigma --
# ring corrections of up to a third of a pair's singular value
FP64_CASES = list(_cases([(6007, 16, 4, 2.0, 1.5), (8191, 12, 5, 2.0, 2.0),
                          (5000, 8, 2, 8.0, 1.2), (12000, 20, 6, 2.5, 1.7)], (3.0, 1.5)))
# FP32: the cutoff is a hard threshold, where the correction jumps by
# exp(-a^2 / 2 sigma^2) of the pair's singular value; a pair within FP32
# rounding of r = a may be decided either way, so these cases keep that jump
# below the FP32 bar (a >= 4.4 sigma) while the ring corrections stay visible
# (leaf / sigma = 2.2 to 2.6)
FP32_CASES = list(_cases([(6007, 16, 4, 2.0, 1.9), (8191, 12, 5, 1.1, 1.8),
                          (5000, 8, 2, 8.0, 2.0), (12000, 20, 6, 0.7, 1.9)], (1.8, 1.9)))


@pytest.mark.parametrize("name,make,af", FP64_CASES, ids=[c[0] for c in FP64_CASES])
def test_fp64_cutoff_matches_oracle(name, make, af):
    w = make(np.float64)
    a = af * _leaf(w)
    ref = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.p, w.L, w.root, a=a)
    xy, g = _dev(w, torch.float64)
    with _plan(w, "fp64", a) as plan:
        uv = plan.velocity(xy, g, check=True).cpu().numpy()
    assert _rel(uv, ref) <= FP64_TOL, _rel(uv, ref)
    # the cutoff changed the result: without it the FMM is far from this one
    plain = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.p, w.L, w.root)
    assert _rel(plain, ref) > 1e3 * FP64_TOL


@pytest.mark.parametrize("prec", ["fp32", "fp32_tc"])
@pytest.mark.parametrize("name,make,af", FP32_CASES, ids=[c[0] for c in FP32_CASES])
def test_fp32_cutoff_matches_oracle(name, make, af, prec):
    w = make(np.float32)
    a = af * _leaf(w)
    assert a >= 4.4 * w.sigma
    ref = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.p, w.L, w.root, a=a)
    xy, g = _dev(w, torch.float32)
    with _plan(w, prec, a) as plan:
        uv = plan.velocity(xy, g, check=True).double().cpu().numpy()
    assert _rel(uv, ref) <= FP32_TOL, _rel(uv, ref)
    # the ring corrections are visible at the FP32 bar
    plain = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.p, w.L, w.root)
    assert _rel(plain, ref) > 10 * FP32_TOL, _rel(plain, ref)


# (n, p, L, sigma / h, a / leaf width) where ring strips apply (a at most 1.5
# leaf widths) and a >= 4.4 sigma, so that the FP32 bar holds against the
# oracle's cut FMM: mean occupancy 47 and 39 per leaf (the warp path for
# every leaf, its ring gathered from the strips), and 8 (mostly the
# per-target-lane pass, which walks whole ring leaves).
STRIP_ORACLE_CASES = [(12000, 14, 4, 2.0, 1.40), (40000, 12, 5, 1.8, 1.45),
                      (8192, 10, 5, 0.83, 1.45)]


@pytest.mark.parametrize("prec", ["fp32", "fp32_tc"])
@pytest.mark.parametrize("n,p,L,soh,af", STRIP_ORACLE_CASES)
def test_strip_geometry_matches_oracle(n, p, L, soh, af, prec):
    w = W.uniform_random(n, n + 11, 2.0 / np.sqrt(n), sigma_over_h=soh, p=p, L=L,
                         dtype=np.float32)
    a = af * _leaf(w)
    assert a >= 4.4 * w.sigma
    ref = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.p, w.L, w.root, a=a)
    xy, g = _dev(w, torch.float32)
    with _plan(w, prec, a) as plan:
        uv = plan.velocity(xy, g, check=True).double().cpu().numpy()
    assert _rel(uv, ref) <= FP32_TOL, _rel(uv, ref)
    # the ring corrections are there: without them the FMM is off the bar
    plain = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.p, w.L, w.root)
    assert _rel(plain, ref) > FP32_TOL, _rel(plain, ref)


# (n, L, sigma / h, a / leaf width): the ring sources of every leaf fit one
# shared-memory chunk (at most 558) from whole leaves and from strips alike;
# strips are used up to a = 1.5 leaf widths (half-leaf strips)
STRIP_CASES = [(6007, 4, 2.0, 1.2), (8191, 5, 1.1, 1.31), (12000, 6, 0.7, 1.45),
               (24000, 5, 2.0, 1.499)]


@pytest.mark.parametrize("prec", ["fp32", "fp32_tc"])
@pytest.mark.parametrize("n,L,soh,af", STRIP_CASES)
def test_ring_strips_keep_the_whole_leaves_sources(n, L, soh, af, prec):
    """The FP32 near field gathers each ring leaf's strip on the side facing
    the target leaf instead of the whole leaf: the strip must hold every
    source the whole leaf would give (closer than a, with the kernel's
    margin, to the target leaf's square), in the same order, so the
    velocities agree bit for bit.  A strip too narrow would drop the ring
    pairs nearest the cutoff, whose corrections are below the FP32 bar."""
    w = W.uniform_random(n, n + 7, 2.0 / np.sqrt(n), sigma_over_h=soh, p=10, L=L,
                         dtype=np.float32)
    xy, g = _dev(w, torch.float32)
    with _plan(w, prec, af * _leaf(w)) as plan:
        strips = plan.velocity(xy, g, check=True).clone()
        plan.set_ring_strips(False)
        whole = plan.velocity(xy, g, check=True).clone()
        plan.set_ring_strips(True)
        again = plan.velocity(xy, g, check=True)
    assert torch.equal(strips, whole)
    assert torch.equal(strips, again)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_tc"])
def test_cutoff_within_a_leaf_changes_nothing(prec):
    """Leaves two apart are at least a leaf width apart: a cutoff below one
    leaf width corrects no pair, and the result is bit for bit the plain one
    (the ring is gathered and found empty)."""
    dt = np.float64 if prec == "fp64" else np.float32
    w = W.uniform_random(20000, 41, 2.0 / 141, sigma_over_h=2.0, p=10, L=5, dtype=dt)
    xy, g = _dev(w, torch.float64 if prec == "fp64" else torch.float32)
    with _plan(w, prec, 0.0) as plan:
        plain = plan.velocity(xy, g, check=True).clone()
    with _plan(w, prec, 0.99 * _leaf(w)) as plan:
        cut = plan.velocity(xy, g, check=True)
    assert torch.equal(plain, cut)


def test_cutoff_is_ignored_without_far_field():
    """With L < 2 every pair is in the local list and keeps K_sigma anyway."""
    w = W.uniform_random(3000, 42, 2.0 / 55, sigma_over_h=2.0, p=6, L=1, dtype=np.float64)
    xy, g = _dev(w, torch.float64)
    with _plan(w, "fp64", 0.0) as plan:
        plain = plan.velocity(xy, g, check=True).clone()
    with _plan(w, "fp64", 5.0) as plan:  # any cutoff is accepted at L < 2
        cut = plan.velocity(xy, g, check=True)
    assert torch.equal(plain, cut)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_hybrid_yardstick_with_cutoff(prec):
    dtype = np.float64 if prec == "fp64" else np.float32
    w = W.uniform_random(9000, 43, 2.0 / 95, sigma_over_h=2.0, p=8, L=5, dtype=dtype)
    a = 1.6 * _leaf(w)
    t = W.sample_targets(w.n, 333, 6)
    xy, g = _dev(w, torch.float64 if prec == "fp64" else torch.float32)
    with _plan(w, prec, a) as plan:
        got = plan.direct_sampled(xy, g, torch.tensor(t, device="cuda"), kernel=1)
        plan.check()
    ref = oracle.hybrid(w.x, w.y, w.gamma, w.sigma, w.root, w.L, targets=t, a=a)
    assert _rel(got.cpu().numpy(), ref) <= 1e-13


def test_cutoff_beyond_two_leaves_is_rejected():
    from paper_0809_1810_gb300 import FMMError

    w = W.uniform_random(100, 44, 0.1, p=6, L=4, dtype=np.float32)
    with pytest.raises(FMMError):
        _plan(w, "fp32", 2.01 * _leaf(w))


def test_benchmark_configuration_meets_the_bar_with_the_cutoff():
    """2^20 uniform particles, sigma = 2h, p = 16, L = 7 (leaves of 4 sigma),
    FP32_TC.  Under the plain 3x3 rule the kernel substitution of Eq. 29
    leaves max |du| / max |u| above 1e-6 against the regularised direct sum;
    with a = 5 sigma every output is within 1e-6 of the oracle's cut FMM and
    the metric's bar holds at 256 seeded particles."""
    w = W.uniform_1m()
    assert (w.p, w.L) == (16, 7)
    a = 5.0 * w.sigma
    xy, g = _dev(w, torch.float32)
    t = W.sample_targets(w.n, 256, 14)
    o1 = oracle.direct(w.x, w.y, w.gamma, w.sigma, targets=t)
    with _plan(w, "fp32_tc", 0.0) as plan:
        plain = plan.velocity(xy, g, check=True).double().cpu().numpy()
    assert _rel_speed(plain[t], o1) > 1e-6
    with _plan(w, "fp32_tc", a) as plan:
        uv = plan.velocity(xy, g, check=True).double().cpu().numpy()
    assert _rel_speed(uv[t], o1) <= 1e-6, _rel_speed(uv[t], o1)
    ref = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.p, w.L, w.root, a=a)
    assert _rel(uv, ref) <= FP32_TOL, _rel(uv, ref)
