"""Velocities at separate evaluation points (fmm2d_velocity_targets): the
velocity field of Eq. 7 at points that carry no circulation, as the
single-source experiment of Sec. 5.2 uses (one source, a lattice of
evaluation points; its error maps are the per-point errors returned here).

Bars as in test_gpu_parity: FP64 within 1e-12 of the oracle FMM run on the
particles plus the points as zero-circulation particles, FP32 / FP32_TC
within 1e-6.
"""
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


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _t(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _leaf_xy(x, y, root, L):
    s = 2 ** L / root[2]
    top = 2 ** L - 1
    return (np.clip(np.floor((x - root[0]) * s), 0, top).astype(int),
            np.clip(np.floor((y - root[1]) * s), 0, top).astype(int))


@pytest.mark.parametrize("prec", ["fp64", "fp32_tc"])
def test_single_source_error_map(prec):
    """Sec. 5.2: a unit source at the centre, a 94 x 94 lattice of evaluation
    points, L = 4.  Against the oracle FMM at the same p: 1e-12 (FP64) or 1e-6
    (FP32_TC).  Against the direct sum (the error map): points whose leaf has
    the source in its local list see only rounding (the source is summed
    directly and no other leaf carries circulation); the others see the
    truncation error of the expansions, which falls as p grows."""
    from paper_0809_1810_gb300 import Plan

    dt, npdt = (torch.float64, np.float64) if prec == "fp64" else (torch.float32, np.float32)
    w = W.single_source(n_side=94, sigma=0.02, L=4, dtype=npdt)
    src_xy = np.stack([w.x[:1], w.y[:1]], 1)
    pts = np.stack([w.x[1:], w.y[1:]], 1)
    ref_dir = oracle.direct(w.x, w.y, w.gamma, w.sigma)[1:]
    lx, ly = _leaf_xy(w.x.astype(np.float64), w.y.astype(np.float64), w.root, w.L)
    near = (np.abs(lx[1:] - lx[0]) <= 1) & (np.abs(ly[1:] - ly[0]) <= 1)
    assert near.any() and (~near).any()
    m = np.linalg.norm(ref_dir, axis=1).max()
    prev = None
    for p in (5, 10, 15):
        with Plan(p, w.L, w.sigma, prec, root=w.root, max_n=w.n) as plan:
            uv = plan.velocity_at(_t(src_xy, dt), _t(w.gamma[:1], dt), _t(pts, dt),
                                  check=True).double().cpu().numpy()
        ref = oracle.fmm(w.x, w.y, w.gamma, w.sigma, p, w.L, w.root)[1:]
        assert _rel(uv, ref) <= (1e-12 if prec == "fp64" else 1e-6), (p, _rel(uv, ref))
        err = np.linalg.norm(uv - ref_dir, axis=1) / m
        assert err[near].max() <= (1e-14 if prec == "fp64" else 1e-6), err[near].max()
        far = err[~near].max()
        if prec == "fp64":
            assert far > 1e-14
            if prev is not None:
                assert far < prev, (p, far, prev)
            prev = far


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_tc"])
@pytest.mark.parametrize("cutoff_sigmas", [0.0, 4.6])
def test_points_among_many_particles(prec, cutoff_sigmas):
    """20,000 particles and 5,000 evaluation points, with and without the
    cutoff of Sec. 4.1, against the oracle FMM on the combined set."""
    from paper_0809_1810_gb300 import Plan

    dt, npdt = (torch.float64, np.float64) if prec == "fp64" else (torch.float32, np.float32)
    # leaves of 2.3 sigma: a = 4.6 sigma reaches two leaf widths
    w = W.uniform_random(20000, 61, 2.0 / 141, sigma_over_h=0.95, p=14, L=6, dtype=npdt)
    rng = np.random.Generator(np.random.PCG64(62))
    pts = rng.uniform(-1.0, 1.0, (5000, 2)).astype(npdt)
    a = cutoff_sigmas * w.sigma
    with Plan(w.p, w.L, w.sigma, prec, root=w.root, max_n=w.n + len(pts), cutoff=a) as plan:
        uv = plan.velocity_at(_t(np.stack([w.x, w.y], 1), dt), _t(w.gamma, dt), _t(pts, dt),
                              check=True).double().cpu().numpy()
    x = np.concatenate([w.x, pts[:, 0]])
    y = np.concatenate([w.y, pts[:, 1]])
    g = np.concatenate([w.gamma, np.zeros(len(pts), npdt)])
    ref = oracle.fmm(x, y, g, w.sigma, w.p, w.L, w.root, a=a)[w.n:]
    assert _rel(uv, ref) <= (1e-12 if prec == "fp64" else 1e-6), _rel(uv, ref)


def test_points_at_particles_see_the_particle_velocities():
    """An evaluation point on a particle gets K_sigma(0) = 0 from it: the
    velocity there is the particle's own (Eq. 9), up to the rounding of the
    other tree the points make."""
    from paper_0809_1810_gb300 import Plan

    w = W.uniform_random(8000, 63, 2.0 / 89, sigma_over_h=1.5, p=16, L=5, dtype=np.float64)
    xy = _t(np.stack([w.x, w.y], 1), torch.float64)
    g = _t(w.gamma, torch.float64)
    idx = np.arange(0, w.n, 7)
    with Plan(w.p, w.L, w.sigma, "fp64", root=w.root, max_n=w.n + len(idx)) as plan:
        own = plan.velocity(xy, g, check=True).cpu().numpy()[idx]
        at = plan.velocity_at(xy, g, xy[torch.tensor(idx, device="cuda")], check=True)
    assert _rel(at.cpu().numpy(), own) <= 1e-12


def test_targets_need_room_in_the_plan():
    from paper_0809_1810_gb300 import FMMError, Plan

    w = W.uniform_random(1000, 64, 0.06, p=6, L=3, dtype=np.float32)
    xy = _t(np.stack([w.x, w.y], 1), torch.float32)
    g = _t(w.gamma, torch.float32)
    with Plan(w.p, w.L, w.sigma, "fp32", root=w.root, max_n=1200) as plan:
        with pytest.raises(FMMError):
            plan.velocity_at(xy, g, xy[:201])
        plan.velocity_at(xy, g, xy[:200], check=True)  # n + m = max_n fits
