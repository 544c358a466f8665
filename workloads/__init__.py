"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the oracle side and the CUDA side of every test and
of the benchmark, and holds none of the FMM's arithmetic: it only draws
particle positions and circulations.  Every draw uses numpy's PCG64 generator
with an explicit seed, so both sides see identical bits.

Workloads (root box [-1, 1]^2 throughout, the reading adopted for the paper's
unstated root box):

* :func:`lamb_oseen_lattice` -- the Lamb-Oseen setup of Sec. 5.1: a cell-centred
  square lattice with spacing h whose circulations sample the vorticity of
  Eq. 32, Gamma_j = h^2 Gamma0 / (4 pi nu t) exp(-r_j^2 / (4 nu t)).
* :func:`uniform_random` -- uniform positions, signed circulations h^2 N(0,1):
  the mixed-sign case the paper singles out in Sec. 1.
* :func:`clustered_patches` -- a mixture of Gaussian patches with signed
  patch circulations, giving uneven leaf occupancy.
* :func:`single_source` -- the single-source problem of Sec. 5.2: one unit
  source at the centre and zero-circulation lattice points as evaluation points.
* :func:`batch_instances` -- a sweep of many small instances of uneven N, p
  and L, like the paper's parameter study of about 1000 runs (Sec. 5).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ROOT = (-1.0, -1.0, 2.0)  # (x0, y0, W): the square [-1, 1]^2


@dataclass
class Workload:
    name: str
    x: np.ndarray
    y: np.ndarray
    gamma: np.ndarray
    sigma: float
    p: int
    L: int
    h: float
    root: tuple = ROOT
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def dtype(self):
        return self.x.dtype


def lattice_coords(n_side: int, root=ROOT):
    """Cell-centred lattice x_i = x0 + (i + 1/2) h, h = W / n_side (row-major)."""
    x0, y0, W = root
    h = W / n_side
    c = (np.arange(n_side, dtype=np.float64) + 0.5) * h
    gx, gy = np.meshgrid(x0 + c, y0 + c, indexing="xy")
    return gx.ravel(), gy.ravel(), h


def lamb_oseen_lattice(n_side: int, nu_t: float = 0.05, gamma0: float = 1.0,
                       sigma_over_h: float = 1.0, p: int = 10, L: int = 3,
                       dtype=np.float64) -> Workload:
    x, y, h = lattice_coords(n_side)
    r2 = x * x + y * y
    g = h * h * gamma0 / (4.0 * math.pi * nu_t) * np.exp(-r2 / (4.0 * nu_t))
    return Workload(f"lamb_oseen_{n_side}x{n_side}", x.astype(dtype), y.astype(dtype),
                    g.astype(dtype), sigma_over_h * h, p, L, h,
                    extra={"nu_t": nu_t, "gamma0": gamma0})


def lamb_oseen_fixed_spacing(n_side: int, h: float = 0.016, sigma: float = 0.02,
                             nu_t: float = 0.0005 * 4, gamma0: float = 1.0, p: int = 13,
                             L: int = 4, dtype=np.float64) -> Workload:
    """The Lamb-Oseen setup of Sec. 5.1 at a fixed lattice spacing: sigma =
    0.02, h / sigma = 0.8, nu = 0.0005, t = 4; the square domain grows with
    the particle count (side n_side h, centred on the vortex), as in the
    domain-size series of Fig. 19 (63^2, 88^2, 138^2 particles).  The root box
    is the domain."""
    side = n_side * h
    root = (-0.5 * side, -0.5 * side, side)
    x, y, _ = lattice_coords(n_side, root)
    r2 = x * x + y * y
    g = h * h * gamma0 / (4.0 * math.pi * nu_t) * np.exp(-r2 / (4.0 * nu_t))
    return Workload(f"lamb_oseen_{n_side}x{n_side}_h{h:g}", x.astype(dtype), y.astype(dtype),
                    g.astype(dtype), sigma, p, L, h, root=root,
                    extra={"nu_t": nu_t, "gamma0": gamma0})


def uniform_random(n: int, seed: int, h: float, sigma_over_h: float = 2.0, p: int = 16,
                   L: int = 7, dtype=np.float32) -> Workload:
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.uniform(-1.0, 1.0, n).astype(dtype)
    y = rng.uniform(-1.0, 1.0, n).astype(dtype)
    g = (h * h * rng.standard_normal(n)).astype(dtype)
    return Workload(f"uniform_{n}", x, y, g, sigma_over_h * h, p, L, h)


def clustered_patches(n: int, seed: int, npatch: int = 64, h: float = 2.0 / 4096,
                      sigma_over_h: float = 1.0, p: int = 20, L: int = 9,
                      std_range=(0.02, 0.2), centre_range=(-0.8, 0.8),
                      dtype=np.float32) -> Workload:
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.uniform(centre_range[0], centre_range[1], (npatch, 2))
    stds = np.exp(rng.uniform(math.log(std_range[0]), math.log(std_range[1]), npatch))
    strength = rng.standard_normal(npatch)
    counts = np.full(npatch, n // npatch)
    counts[: n - counts.sum()] += 1
    xs, ys, gs = [], [], []
    for k in range(npatch):
        m = int(counts[k])
        px = np.empty(m)
        py = np.empty(m)
        todo = np.arange(m)
        while todo.size:  # resample points that fall outside the root box
            px[todo] = rng.normal(centres[k, 0], stds[k], todo.size)
            py[todo] = rng.normal(centres[k, 1], stds[k], todo.size)
            bad = (np.abs(px[todo]) >= 1.0) | (np.abs(py[todo]) >= 1.0)
            todo = todo[bad]
        xs.append(px)
        ys.append(py)
        gs.append(np.full(m, strength[k] * h * h))
    x = np.concatenate(xs).astype(dtype)
    y = np.concatenate(ys).astype(dtype)
    g = np.concatenate(gs).astype(dtype)
    return Workload(f"clustered_{n}", x, y, g, sigma_over_h * h, p, L, h,
                    extra={"npatch": npatch})


def single_source(n_side: int = 94, sigma: float = 0.02, p: int = 13, L: int = 4,
                  dtype=np.float64) -> Workload:
    """Sec. 5.2: unit source at the domain centre plus zero-circulation lattice
    points that serve as evaluation points (the source is particle 0)."""
    x, y, h = lattice_coords(n_side)
    x = np.concatenate([[0.0], x])
    y = np.concatenate([[0.0], y])
    g = np.zeros_like(x)
    g[0] = 1.0
    return Workload(f"single_source_{n_side}", x.astype(dtype), y.astype(dtype),
                    g.astype(dtype), sigma, p, L, h)


def sample_targets(n: int, s: int, seed: int) -> np.ndarray:
    """s distinct particle indices, sorted, drawn with a fixed seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = min(s, n)
    return np.sort(rng.choice(n, size=s, replace=False)).astype(np.int64)


# --- the named workloads ---------------------------------------------------

def lamb_oseen_4096() -> Workload:
    """N = 4096 lattice (64 x 64, h = 2/64), sigma = h, nu t = 0.05, p = 10, L = 3."""
    return lamb_oseen_lattice(64, nu_t=0.05, sigma_over_h=1.0, p=10, L=3)


def uniform_1m(seed: int = 2) -> Workload:
    """N = 2^20 uniform, h = 2/1024, sigma = 2h, p = 16, L = 7, float32."""
    return uniform_random(1 << 20, seed, 2.0 / 1024, sigma_over_h=2.0, p=16, L=7)


def clustered_16m(seed: int = 5) -> Workload:
    """N = 2^24 from 64 Gaussian patches, h = 2/4096, sigma = h, p = 20, L = 9."""
    return clustered_patches(1 << 24, seed)


@dataclass
class InstanceSpec:
    index: int
    n: int
    p: int
    L: int
    sigma_over_h: float
    kind: str  # "lamb_oseen" or "uniform"
    seed: int


def batch_instances(count: int = 512, seed: int = 3, log2n=(12.0, 17.0)):
    """Instance descriptors of the batched sweep: N = floor(2^U(12,17)),
    p in {4, 6, ..., 24}, L in {3..7}, sigma/h in {0.8, 1, 1.5, 2}; even
    indices are Lamb-Oseen lattices (N rounded to a square), odd ones uniform."""
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for i in range(count):
        n = int(math.floor(2.0 ** rng.uniform(*log2n)))
        p = int(rng.choice(np.arange(4, 25, 2)))
        L = int(rng.integers(3, 8))
        soh = float(rng.choice([0.8, 1.0, 1.5, 2.0]))
        kind = "lamb_oseen" if i % 2 == 0 else "uniform"
        if kind == "lamb_oseen":
            side = max(2, int(round(math.sqrt(n))))
            n = side * side
        specs.append(InstanceSpec(i, n, p, L, soh, kind, seed * 100003 + i))
    return specs


def make_instance(spec: InstanceSpec, dtype=np.float32) -> Workload:
    if spec.kind == "lamb_oseen":
        side = int(round(math.sqrt(spec.n)))
        w = lamb_oseen_lattice(side, nu_t=0.05, sigma_over_h=spec.sigma_over_h, p=spec.p,
                               L=spec.L, dtype=dtype)
    else:
        h = 2.0 / math.sqrt(spec.n)
        w = uniform_random(spec.n, spec.seed, h, sigma_over_h=spec.sigma_over_h, p=spec.p,
                           L=spec.L, dtype=dtype)
    w.name = f"instance_{spec.index}_{w.name}"
    return w
