"""GB300-native 2D vortex-particle FMM (Cruz & Barba 2008) -- Python binding.

The computation lives in libfmm2d (hand-written CUDA for sm_103a behind the C
ABI of include/fmm2d.h).  This module only marshals torch tensors (device
memory and the current CUDA stream) into those calls.

    plan = Plan(p=16, L=7, sigma=2 * h, precision="fp32")
    uv = plan.velocity(xy, gamma)          # xy (n, 2), gamma (n,) on cuda:0

Everything raises :class:`FMMError` on a non-OK status.
"""
from __future__ import annotations

import ctypes

import torch

from . import _native
from ._native import FP32, FP32_TC, FP64, NUM_PHASES, PHASES

__all__ = ["Plan", "BatchPlan", "FMMError", "FP64", "FP32", "FP32_TC", "PHASES", "library",
           "cutoff_for"]

_PREC = {"fp64": FP64, "fp32": FP32, "fp32_tc": FP32_TC}


class FMMError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = _native.load()
        name = lib.fmm2d_status_string(status).decode()
        if where.startswith("batch"):
            getter = lib.fmm2d_batch_last_error
        elif where.startswith(("mlp", "features", "propose")):
            getter = lib.fmm2d_mlp_last_error
        else:
            getter = lib.fmm2d_last_error
        detail = getter().decode()
        super().__init__(f"{where}: {name} ({detail})" if detail else f"{where}: {name}")
        self.status = status


def cutoff_for(sigma: float, leaf: float, tol: float) -> float:
    """The cutoff a of Sec. 4.1 for a relative tolerance: a pair left on the
    singular kernel (r >= a) differs from the regularised one by
    |K_sigma - K'| / |K'| = exp(-r^2 / 2 sigma^2) <= exp(-a^2 / 2 sigma^2) = tol
    (Eq. 29 pair by pair), so a = sigma sqrt(2 ln(1/tol)).  0 when the leaves
    are at least that wide (no non-neighbour pair is closer); at most two leaf
    widths, the reach of the kernels' ring."""
    import math

    a = sigma * math.sqrt(2.0 * math.log(1.0 / tol))
    if leaf >= a:
        return 0.0
    return min(a, 2.0 * leaf)


def library():
    """The loaded ctypes library (built in-tree on first use)."""
    return _native.load()


def _check(status: int, where: str):
    if status != _native.OK:
        raise FMMError(status, where)


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr() if t is not None else 0)


class Plan:
    """An FMM configuration (p, L, sigma, precision, root box, cutoff) and its
    device workspace for up to ``max_n`` particles (fmm2d_plan_create).
    ``cutoff`` is the distance a of Sec. 4.1: pairs closer than a keep the
    regularised kernel even outside the 3x3 leaf neighbourhood (0: off; at
    most two leaf widths)."""

    def __init__(self, p: int, L: int, sigma: float, precision="fp32",
                 root=(-1.0, -1.0, 2.0), max_n: int = 1 << 20, cutoff: float = 0.0):
        self._lib = _native.load()
        self.p, self.L, self.sigma = int(p), int(L), float(sigma)
        self.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
        self.dtype = torch.float64 if self.precision == FP64 else torch.float32
        self.root = tuple(float(v) for v in root)
        self.max_n = int(max_n)
        self.cutoff = float(cutoff)
        prm = _native.Params(self.p, self.L, self.sigma, self.precision, self.root[0],
                             self.root[1], self.root[2], self.max_n, self.cutoff)
        h = ctypes.c_void_p()
        _check(self._lib.fmm2d_plan_create(ctypes.byref(h), ctypes.byref(prm)), "plan_create")
        self._h = h

    # -- lifetime ----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.fmm2d_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- helpers -----------------------------------------------------------
    def _inputs(self, xy, gamma):
        if xy.dtype != self.dtype or gamma.dtype != self.dtype:
            raise TypeError(f"inputs must be {self.dtype}")
        if not (xy.is_cuda and gamma.is_cuda):
            raise TypeError("inputs must be CUDA tensors")
        xy = xy.contiguous()
        gamma = gamma.contiguous()
        n = gamma.shape[0]
        if xy.numel() != 2 * n:
            raise ValueError("xy must hold 2 n values")
        return xy, gamma, n

    # -- the FMM -------------------------------------------------------------
    def velocity(self, xy, gamma, out=None, stream=None, check=False):
        """Velocities (n, 2) at the particles (fmm2d_velocity)."""
        xy, gamma, n = self._inputs(xy, gamma)
        if out is None:
            out = torch.empty((n, 2), dtype=self.dtype, device=xy.device)
        _check(self._lib.fmm2d_velocity(self._h, n, _ptr(xy), _ptr(gamma), _ptr(out),
                                        _stream(stream)), "velocity")
        if check:
            self.check(stream)
        return out

    def velocity_at(self, xy, gamma, targets, out=None, stream=None, check=False):
        """Velocities (m, 2) at m points `targets` (m, 2) that carry no
        circulation, induced by the particles (fmm2d_velocity_targets)."""
        xy, gamma, n = self._inputs(xy, gamma)
        if targets.dtype != self.dtype or not targets.is_cuda:
            raise TypeError(f"targets must be {self.dtype} CUDA tensors")
        targets = targets.contiguous()
        m = targets.numel() // 2
        if targets.numel() != 2 * m:
            raise ValueError("targets must hold 2 m values")
        if out is None:
            out = torch.empty((m, 2), dtype=self.dtype, device=xy.device)
        _check(self._lib.fmm2d_velocity_targets(self._h, n, _ptr(xy), _ptr(gamma), m,
                                                _ptr(targets), _ptr(out), _stream(stream)),
               "velocity_targets")
        if check:
            self.check(stream)
        return out

    def convect(self, xy, gamma, dt: float, order: int = 2, stream=None, check=False):
        """One convection step of Eq. 5 in place (fmm2d_convect): forward
        Euler (order 1) or Heun (order 2) on the FMM velocities.  xy must be
        a contiguous CUDA tensor of the plan dtype; it holds the new
        positions afterwards."""
        if not xy.is_contiguous():
            raise ValueError("xy must be contiguous (it is updated in place)")
        _, gamma, n = self._inputs(xy, gamma)
        _check(self._lib.fmm2d_convect(self._h, n, _ptr(xy), _ptr(gamma), float(dt), int(order),
                                       _stream(stream)), "convect")
        if check:
            self.check(stream)
        return xy

    def velocity_host(self, xy, gamma, out, stream=None):
        """Host-buffer form (fmm2d_velocity_host): xy, gamma, out are CPU
        tensors (page-locked for asynchronous copies); synchronous."""
        n = gamma.shape[0]
        for t in (xy, gamma, out):
            if t.is_cuda or t.dtype != self.dtype or not t.is_contiguous():
                raise TypeError("host tensors of the plan dtype, contiguous")
        _check(self._lib.fmm2d_velocity_host(self._h, n, _ptr(xy), _ptr(gamma), _ptr(out),
                                             _stream(stream)), "velocity_host")
        return out

    def velocity_host_many(self, xys, gammas, outs, stream=None):
        """count independent sets from host buffers, pipelined
        (fmm2d_velocity_host_many): xys[k], gammas[k], outs[k] are CPU tensors
        of set k (page-locked for the copies to overlap), all sets of the
        same size; synchronous."""
        count = len(xys)
        if len(gammas) != count or len(outs) != count:
            raise ValueError("xys, gammas and outs must have the same length")
        n = gammas[0].shape[0] if count else 0
        for t in list(xys) + list(gammas) + list(outs):
            if t.is_cuda or t.dtype != self.dtype or not t.is_contiguous():
                raise TypeError("host tensors of the plan dtype, contiguous")
        for k in range(count):
            if gammas[k].shape[0] != n or tuple(xys[k].shape) != (n, 2) or \
                    tuple(outs[k].shape) != (n, 2):
                raise ValueError("every set must hold the same number of particles")
        arr = ctypes.c_void_p * max(count, 1)
        pxy = arr(*[_ptr(t) for t in xys])
        pg = arr(*[_ptr(t) for t in gammas])
        pout = arr(*[_ptr(t) for t in outs])
        _check(self._lib.fmm2d_velocity_host_many(self._h, count, n, pxy, pg, pout,
                                                  _stream(stream)), "velocity_host_many")
        return outs

    def check(self, stream=None):
        """Raise if the device recorded an input error (fmm2d_plan_check)."""
        _check(self._lib.fmm2d_plan_check(self._h, _stream(stream)), "plan_check")

    def tree(self, n, stream=None):
        """(sorted keys, permutation, leaf_start) of the last evaluation."""
        dev = torch.device("cuda", torch.cuda.current_device())
        keys = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        perm = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        start = torch.empty((1 << (2 * self.L)) + 1, dtype=torch.int32, device=dev)
        _check(self._lib.fmm2d_tree_debug(self._h, _ptr(keys), _ptr(perm), _ptr(start),
                                          _stream(stream)), "tree_debug")
        return keys[:n], perm[:n], start

    # -- yardsticks ----------------------------------------------------------
    def direct_sampled(self, xy, gamma, targets, kernel=0, stream=None):
        """FP64 direct velocities (s, 2) at sampled particle indices:
        kernel 0 regularised everywhere, 1 the FMM's hybrid limit."""
        xy, gamma, n = self._inputs(xy, gamma)
        targets = targets.to(device=xy.device, dtype=torch.int64).contiguous()
        out = torch.empty((targets.shape[0], 2), dtype=torch.float64, device=xy.device)
        _check(self._lib.fmm2d_direct_sampled(self._h, int(kernel), n, _ptr(xy), _ptr(gamma),
                                              targets.shape[0], _ptr(targets), _ptr(out),
                                              _stream(stream)), "direct_sampled")
        return out

    def error_stats(self, xy, uv, targets, uv_ref, per_leaf=False, stream=None):
        """(max|du|, max|u_ref|, sum|du|^2, sum|u_ref|^2) as a float64 device
        tensor, plus per-leaf max |du| when per_leaf is set."""
        n = uv.shape[0]
        targets = targets.to(device=uv.device, dtype=torch.int64).contiguous()
        stats = torch.empty(4, dtype=torch.float64, device=uv.device)
        leaf = (torch.empty(1 << (2 * self.L), dtype=torch.float64, device=uv.device)
                if per_leaf else None)
        _check(self._lib.fmm2d_error_stats(self._h, n, _ptr(xy.contiguous()),
                                           _ptr(uv.contiguous()), targets.shape[0],
                                           _ptr(targets), _ptr(uv_ref.contiguous()), _ptr(stats),
                                           _ptr(leaf), _stream(stream)), "error_stats")
        return (stats, leaf) if per_leaf else stats

    # -- tracing ---------------------------------------------------------------
    def set_timing(self, ring: int):
        _check(self._lib.fmm2d_plan_set_timing(self._h, int(ring)), "set_timing")

    def kernels_per_call(self) -> int:
        """Kernel launches one velocity call makes (-1 before the first)."""
        return int(self._lib.fmm2d_plan_kernels_per_call(self._h))

    def multipole_reals(self) -> int:
        """Length of the plan's multipole array (fmm2d_plan_multipole_reals)."""
        return int(self._lib.fmm2d_plan_multipole_reals(self._h))

    def multipoles(self, xy, gamma, out=None, stream=None):
        """Multipoles of every box from these particles (tree, P2M, M2M)."""
        n = xy.shape[0]
        if out is None:
            out = torch.zeros(max(self.multipole_reals(), 1), dtype=xy.dtype, device=xy.device)
        _check(self._lib.fmm2d_multipoles(self._h, n, _ptr(xy), _ptr(gamma), _ptr(out),
                                          _stream(stream)), "multipoles")
        return out

    def velocity_from_multipoles(self, xy, gamma, me, out=None, stream=None):
        """The evaluation with P2M and M2M replaced by the given multipoles."""
        n = xy.shape[0]
        if out is None:
            out = torch.empty((n, 2), dtype=xy.dtype, device=xy.device)
        _check(self._lib.fmm2d_velocity_from_multipoles(self._h, n, _ptr(xy), _ptr(gamma),
                                                        _ptr(me), _ptr(out), _stream(stream)),
               "velocity_from_multipoles")
        return out

    def set_spin_limit(self, polls: int):
        """Poll limit of the tensor-core M2L's device waits (0: the default);
        a small limit makes them run out (FMM2D_TIMEOUT at the next check)."""
        _check(self._lib.fmm2d_plan_set_spin_limit(self._h, int(polls)), "set_spin_limit")

    def set_ring_strips(self, enable: bool):
        """Gather the FP32 near field's cutoff ring from per-side strips of
        the ring leaves (True, the default) or from the whole leaves."""
        _check(self._lib.fmm2d_plan_set_ring_strips(self._h, 1 if enable else 0),
               "set_ring_strips")

    def phase_ms(self, age: int = 0):
        buf = (ctypes.c_double * NUM_PHASES)()
        _check(self._lib.fmm2d_plan_phase_ms(self._h, int(age), buf), "phase_ms")
        return dict(zip(PHASES, list(buf)))


class BatchPlan:
    """Many independent instances evaluated together (fmm2d_batch_*): FP32
    or FP32_TC (``precision``), one CUDA graph per call.  ``instances`` is a
    list of dicts with keys n, p, L, sigma and optionally root=(x0, y0, W) and
    cutoff (the distance a of Sec. 4.1, 0 by default)."""

    def __init__(self, instances, precision="fp32"):
        self._lib = _native.load()
        arr = (_native.Instance * len(instances))()
        for k, d in enumerate(instances):
            root = d.get("root", (-1.0, -1.0, 2.0))
            arr[k] = _native.Instance(int(d["n"]), int(d["p"]), int(d["L"]), float(d["sigma"]),
                                      float(root[0]), float(root[1]), float(root[2]),
                                      float(d.get("cutoff", 0.0)))
        self.precision = precision
        self.instances = [dict(d) for d in instances]
        self.offsets = [0]
        for d in instances:
            self.offsets.append(self.offsets[-1] + int(d["n"]))
        h = ctypes.c_void_p()
        _check(self._lib.fmm2d_batch_plan_create_ex(ctypes.byref(h), len(instances), arr,
                                                    _PREC[precision]), "batch_plan_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.fmm2d_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def n_total(self) -> int:
        return self.offsets[-1]

    def velocity(self, xy, gamma, out=None, stream=None):
        if xy.dtype != torch.float32 or gamma.dtype != torch.float32 or not xy.is_cuda:
            raise TypeError("float32 CUDA tensors")
        if gamma.shape[0] != self.n_total:
            raise ValueError("packed arrays must hold every instance")
        if out is None:
            out = torch.empty((self.n_total, 2), dtype=torch.float32, device=xy.device)
        _check(self._lib.fmm2d_batch_velocity(self._h, _ptr(xy.contiguous()),
                                              _ptr(gamma.contiguous()), _ptr(out),
                                              _stream(stream)), "batch_velocity")
        return out

    def check(self, stream=None):
        _check(self._lib.fmm2d_batch_check(self._h, _stream(stream)), "batch_check")

    def autotune(self, xy, gamma, out, stream=None):
        _check(self._lib.fmm2d_batch_autotune(self._h, _ptr(xy), _ptr(gamma), _ptr(out),
                                              _stream(stream)), "batch_autotune")
        return self.info()

    def info(self):
        n = ctypes.c_int64()
        leaves = ctypes.c_int64()
        k = ctypes.c_int()
        cps = ctypes.c_int()
        th = ctypes.c_int()
        _check(self._lib.fmm2d_batch_info(self._h, ctypes.byref(n), ctypes.byref(leaves),
                                          ctypes.byref(k), ctypes.byref(cps), ctypes.byref(th)),
               "batch_info")
        cls = ctypes.c_int()
        tiles = ctypes.c_int()
        st = ctypes.c_int()
        pol = ctypes.c_int()
        _check(self._lib.fmm2d_batch_info_tc(self._h, ctypes.byref(cls), ctypes.byref(tiles),
                                             ctypes.byref(st), ctypes.byref(pol)),
               "batch_info_tc")
        return {"n_total": n.value, "leaves_total": leaves.value, "kernels_per_call": k.value,
                "p2p_ctas_per_sm": cps.value, "m2l_threads": th.value,
                "precision": self.precision, "tc_classes": cls.value, "tc_tiles": tiles.value,
                "tc_b_stages": st.value, "tc_tile_policy": pol.value}

    def profile(self, xy, gamma, out, stream=None):
        """Phase durations (ms) of one evaluation run step by step."""
        buf = (ctypes.c_double * 5)()
        _check(self._lib.fmm2d_batch_profile(self._h, _ptr(xy), _ptr(gamma), _ptr(out), buf,
                                             _stream(stream)), "batch_profile")
        return dict(zip(("tree", "upward", "m2l", "l2l", "near"), list(buf)))

    def direct_sampled(self, xy, gamma, targets, kernel=0, stream=None):
        targets = targets.to(device=xy.device, dtype=torch.int64).contiguous()
        out = torch.empty((targets.shape[0], 2), dtype=torch.float64, device=xy.device)
        _check(self._lib.fmm2d_batch_direct_sampled(self._h, int(kernel), _ptr(xy), _ptr(gamma),
                                                    targets.shape[0], _ptr(targets), _ptr(out),
                                                    _stream(stream)), "batch_direct_sampled")
        return out

    def error_stats(self, xy, uv, targets, uv_ref, per_leaf=False, stream=None):
        """(count, 4) float64: max|du|, max|u_ref|, sum|du|^2, sum|u_ref|^2 per
        instance; plus per-leaf max |du| (global leaf order) when asked."""
        targets = targets.to(device=uv.device, dtype=torch.int64).contiguous()
        stats = torch.empty((len(self.instances), 4), dtype=torch.float64, device=uv.device)
        leaf = None
        if per_leaf:
            nleaf = sum(1 << (2 * int(d["L"])) for d in self.instances)
            leaf = torch.empty(nleaf, dtype=torch.float64, device=uv.device)
        _check(self._lib.fmm2d_batch_error_stats(self._h, _ptr(xy), _ptr(uv), targets.shape[0],
                                                 _ptr(targets), _ptr(uv_ref.contiguous()),
                                                 _ptr(stats), _ptr(leaf), _stream(stream)),
               "batch_error_stats")
        return (stats, leaf) if per_leaf else stats
