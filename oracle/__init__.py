"""CPU FP64 oracle for the 2D vortex-particle FMM (Cruz & Barba 2008).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import this package.  The CUDA library
never does, and this package never imports the CUDA library: the two share no
code.  The arithmetic lives in ``fmm2d_oracle.c`` (plain C, double precision);
this module only compiles it with gcc and marshals numpy arrays through ctypes.

Functions and the paper passage each follows:

* :func:`morton_keys`, :func:`sort_by_key` -- uniform quadtree, Sec. 3.3 / Fig. 6.
* :func:`direct` -- O1, the discrete Biot-Savart sum of Eq. 7 with Eq. 6 and
  the self term excluded (Eq. 9).
* :func:`hybrid` -- O2, regularised kernel inside the 3x3 leaf neighbourhood
  (and, with a cutoff a > 0, for every pair closer than a: Sec. 4.1, Eq. 29),
  singular kernel (Eq. 27) elsewhere: the FMM's limit as p grows (Eq. 10).
* :func:`fmm` -- O3, the plain FMM in the order of Sec. 3.1 / Fig. 3, with the
  same optional cutoff.
* ``op_*`` -- single expansions and translations: Eqs. 20-22, Secs. 3.3.2-3.3.3.
* :func:`convect` -- one convection step of Eq. 5 (forward Euler or Heun)
  on a given velocity function.
* :func:`kernel_error_estimate` -- Eq. 29 (squared-distance reading).
* :func:`truncation_bound` -- Eqs. 30-31 (geometric-tail reading).

Every function is pinned by a ``-m "not gpu"`` test against something other
than itself (closed forms, the Lamb-Oseen vortex, exact invariants, Table 1).
Parity unpinned: Table 1 levels 4-5 (not reproducible under any reading).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm2d_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

OK, INVALID_ARG, OUT_OF_DOMAIN, NONFINITE = 0, 1, 2, 3

_lib = None
_lock = threading.Lock()


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, OpenMP on)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        d, i64, i32, vp = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        lib.orc_num_threads.restype = i32
        lib.orc_morton_keys.argtypes = [i64, vp, vp, d, d, d, i32, vp]
        lib.orc_morton_keys.restype = i32
        lib.orc_sort_by_key.argtypes = [i64, vp, i32, vp, vp]
        lib.orc_sort_by_key.restype = None
        lib.orc_direct.argtypes = [i64, vp, vp, vp, d, i64, vp, vp, vp]
        lib.orc_direct.restype = i32
        lib.orc_hybrid.argtypes = [i64, vp, vp, vp, d, d, d, d, i32, i64, vp, vp, vp]
        lib.orc_hybrid.restype = i32
        lib.orc_fmm.argtypes = [i64, vp, vp, vp, d, i32, i32, d, d, d, vp, vp]
        lib.orc_fmm.restype = i32
        lib.orc_hybrid_cut.argtypes = [i64, vp, vp, vp, d, d, d, d, i32, d, i64, vp, vp, vp]
        lib.orc_hybrid_cut.restype = i32
        lib.orc_fmm_cut.argtypes = [i64, vp, vp, vp, d, i32, i32, d, d, d, d, vp, vp]
        lib.orc_fmm_cut.restype = i32
        lib.orc_op_p2m.argtypes = [i64, vp, vp, vp, d, d, i32, vp]
        lib.orc_op_m2m.argtypes = [i32, vp, d, d, d, d, vp]
        lib.orc_op_m2l.argtypes = [i32, vp, d, d, d, d, vp]
        lib.orc_op_l2l.argtypes = [i32, vp, d, d, d, d, vp]
        lib.orc_op_l2p.argtypes = [i32, vp, d, d, i64, vp, vp, vp]
        lib.orc_op_me_eval.argtypes = [i32, vp, d, d, i64, vp, vp, vp]
        for f in ("orc_op_p2m", "orc_op_m2m", "orc_op_m2l", "orc_op_l2l", "orc_op_l2p",
                  "orc_op_me_eval"):
            getattr(lib, f).restype = None
        lib.orc_kernel_error_estimate.argtypes = [d, d, d]
        lib.orc_kernel_error_estimate.restype = d
        lib.orc_truncation_bound.argtypes = [d, d, i32, d]
        lib.orc_truncation_bound.restype = d
        _lib = lib
        return lib


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(status, what):
    if status != OK:
        names = {INVALID_ARG: "invalid argument", OUT_OF_DOMAIN: "point outside root box",
                 NONFINITE: "non-finite input"}
        raise OracleError(f"{what}: {names.get(status, status)}")


def num_threads() -> int:
    """Threads the oracle's OpenMP loops use."""
    return int(_load().orc_num_threads())


def morton_keys(x, y, root, L):
    """Leaf Morton keys (x index in even bits, y in odd) at level L."""
    lib = _load()
    x, y = _f64(x), _f64(y)
    key = np.empty(x.shape[0], dtype=np.uint32)
    _check(lib.orc_morton_keys(x.shape[0], _ptr(x), _ptr(y), root[0], root[1], root[2], L,
                               _ptr(key)), "morton_keys")
    return key


def sort_by_key(key, L):
    """Stable counting sort: (perm, leaf_start[4^L + 1])."""
    lib = _load()
    key = np.ascontiguousarray(key, dtype=np.uint32)
    perm = np.empty(key.shape[0], dtype=np.uint32)
    start = np.empty((1 << (2 * L)) + 1, dtype=np.uint32)
    lib.orc_sort_by_key(key.shape[0], _ptr(key), L, _ptr(perm), _ptr(start))
    return perm, start


def _targets(n, targets):
    if targets is None:
        return np.arange(n, dtype=np.int64)
    return np.ascontiguousarray(targets, dtype=np.int64)


def direct(x, y, gamma, sigma, targets=None):
    """O1: regularised direct sum at the given particle indices -> (m, 2)."""
    lib = _load()
    x, y, g = _f64(x), _f64(y), _f64(gamma)
    t = _targets(x.shape[0], targets)
    u = np.empty(t.shape[0])
    v = np.empty(t.shape[0])
    _check(lib.orc_direct(x.shape[0], _ptr(x), _ptr(y), _ptr(g), sigma, t.shape[0], _ptr(t),
                          _ptr(u), _ptr(v)), "direct")
    return np.stack([u, v], axis=1)


def hybrid(x, y, gamma, sigma, root, L, targets=None, a=0.0):
    """O2: regularised kernel in the 3x3 leaf neighbourhood and for every pair
    closer than the cutoff a (Sec. 4.1), singular elsewhere."""
    lib = _load()
    x, y, g = _f64(x), _f64(y), _f64(gamma)
    t = _targets(x.shape[0], targets)
    u = np.empty(t.shape[0])
    v = np.empty(t.shape[0])
    if a == 0.0:
        st = lib.orc_hybrid(x.shape[0], _ptr(x), _ptr(y), _ptr(g), sigma, root[0], root[1],
                            root[2], L, t.shape[0], _ptr(t), _ptr(u), _ptr(v))
    else:
        st = lib.orc_hybrid_cut(x.shape[0], _ptr(x), _ptr(y), _ptr(g), sigma, root[0], root[1],
                                root[2], L, float(a), t.shape[0], _ptr(t), _ptr(u), _ptr(v))
    _check(st, "hybrid")
    return np.stack([u, v], axis=1)


def fmm(x, y, gamma, sigma, p, L, root, a=0.0):
    """O3: plain FP64 FMM velocity at every particle -> (n, 2); with a > 0,
    pairs closer than a in non-neighbour leaves keep the regularised kernel
    (Sec. 4.1)."""
    lib = _load()
    x, y, g = _f64(x), _f64(y), _f64(gamma)
    n = x.shape[0]
    u = np.empty(n)
    v = np.empty(n)
    if a == 0.0:
        st = lib.orc_fmm(n, _ptr(x), _ptr(y), _ptr(g), sigma, p, L, root[0], root[1], root[2],
                         _ptr(u), _ptr(v))
    else:
        st = lib.orc_fmm_cut(n, _ptr(x), _ptr(y), _ptr(g), sigma, p, L, root[0], root[1],
                             root[2], float(a), _ptr(u), _ptr(v))
    _check(st, "fmm")
    return np.stack([u, v], axis=1)


def _cplx(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    return a.view(np.float64)


def op_p2m(x, y, gamma, centre, p):
    """ME coefficients a_m (complex, length p) of the given particles (Eq. 20)."""
    lib = _load()
    x, y, g = _f64(x), _f64(y), _f64(gamma)
    out = np.zeros(2 * p)
    lib.orc_op_p2m(x.shape[0], _ptr(x), _ptr(y), _ptr(g), centre[0], centre[1], p, _ptr(out))
    return out.view(np.complex128).copy()


def _op2(fn, p, coeffs, c_from, c_to):
    a = _cplx(coeffs)
    out = np.zeros(2 * p)
    fn(p, _ptr(a), c_from[0], c_from[1], c_to[0], c_to[1], _ptr(out))
    return out.view(np.complex128).copy()


def op_m2m(a, child_centre, parent_centre):
    return _op2(_load().orc_op_m2m, len(a), a, child_centre, parent_centre)


def op_m2l(a, source_centre, target_centre):
    return _op2(_load().orc_op_m2l, len(a), a, source_centre, target_centre)


def op_l2l(coeffs, parent_centre, child_centre):
    return _op2(_load().orc_op_l2l, len(coeffs), coeffs, parent_centre, child_centre)


def _eval(fn, coeffs, centre, yx, yy):
    a = _cplx(coeffs)
    yx, yy = _f64(np.atleast_1d(yx)), _f64(np.atleast_1d(yy))
    out = np.zeros(2 * yx.shape[0])
    fn(len(coeffs), _ptr(a), centre[0], centre[1], yx.shape[0], _ptr(yx), _ptr(yy), _ptr(out))
    return out.view(np.complex128).copy()


def op_l2p(coeffs, centre, yx, yy):
    """LE polynomial sum_n L_n (y - c)^n at points."""
    return _eval(_load().orc_op_l2p, coeffs, centre, yx, yy)


def op_me_eval(a, centre, yx, yy):
    """ME series sum_m a_m (y - c)^(-m-1) at points."""
    return _eval(_load().orc_op_me_eval, a, centre, yx, yy)


def kernel_error_estimate(a, sigma, sum_gamma):
    return float(_load().orc_kernel_error_estimate(a, sigma, sum_gamma))


def truncation_bound(A, b, p, dist):
    return float(_load().orc_truncation_bound(A, b, p, dist))


def convect(x, y, gamma, dt, velocity, order=2):
    """One convection step of the vortex method (Eq. 5, dx_i/dt = u(x_i)),
    with `velocity(x, y) -> (n, 2)` the velocity at the particles: forward
    Euler (order 1) or Heun's explicit trapezoid rule (order 2).  Returns the
    new (x, y) in float64."""
    x, y = _f64(x), _f64(y)
    u1 = velocity(x, y)
    if order == 1:
        return x + dt * u1[:, 0], y + dt * u1[:, 1]
    if order != 2:
        raise ValueError("order must be 1 or 2")
    xs, ys = x + dt * u1[:, 0], y + dt * u1[:, 1]
    u2 = velocity(xs, ys)
    return x + 0.5 * dt * (u1[:, 0] + u2[:, 0]), y + 0.5 * dt * (u1[:, 1] + u2[:, 1])
