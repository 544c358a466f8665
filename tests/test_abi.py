"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function include/fmm2d.h declares, and rejects
invalid parameters before touching the device.  Also checks that the oracle
and the CUDA path stay independent."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_0809_1810_gb300 import _native, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _native.load()


def test_every_declared_symbol_is_exported(lib):
    names = _native.declared_functions()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("field,value", [("p", 0), ("p", 33), ("L", -1), ("L", 13),
                                         ("sigma", 0.0), ("sigma", float("nan")), ("W", 0.0),
                                         ("W", -2.0), ("precision", 9), ("max_n", -5),
                                         ("cutoff", -0.01), ("cutoff", float("nan")),
                                         ("cutoff", float("inf")),
                                         ("cutoff", 0.0313)])  # > 2 leaf widths at L = 7
def test_invalid_parameters_are_rejected(lib, field, value):
    prm = _native.Params(16, 7, 0.01, _native.FP32, -1.0, -1.0, 2.0, 1000)
    setattr(prm, field, value)
    h = ctypes.c_void_p(1234)
    st = lib.fmm2d_plan_create(ctypes.byref(h), ctypes.byref(prm))
    assert st == _native.INVALID_ARG
    assert h.value is None
    assert lib.fmm2d_last_error()


def test_null_arguments_are_rejected(lib):
    assert lib.fmm2d_plan_create(None, None) == _native.INVALID_ARG
    assert lib.fmm2d_velocity(None, 0, None, None, None, None) == _native.INVALID_ARG
    assert lib.fmm2d_plan_check(None, None) == _native.INVALID_ARG
    assert lib.fmm2d_velocity_targets(None, 0, None, None, 0, None, None, None) == \
        _native.INVALID_ARG
    assert lib.fmm2d_convect(None, 0, None, None, 0.1, 2, None) == _native.INVALID_ARG
    assert lib.fmm2d_plan_set_timing(None, 4) == _native.INVALID_ARG
    assert lib.fmm2d_velocity_host_many(None, 2, 10, None, None, None, None) == \
        _native.INVALID_ARG
    assert lib.fmm2d_plan_set_ring_strips(None, 1) == _native.INVALID_ARG
    lib.fmm2d_plan_destroy(None)  # accepted


def test_status_strings(lib):
    for s in range(8):
        assert lib.fmm2d_status_string(s)
    assert lib.fmm2d_status_string(99) == b"unknown status"


def _imports(path):
    with open(path) as f:
        text = f.read()
    return set(re.findall(r"^\s*(?:from|import)\s+([A-Za-z_][\w.]*)", text, flags=re.M))


def test_oracle_and_cuda_path_share_nothing():
    pkg = os.path.join(ROOT, "paper_0809_1810_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            p = os.path.join(dirpath, f)
            if f.endswith(".py"):
                assert not any(m.split(".")[0] == "oracle" for m in _imports(p)), p
            if f.endswith((".cu", ".cuh", ".py", ".h")):
                with open(p) as fh:
                    assert "fmm2d_oracle" not in fh.read(), p
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        p = os.path.join(ROOT, "oracle", f)
        if f.endswith(".py"):
            assert not any(m.split(".")[0] == "paper_0809_1810_gb300" for m in _imports(p)), p
        if f.endswith(".c"):
            with open(p) as fh:
                assert "fmm2d.h" not in fh.read()


@pytest.mark.parametrize("field,value", [("n", -1), ("p", 0), ("p", 40), ("L", 13),
                                         ("sigma", 0.0), ("W", 0.0)])
def test_batch_rejects_invalid_instances(lib, field, value):
    good = _native.Instance(100, 8, 3, 0.01, -1.0, -1.0, 2.0)
    bad = _native.Instance(100, 8, 3, 0.01, -1.0, -1.0, 2.0)
    setattr(bad, field, value)
    arr = (_native.Instance * 2)(good, bad)
    h = ctypes.c_void_p(99)
    assert lib.fmm2d_batch_plan_create(ctypes.byref(h), 2, arr) == _native.INVALID_ARG
    assert h.value is None
    assert b"instance 1" in lib.fmm2d_batch_last_error()


def test_batch_rejects_empty_and_oversized(lib):
    h = ctypes.c_void_p()
    assert lib.fmm2d_batch_plan_create(ctypes.byref(h), 0, None) == _native.INVALID_ARG
    big = (_native.Instance * 300)(*[_native.Instance(10, 4, 12, 0.01, -1.0, -1.0, 2.0)] * 300)
    assert lib.fmm2d_batch_plan_create(ctypes.byref(h), 300, big) == _native.INVALID_ARG


def test_proposer_calls_validate_before_touching_the_device(lib):
    h = ctypes.c_void_p(7)
    assert lib.fmm2d_mlp_create(ctypes.byref(h), 0, 1) == _native.INVALID_ARG
    assert h.value is None
    assert lib.fmm2d_mlp_create(None, 16, 1) == _native.INVALID_ARG
    assert lib.fmm2d_mlp_forward(None, 1, None, None, None) == _native.INVALID_ARG
    assert lib.fmm2d_mlp_train_step(None, 1, None, None, ctypes.c_float(1e-3), None,
                                    None) == _native.INVALID_ARG
    assert lib.fmm2d_features(0, None, None, 0.1, -1.0, -1.0, 2.0, 8, 3, None,
                              None) == _native.INVALID_ARG
    p, L = ctypes.c_int(), ctypes.c_int()
    assert lib.fmm2d_propose(None, 0, None, None, 1e-6, 0.3, 20, 6, ctypes.byref(p),
                             ctypes.byref(L), None, None) == _native.INVALID_ARG
    assert lib.fmm2d_mlp_last_error()
    lib.fmm2d_mlp_destroy(None)


def test_proposer_fallback_rule():
    from paper_0809_1810_gb300 import proposer as PR

    h = 2.0 / 1024
    # 2^20 uniform, sigma = 2h: occupancy gives L = 7, but a leaf must span
    # 6 sigma = 0.0234, so L = floor(log2(2 / 0.0234)) = 6
    assert PR.fallback(1 << 20, 2 * h, (-1.0, -1.0, 2.0)) == (20, 6)
    assert PR.fallback(1 << 20, 0.5 * h, (-1.0, -1.0, 2.0)) == (20, 7)
    assert PR.fallback(10, 0.01, (-1.0, -1.0, 2.0)) == (20, 0)
    assert PR.depth_candidates(1 << 20) == [5, 6, 7, 8, 9]
    assert PR.depth_candidates(1 << 18) == [4, 5, 6, 7, 8]
    t = PR.cost_terms(np.array([16, 7, 0, 20, 6, 0.0, 1, 0, 0, 0, 0, 0], np.float32))
    np.testing.assert_allclose(t, [1, 2 ** 20, 16 * 2 ** 20, (4 ** 8 - 1) / 3 * 256,
                                   9 * 4 ** 7 * 64 * 64, 16 * 4 ** 7 * 64 * 64])
    # the cutoff each candidate runs with: a = sigma sqrt(2 ln 10^6) where the
    # leaf is narrower, capped at two leaf widths
    s = 2 * h
    assert PR.cutoff(s, (-1.0, -1.0, 2.0), 6) == 0.0            # leaf = 8 sigma
    assert abs(PR.cutoff(s, (-1.0, -1.0, 2.0), 7) / s - 5.2565) < 1e-4  # leaf = 4 sigma
    assert PR.cutoff(s, (-1.0, -1.0, 2.0), 9) == 2.0 * 2.0 / 512  # capped
