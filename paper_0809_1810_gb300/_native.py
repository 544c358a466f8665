"""ctypes view of libfmm2d (include/fmm2d.h).  Argument marshalling only:
every step of the computation runs in the library's CUDA kernels.  There is
no fallback: if the library is missing the import fails loudly."""
from __future__ import annotations

import ctypes
import os
import re

from . import build as _build

OK, INVALID_ARG, OUT_OF_DOMAIN, NONFINITE, CUDA_ERROR, TIMEOUT, OUT_OF_MEMORY, UNSUPPORTED = range(8)
FP64, FP32, FP32_TC = 0, 1, 2
NUM_PHASES = 6
MLP_INPUTS, MLP_OUTPUTS, MLP_PARAMS = 12, 2, 34946
PHASES = ("tree", "p2m", "m2m", "m2l", "l2l", "p2p_l2p")

HEADER = os.path.join(_build.INCLUDE, "fmm2d.h")


class Params(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("L", ctypes.c_int), ("sigma", ctypes.c_double),
                ("precision", ctypes.c_int), ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("W", ctypes.c_double), ("max_n", ctypes.c_int64), ("cutoff", ctypes.c_double)]


class Instance(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("p", ctypes.c_int), ("L", ctypes.c_int),
                ("sigma", ctypes.c_double), ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("W", ctypes.c_double), ("cutoff", ctypes.c_double)]


_lib = None


def declared_functions():
    """Names of the functions include/fmm2d.h declares."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fmm2d_[a-z_0-9]+)\s*\(", text)))


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"libfmm2d not built: {path} is missing")
        _build.build()
    lib = ctypes.CDLL(path)
    vp, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sigs = {
        "fmm2d_status_string": ([i32], ctypes.c_char_p),
        "fmm2d_last_error": ([], ctypes.c_char_p),
        "fmm2d_plan_create": ([ctypes.POINTER(vp), ctypes.POINTER(Params)], i32),
        "fmm2d_plan_destroy": ([vp], None),
        "fmm2d_velocity": ([vp, i64, vp, vp, vp, vp], i32),
        "fmm2d_velocity_host": ([vp, i64, vp, vp, vp, vp], i32),
        "fmm2d_velocity_host_many": ([vp, i32, i64, vp, vp, vp, vp], i32),
        "fmm2d_velocity_targets": ([vp, i64, vp, vp, i64, vp, vp, vp], i32),
        "fmm2d_convect": ([vp, i64, vp, vp, d, i32, vp], i32),
        "fmm2d_plan_check": ([vp, vp], i32),
        "fmm2d_tree_debug": ([vp, vp, vp, vp, vp], i32),
        "fmm2d_direct_sampled": ([vp, i32, i64, vp, vp, i64, vp, vp, vp], i32),
        "fmm2d_error_stats": ([vp, i64, vp, vp, i64, vp, vp, vp, vp, vp], i32),
        "fmm2d_plan_set_timing": ([vp, i32], i32),
        "fmm2d_plan_phase_ms": ([vp, i32, vp], i32),
        "fmm2d_plan_kernels_per_call": ([vp], i32),
        "fmm2d_plan_set_spin_limit": ([vp, ctypes.c_uint32], i32),
        "fmm2d_plan_set_ring_strips": ([vp, i32], i32),
        "fmm2d_plan_multipole_reals": ([vp], i64),
        "fmm2d_multipoles": ([vp, i64, vp, vp, vp, vp], i32),
        "fmm2d_velocity_from_multipoles": ([vp, i64, vp, vp, vp, vp, vp], i32),
        "fmm2d_tree_build_noalloc": ([i32, i64, vp, vp, i32, d, d, d, vp, vp, vp, vp, vp], i32),
        "fmm2d_batch_last_error": ([], ctypes.c_char_p),
        "fmm2d_batch_plan_create": ([ctypes.POINTER(vp), i32, vp], i32),
        "fmm2d_batch_plan_create_ex": ([ctypes.POINTER(vp), i32, vp, i32], i32),
        "fmm2d_batch_plan_destroy": ([vp], None),
        "fmm2d_batch_velocity": ([vp, vp, vp, vp, vp], i32),
        "fmm2d_batch_check": ([vp, vp], i32),
        "fmm2d_batch_autotune": ([vp, vp, vp, vp, vp], i32),
        "fmm2d_batch_direct_sampled": ([vp, i32, vp, vp, i64, vp, vp, vp], i32),
        "fmm2d_batch_error_stats": ([vp, vp, vp, i64, vp, vp, vp, vp, vp], i32),
        "fmm2d_batch_info": ([vp, vp, vp, vp, vp, vp], i32),
        "fmm2d_batch_info_tc": ([vp, vp, vp, vp, vp], i32),
        "fmm2d_batch_profile": ([vp, vp, vp, vp, vp, vp], i32),
        "fmm2d_batch_tree_debug": ([vp, vp, vp, vp, vp], i32),
        "fmm2d_mlp_last_error": ([], ctypes.c_char_p),
        "fmm2d_mlp_create": ([ctypes.POINTER(vp), i32, ctypes.c_uint64], i32),
        "fmm2d_mlp_destroy": ([vp], None),
        "fmm2d_mlp_set_normalization": ([vp, vp, vp, vp, vp], i32),
        "fmm2d_mlp_params": ([vp, vp, vp], i32),
        "fmm2d_mlp_forward": ([vp, i32, vp, vp, vp], i32),
        "fmm2d_mlp_gradients": ([vp, i32, vp, vp, vp, vp, vp], i32),
        "fmm2d_mlp_train_step": ([vp, i32, vp, vp, ctypes.c_float, vp, vp], i32),
        "fmm2d_features": ([i64, vp, vp, d, d, d, d, i32, i32, vp, vp], i32),
        "fmm2d_propose": ([vp, i32, vp, vp, d, d, i32, i32, vp, vp, vp, vp], i32),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib
