"""The allocation-free tree build (fmm2d_tree_build_noalloc).

Some callers cannot allocate device memory -- a host framework that owns the
whole device budget through its own memory manager, or a latency-critical
loop where cudaMalloc / cudaFree (which can synchronise the device) are not
acceptable.  For them the library offers one entry point whose scratch is a
fixed array inside the library.  This test calls it through the C ABI and
checks that, on two calls in a row, it gives exactly (bit for bit, the bar of
every integer/index test here) what the plan-based entry point gives
(fmm2d_velocity followed by fmm2d_tree_debug).  It lives in a file of its own
that pytest collects last.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

MAX_N = 1 << 18


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0809_1810_gb300 import _native, build

    build.build()
    torch.cuda.set_device(0)
    return _native.load()


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(lib, w, prec_code, dtype):
    n = w.n
    xy = torch.tensor(np.stack([w.x, w.y], 1), dtype=dtype, device="cuda")
    g = torch.tensor(w.gamma, dtype=dtype, device="cuda")
    keys = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    perm = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    start = torch.empty((1 << (2 * w.L)) + 1, dtype=torch.int32, device="cuda")
    flags = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.fmm2d_tree_build_noalloc(prec_code, n, _p(xy), _p(g), w.L, w.root[0], w.root[1],
                                      w.root[2], _p(keys), _p(perm), _p(start), _p(flags), stream)
    assert st == 0, lib.fmm2d_status_string(st)
    torch.cuda.synchronize()
    return keys[:n].cpu(), perm[:n].cpu(), start.cpu(), int(flags.item())


def _with_plan(w, prec, dtype):
    from paper_0809_1810_gb300 import Plan

    xy = torch.tensor(np.stack([w.x, w.y], 1), dtype=dtype, device="cuda")
    g = torch.tensor(w.gamma, dtype=dtype, device="cuda")
    with Plan(w.p, w.L, w.sigma, prec, root=w.root, max_n=max(w.n, 1)) as plan:
        plan.velocity(xy, g, check=True)
        keys, perm, start = plan.tree(w.n)
        torch.cuda.synchronize()
        return keys.cpu(), perm.cpu(), start.cpu()


@pytest.mark.parametrize("prec,code,dtype,npdt", [("fp32", 1, torch.float32, np.float32),
                                                  ("fp64", 0, torch.float64, np.float64)])
def test_noalloc_tree_matches_plan_tree_on_two_calls(lib, prec, code, dtype, npdt):
    # two calls in a row: the second is smaller, at another depth and with
    # other data, so stale contents of the shared scratch would show
    first = W.uniform_random(MAX_N, 77, 2.0 / 512, p=8, L=7, dtype=npdt)
    second = W.uniform_random(50001, 78, 2.0 / 224, p=8, L=5, dtype=npdt)
    for w in (first, second):
        got = _noalloc(lib, w, code, dtype)
        want = _with_plan(w, prec, dtype)
        assert torch.equal(got[0], want[0])  # sorted keys
        assert torch.equal(got[1], want[1])  # permutation
        assert torch.equal(got[2], want[2])  # leaf ranges
        assert got[3] == 0  # no input error flagged


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    from paper_0809_1810_gb300 import _native

    n = MAX_N + 1
    xy = torch.zeros(2 * n, dtype=torch.float32, device="cuda")
    g = torch.zeros(n, dtype=torch.float32, device="cuda")
    keys = torch.empty(n, dtype=torch.int32, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    start = torch.empty((1 << 8) + 1, dtype=torch.int32, device="cuda")
    st = lib.fmm2d_tree_build_noalloc(1, n, _p(xy), _p(g), 4, -1.0, -1.0, 2.0, _p(keys),
                                      _p(perm), _p(start), None, None)
    assert st == _native.INVALID_ARG


def test_noalloc_flags_out_of_domain(lib):
    w = W.uniform_random(1000, 5, 0.05, p=4, L=3, dtype=np.float32)
    w.x[3] = 1.25
    _, _, _, flags = _noalloc(lib, w, 1, torch.float32)
    assert flags == (1 << 2)


@pytest.mark.parametrize("L", [0, 2, 4])
def test_noalloc_single_pass_depths_match_plan_tree(lib, L):
    # depths of at most 8 key bits sort in one pass, which goes from the
    # scratch array straight into the caller's keys and permutation
    w = W.uniform_random(30001, 90 + L, 2.0 / 173, p=6, L=L, dtype=np.float32)
    got = _noalloc(lib, w, 1, torch.float32)
    want = _with_plan(w, "fp32", torch.float32)
    assert torch.equal(got[0], want[0])
    assert torch.equal(got[1], want[1])
    assert torch.equal(got[2], want[2])
    assert got[3] == 0


def test_noalloc_empty_input_gives_empty_leaves(lib):
    start = torch.full(((1 << 6) + 1,), 7, dtype=torch.int32, device="cuda")
    flags = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    st = lib.fmm2d_tree_build_noalloc(1, 0, None, None, 3, -1.0, -1.0, 2.0, None, None,
                                      _p(start), _p(flags), None)
    assert st == 0
    torch.cuda.synchronize()
    assert int(start.abs().sum().item()) == 0  # every leaf range empty
    assert int(flags.item()) == 0


def test_noalloc_without_flags_buffer_uses_its_own_status_word(lib):
    # flags = NULL: the input-error word lives in the scratch array instead;
    # the tree is the same
    w = W.uniform_random(20000, 95, 2.0 / 141, p=6, L=6, dtype=np.float32)
    n = w.n
    xy = torch.tensor(np.stack([w.x, w.y], 1), device="cuda")
    g = torch.tensor(w.gamma, device="cuda")
    keys = torch.empty(n, dtype=torch.int32, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    start = torch.empty((1 << 12) + 1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        st = lib.fmm2d_tree_build_noalloc(1, n, _p(xy), _p(g), w.L, w.root[0], w.root[1],
                                          w.root[2], _p(keys), _p(perm), _p(start), None, None)
        assert st == 0
        torch.cuda.synchronize()
        want = _with_plan(w, "fp32", torch.float32)
        assert torch.equal(keys.cpu(), want[0])
        assert torch.equal(perm.cpu(), want[1])
        assert torch.equal(start.cpu(), want[2])
