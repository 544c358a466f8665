"""Batched evaluation (fmm2d_batch_*): many uneven instances in one graph.

Bars:
* velocities of every instance bit-identical to a single-instance FP32 plan
  with the same parameters (same kernels and summation order; the batch only
  packs index spaces);
* quadtree of every instance bit-exact against the oracle;
* FP64 batched yardsticks within 1e-13 of the oracle;
* the 512-instance sweep (N log-uniform in [2^12, 2^17], p in {4..24},
  L in {3..7}, sigma/h in {0.8..2}) against the oracle FMM on sampled
  instances within the FP32 bound of 1e-6.
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


def _mixed_instances():
    out = []
    specs = [(3000, 10, 3, 1.0, "lo"), (0, 8, 3, 1.0, "u"), (1, 4, 0, 1.0, "u"),
             (2500, 1, 2, 1.0, "u"), (5000, 17, 4, 2.0, "u"), (4096, 16, 4, 1.5, "lo"),
             (7000, 24, 5, 0.8, "u"), (1500, 12, 1, 1.0, "u"), (6000, 32, 3, 1.0, "u"),
             (3500, 6, 5, 2.0, "u")]
    for k, (n, p, L, soh, kind) in enumerate(specs):
        if kind == "lo":
            side = int(round(np.sqrt(n)))
            w = W.lamb_oseen_lattice(side, sigma_over_h=soh, p=p, L=L, dtype=np.float32)
        else:
            h = 2.0 / np.sqrt(max(n, 1))
            w = W.uniform_random(n, 40 + k, h, sigma_over_h=soh, p=p, L=L, dtype=np.float32)
        out.append(w)
    return out


def _pack(ws):
    xy = np.concatenate([np.stack([w.x, w.y], 1) for w in ws]).astype(np.float32)
    g = np.concatenate([w.gamma for w in ws]).astype(np.float32)
    return (torch.tensor(xy, device="cuda"), torch.tensor(g, device="cuda"))


def _batch(ws):
    from paper_0809_1810_gb300 import BatchPlan

    return BatchPlan([{"n": w.n, "p": w.p, "L": w.L, "sigma": w.sigma, "root": w.root}
                      for w in ws])


def test_batch_equals_single_instance_plans():
    from paper_0809_1810_gb300 import Plan

    ws = _mixed_instances()
    xy, g = _pack(ws)
    with _batch(ws) as bp:
        uv = bp.velocity(xy, g)
        uv2 = bp.velocity(xy, g)  # graph replay
        bp.check()
        info = bp.info()
    assert info["kernels_per_call"] > 0
    assert torch.equal(uv, uv2)
    off = 0
    for w in ws:
        if w.n:
            with Plan(w.p, w.L, w.sigma, "fp32", root=w.root, max_n=w.n) as plan:
                xyi = torch.tensor(np.stack([w.x, w.y], 1), device="cuda")
                gi = torch.tensor(w.gamma, device="cuda")
                single = plan.velocity(xyi, gi, check=True)
            assert torch.equal(uv[off:off + w.n], single), (w.name, w.p, w.L)
        off += w.n


def test_batch_tree_is_bit_exact():
    from paper_0809_1810_gb300 import _native

    ws = _mixed_instances()
    xy, g = _pack(ws)
    lib = _native.load()
    with _batch(ws) as bp:
        bp.velocity(xy, g)
        bp.check()
        n = bp.n_total
        nleaf = sum(1 << (2 * w.L) for w in ws)
        keys = torch.empty(n, dtype=torch.int32, device="cuda")
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        start = torch.empty(nleaf + 1, dtype=torch.int32, device="cuda")
        import ctypes
        st = lib.fmm2d_batch_tree_debug(bp._h, ctypes.c_void_p(keys.data_ptr()),
                                        ctypes.c_void_p(perm.data_ptr()),
                                        ctypes.c_void_p(start.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0
        torch.cuda.synchronize()
    keys, perm, start = keys.cpu().numpy(), perm.cpu().numpy(), start.cpu().numpy()
    off = 0
    lb = 0
    for w in ws:
        ok = oracle.morton_keys(w.x, w.y, w.root, w.L)
        op, os_ = oracle.sort_by_key(ok, w.L)
        np.testing.assert_array_equal(perm[off:off + w.n].astype(np.int64) - off, op)
        np.testing.assert_array_equal(keys[off:off + w.n].astype(np.int64) - lb, ok[op])
        np.testing.assert_array_equal(start[lb:lb + (1 << (2 * w.L)) + 1].astype(np.int64),
                                      os_.astype(np.int64) + off)
        off += w.n
        lb += 1 << (2 * w.L)


@pytest.mark.parametrize("kernel", [0, 1])
def test_batch_yardsticks(kernel):
    ws = _mixed_instances()
    xy, g = _pack(ws)
    rng = np.random.default_rng(9)
    off, targets, want = 0, [], []
    for w in ws:
        if w.n:
            t = np.sort(rng.choice(w.n, size=min(40, w.n), replace=False))
            targets.append(t + off)
            if kernel == 0:
                want.append(oracle.direct(w.x, w.y, w.gamma, w.sigma, targets=t))
            else:
                want.append(oracle.hybrid(w.x, w.y, w.gamma, w.sigma, w.root, w.L, targets=t))
        off += w.n
    targets = np.concatenate(targets)
    want = np.concatenate(want)
    with _batch(ws) as bp:
        tt = torch.tensor(targets, device="cuda")
        got = bp.direct_sampled(xy, g, tt, kernel=kernel)
        uv = bp.velocity(xy, g)
        stats, leaf = bp.error_stats(xy, uv, tt, got, per_leaf=True)
        bp.check()
    got = got.cpu().numpy()
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * np.abs(want).max())
    # per-instance statistics against numpy
    uvn = uv.double().cpu().numpy()[targets]
    du = np.linalg.norm(uvn - got, axis=1)
    rr = np.linalg.norm(got, axis=1)
    s = stats.cpu().numpy()
    inst_of = np.searchsorted(np.cumsum([w.n for w in ws]), targets, side="right")
    for k in range(len(ws)):
        m = inst_of == k
        if m.any():
            np.testing.assert_allclose(s[k, 0], du[m].max(), rtol=1e-12)
            np.testing.assert_allclose(s[k, 1], rr[m].max(), rtol=1e-12)
        else:
            assert s[k, 0] == 0 and s[k, 1] == 0
    assert leaf.cpu().numpy().max() == pytest.approx(du.max(), rel=1e-12)


def test_autotune_keeps_results():
    ws = _mixed_instances()
    xy, g = _pack(ws)
    with _batch(ws) as bp:
        a = bp.velocity(xy, g).clone()
        out = torch.empty_like(a)
        info = bp.autotune(xy, g, out)
        b = bp.velocity(xy, g)
        bp.check()
    assert info["p2p_ctas_per_sm"] in (2, 3, 4, 5, 6)
    assert info["m2l_threads"] in (64, 128, 256)
    assert torch.equal(a, out) and torch.equal(a, b)


def test_sweep_512_instances_against_oracle():
    """The 512-instance sweep in one graph; sampled instances against the
    oracle FMM (every output) and every instance's sampled direct error sane."""
    specs = W.batch_instances(512)
    ws = [W.make_instance(s) for s in specs]
    xy, g = _pack(ws)
    with _batch(ws) as bp:
        uv = bp.velocity(xy, g)
        bp.check()
        uvn = uv.double().cpu().numpy()
    offs = np.concatenate([[0], np.cumsum([w.n for w in ws])])
    rng = np.random.default_rng(1)
    for k in rng.choice(len(ws), size=6, replace=False):
        w = ws[k]
        ref = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.p, w.L, w.root)
        got = uvn[offs[k]:offs[k + 1]]
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= FP32_TOL, (k, w.n, w.p, w.L, err)


def _cut(w, tol=1e-6):
    """The Sec. 4.1 cutoff for the tolerance where the instance's leaves are
    narrower than it (at most two leaf widths, 0 below L = 2)."""
    from paper_0809_1810_gb300 import cutoff_for

    return cutoff_for(w.sigma, w.root[2] / 2 ** w.L, tol) if w.L >= 2 else 0.0


def _batch_p(ws, precision, cut=True):
    from paper_0809_1810_gb300 import BatchPlan

    return BatchPlan([{"n": w.n, "p": w.p, "L": w.L, "sigma": w.sigma, "root": w.root,
                       "cutoff": _cut(w) if cut else 0.0} for w in ws], precision=precision)


@pytest.mark.parametrize("prec", ["fp32", "fp32_tc"])
def test_batch_with_cutoff_equals_single_plans(prec):
    """Batched instances with the Sec. 4.1 cutoff (where their leaves are
    narrower than it) and, for FP32_TC, the tensor-core M2L per class of p
    rounded up to 4: bit for bit the single plans of the same settings."""
    from paper_0809_1810_gb300 import Plan

    ws = _mixed_instances()
    assert sum(_cut(w) > 0 for w in ws) >= 3  # several instances take the cutoff
    xy, g = _pack(ws)
    with _batch_p(ws, prec) as bp:
        uv = bp.velocity(xy, g)
        uv2 = bp.velocity(xy, g)
        bp.check()
        info = bp.info()
    assert torch.equal(uv, uv2)
    if prec == "fp32_tc":
        assert info["tc_classes"] >= 4 and info["tc_tiles"] > 0
    off = 0
    for w in ws:
        if w.n:
            with Plan(w.p, w.L, w.sigma, prec, root=w.root, max_n=w.n, cutoff=_cut(w)) as plan:
                xyi = torch.tensor(np.stack([w.x, w.y], 1), device="cuda")
                gi = torch.tensor(w.gamma, device="cuda")
                single = plan.velocity(xyi, gi, check=True)
            assert torch.equal(uv[off:off + w.n], single), (w.name, w.p, w.L, _cut(w))
        off += w.n


def test_batch_tc_autotune_keeps_results():
    ws = _mixed_instances()
    xy, g = _pack(ws)
    with _batch_p(ws, "fp32_tc") as bp:
        a = bp.velocity(xy, g).clone()
        out = torch.empty_like(a)
        info = bp.autotune(xy, g, out)
        b = bp.velocity(xy, g)
        bp.check()
    assert info["tc_tile_policy"] in (0, 1) and info["tc_b_stages"] >= 2
    assert torch.equal(a, out) and torch.equal(a, b)


def test_batch_cutoff_yardstick():
    """The batched FMM-limit yardstick honours each instance's cutoff."""
    ws = _mixed_instances()
    xy, g = _pack(ws)
    rng = np.random.default_rng(13)
    off, targets, want = 0, [], []
    for w in ws:
        if w.n:
            t = np.sort(rng.choice(w.n, size=min(30, w.n), replace=False))
            targets.append(t + off)
            want.append(oracle.hybrid(w.x, w.y, w.gamma, w.sigma, w.root, w.L, targets=t,
                                      a=_cut(w)))
        off += w.n
    targets = np.concatenate(targets)
    want = np.concatenate(want)
    with _batch_p(ws, "fp32_tc") as bp:
        got = bp.direct_sampled(xy, g, torch.tensor(targets, device="cuda"), kernel=1)
        bp.check()
    np.testing.assert_allclose(got.cpu().numpy(), want, rtol=0, atol=1e-13 * np.abs(want).max())


def test_sweep_512_tc_with_cutoff_against_oracle():
    """The 512-instance sweep as FP32_TC with each instance's cutoff: sampled
    instances against the oracle's cut FMM within 1e-6."""
    specs = W.batch_instances(512)
    ws = [W.make_instance(s) for s in specs]
    xy, g = _pack(ws)
    with _batch_p(ws, "fp32_tc") as bp:
        uv = bp.velocity(xy, g)
        bp.check()
        uvn = uv.double().cpu().numpy()
    offs = np.concatenate([[0], np.cumsum([w.n for w in ws])])
    rng = np.random.default_rng(2)
    cut_seen = 0
    # FP32 parity with a cutoff needs the correction's jump at r = a,
    # exp(-a^2 / 2 sigma^2) of a pair's value, far below the tolerance: a pair
    # within rounding of r = a is decided either way in FP32 and in FP64
    # (a >= 4.4 sigma, as in the single-plan cutoff tests)
    ok = [k for k, w in enumerate(ws) if _cut(w) == 0.0 or _cut(w) >= 4.4 * w.sigma]
    for k in rng.choice(ok, size=8, replace=False):
        w = ws[k]
        a = _cut(w)
        cut_seen += a > 0
        ref = oracle.fmm(w.x, w.y, w.gamma, w.sigma, w.p, w.L, w.root, a=a)
        got = uvn[offs[k]:offs[k + 1]]
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= FP32_TOL, (k, w.n, w.p, w.L, a / w.sigma, err)
    assert cut_seen > 0
