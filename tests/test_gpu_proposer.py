"""Learned (p, L) proposer on the GPU (fmm2d_mlp_*, fmm2d_features,
fmm2d_propose) against the CPU oracle (oracle/proposer.py).

Tolerances: the kernels accumulate 12- and 128-term dot products in FP32
with O(1) standardised activations through four layers, so outputs and
gradients carry relative errors of a few 1e-6; the bars below (2e-5 on
outputs, 1e-4 of the largest gradient) leave room for that and still catch
a wrong term, sign, index or transposed matrix, all of which move results
at O(1)."""
import ctypes
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import proposer as OP
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


def _net(rows=1024, seed=1, norm_seed=2):
    from paper_0809_1810_gb300.proposer import MLP

    net = MLP(max_rows=rows, seed=seed)
    rng = np.random.default_rng(norm_seed)
    norm = (rng.normal(size=12), rng.uniform(0.5, 2.0, 12), rng.normal(size=2),
            rng.uniform(0.5, 2.0, 2))
    net.set_normalization(*norm)
    return net, tuple(np.asarray(a, np.float32).astype(np.float64) for a in norm)


def test_params_roundtrip_and_initial_scale():
    net, _ = _net()
    w = net.params()
    assert w.shape == (OP.N_PARAMS,)
    layers = OP.unpack(w)
    for (Wl, b), nin in zip(layers, OP.DIMS[:-1]):
        assert np.abs(Wl).max() <= 1.0 / math.sqrt(nin) and not b.any()
    w2 = np.random.default_rng(3).normal(size=OP.N_PARAMS).astype(np.float32) * 0.05
    net.set_params(w2)
    np.testing.assert_array_equal(net.params(), w2)
    net.close()


@pytest.mark.parametrize("rows", [1, 333, 1024])
def test_forward_matches_oracle(rows):
    net, norm = _net()
    rng = np.random.default_rng(rows)
    w = (rng.normal(size=OP.N_PARAMS) * 0.1).astype(np.float32)
    net.set_params(w)
    x = rng.normal(size=(rows, 12)).astype(np.float32) * 3
    y = net.forward(torch.tensor(x, device="cuda")).cpu().numpy()
    want = OP.forward(w, norm, x)
    scale = np.abs(want).max()
    assert np.abs(y - want).max() <= 2e-5 * max(scale, 1.0)
    # the plain float32 weights give a measurably different answer: the
    # kernels really compute with the BF16 copies
    plain = OP.forward(w, norm, x, bf16=False)
    assert np.abs(plain - want).max() > 10 * np.abs(y - want).max()
    net.close()


@pytest.mark.parametrize("rows", [7, 257])
def test_gradients_match_oracle(rows):
    net, norm = _net()
    rng = np.random.default_rng(10 + rows)
    w = (rng.normal(size=OP.N_PARAMS) * 0.1).astype(np.float32)
    net.set_params(w)
    x = rng.normal(size=(rows, 12)).astype(np.float32)
    t = rng.normal(size=(rows, 2)).astype(np.float32)
    g, loss = net.gradients(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"))
    g = g.cpu().numpy()
    want_loss, want = OP.loss_and_grad(w, norm, x, t)
    assert float(loss) == pytest.approx(want_loss, rel=2e-5)
    at = 0
    for i in range(4):  # per layer: weights, then biases
        for size in (OP.DIMS[i + 1] * OP.DIMS[i], OP.DIMS[i + 1]):
            sl = slice(at, at + size)
            assert np.abs(g[sl] - want[sl]).max() <= 1e-4 * np.abs(want[sl]).max(), (i, size)
            at += size
    net.close()


def test_adam_step_matches_oracle():
    net, norm = _net()
    rng = np.random.default_rng(21)
    w0 = (rng.normal(size=OP.N_PARAMS) * 0.1).astype(np.float32)
    net.set_params(w0)
    x = rng.normal(size=(300, 12)).astype(np.float32)
    t = rng.normal(size=(300, 2)).astype(np.float32)
    lr = 1e-3
    net.train_step(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"), lr)
    w1 = net.params().astype(np.float64)
    _, g = OP.loss_and_grad(w0, norm, x, t)
    z = np.zeros_like(g)
    want, _, _ = OP.adam(w0.astype(np.float64), g, z, z, 1, lr)
    # the first step moves each weight by lr * g / (|g| + eps): its size is
    # fixed, only the sign of g matters, so compare where g is clear of
    # FP32 noise; everywhere the move is at most lr
    clear = np.abs(g) > 1e-3 * np.abs(g).max()
    assert clear.mean() > 0.5
    assert np.abs(w1 - want)[clear].max() <= 1e-7
    assert np.abs(w1 - w0).max() <= lr * (1 + 1e-5)
    net.close()


def _particle_sets():
    yield W.uniform_random(3000, 7, 2.0 / 55, sigma_over_h=2.0)
    yield W.lamb_oseen_lattice(64, dtype=np.float32)
    yield W.clustered_patches(5000, 8, npatch=9, h=2.0 / 70)


@pytest.mark.parametrize("L", [0, 2, 5, 9])
def test_features_match_oracle(L):
    from paper_0809_1810_gb300.proposer import features

    for w in _particle_sets():
        xy = torch.tensor(np.stack([w.x, w.y], 1).astype(np.float32), device="cuda")
        g = torch.tensor(w.gamma.astype(np.float32), device="cuda")
        got = features(xy, g, w.sigma, w.root, 13, L)
        want = OP.features(w.x.astype(np.float32), w.y.astype(np.float32),
                           w.gamma.astype(np.float32), w.sigma, w.root, 13, L)
        np.testing.assert_allclose(got, want, rtol=2e-6, atol=2e-6, err_msg=w.name)


def test_training_kernels_fit_a_smooth_function():
    from paper_0809_1810_gb300.proposer import train

    rng = np.random.default_rng(30)
    X = rng.uniform(-2, 2, size=(6144, 12)).astype(np.float32)
    Y = np.stack([np.sin(X[:, 0]) * X[:, 1] + 0.3 * X[:, 2] ** 2,
                  np.exp(-X[:, 3] ** 2) - 0.5 * X[:, 4] * X[:, 5]], 1).astype(np.float32)
    Xv, Yv = X[5120:], Y[5120:]
    net, hist = train(X[:5120], Y[:5120], epochs=150, batch=512, lr=3e-3, seed=4,
                      X_val=Xv, Y_val=Yv)
    assert hist[-1]["train_mse"] < 0.03 * hist[0]["train_mse"]
    rmse = np.array(hist[-1]["val_rmse"])
    assert (rmse < 0.15 * Yv.std(0)).all(), rmse
    net.close()


def test_propose_follows_the_oracle_rule():
    from paper_0809_1810_gb300 import _native

    net, norm = _net(rows=256)
    rng = np.random.default_rng(40)
    w = (rng.normal(size=OP.N_PARAMS) * 0.1).astype(np.float32)
    net.set_params(w)
    nc = 200
    feats = rng.normal(size=(nc, 12)).astype(np.float32)
    feats[:, 0] = rng.integers(4, 29, nc)
    feats[:, 1] = rng.integers(3, 10, nc)
    cost = rng.uniform(1, 100, nc)
    pred = OP.forward(w, norm, feats)[:, 1]
    srt = np.sort(pred)
    lib = _native.load()
    for q in (0.1, 0.5, 0.9):
        k = int(q * nc)
        thr = 0.5 * (srt[k] + srt[k + 1])  # the threshold falls between two predictions
        margin = 0.25
        tol = 10.0 ** (thr + margin)
        p, L, ch = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        out = np.empty((nc, 2), np.float32)
        st = lib.fmm2d_propose(net._h, nc, feats.ctypes.data_as(ctypes.c_void_p),
                               cost.ctypes.data_as(ctypes.c_void_p), tol, margin, 20, 6,
                               ctypes.byref(p), ctypes.byref(L), ctypes.byref(ch),
                               out.ctypes.data_as(ctypes.c_void_p))
        assert st == 0
        want = OP.propose(pred, cost, feats[:, 0], feats[:, 1], tol, margin, (20, 6))
        assert (ch.value, p.value, L.value) == want
        assert np.abs(out[:, 1] - pred).max() < 1e-4 * max(1.0, np.abs(pred).max())
    # nothing qualifies -> the fallback
    st = lib.fmm2d_propose(net._h, nc, feats.ctypes.data_as(ctypes.c_void_p),
                           cost.ctypes.data_as(ctypes.c_void_p), 10.0 ** (srt[0] - 1.0), 0.0,
                           20, 6, ctypes.byref(p), ctypes.byref(L), ctypes.byref(ch), None)
    assert st == 0 and (p.value, L.value, ch.value) == (20, 6, -1)
    # a non-integral p in the candidate table is refused
    bad = feats.copy()
    bad[3, 0] = 7.5
    st = lib.fmm2d_propose(net._h, nc, bad.ctypes.data_as(ctypes.c_void_p),
                           cost.ctypes.data_as(ctypes.c_void_p), 1e-6, 0.3, 20, 6,
                           ctypes.byref(p), ctypes.byref(L), None, None)
    assert st == _native.INVALID_ARG and b"candidate 3" in lib.fmm2d_mlp_last_error()
    net.close()
