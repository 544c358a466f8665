"""Pins of the proposer oracle (oracle/proposer.py) against things other than
itself: central finite differences, torch's bfloat16 conversion and worked
bit patterns, closed forms of SiLU and of Adam's first step, a hand-built
particle set, a worked selection table."""
import math

import numpy as np
import pytest
import torch

from oracle import proposer as P


def _norm(rng=None):
    if rng is None:
        return (np.zeros(12), np.ones(12), np.zeros(2), np.ones(2))
    return (rng.normal(size=12), rng.uniform(0.5, 2.0, 12), rng.normal(size=2),
            rng.uniform(0.5, 2.0, 2))


def _params(rng, scale=1.0):
    layers = []
    for i in range(4):
        nin, nout = P.DIMS[i], P.DIMS[i + 1]
        a = scale / math.sqrt(nin)
        layers.append((rng.uniform(-a, a, (nout, nin)), rng.uniform(-0.1, 0.1, nout)))
    return P.pack(layers)


def test_parameter_count_matches_architecture():
    # 12*128+128 + 2*(128*128+128) + 128*2+2
    assert P.N_PARAMS == 34946
    rng = np.random.default_rng(0)
    w = _params(rng)
    np.testing.assert_array_equal(P.pack(P.unpack(w)), w)


def test_bf16_rounding_worked_values():
    # bfloat16 keeps 8 significant bits: spacing 2^-7 just above 1.
    cases = {1.0: 1.0, 1.0 + 2.0 ** -8: 1.0,                # tie -> even (1.0)
             1.0 + 3 * 2.0 ** -8: 1.0 + 2.0 ** -6,          # tie -> even (..10)
             1.0 + 2.0 ** -8 + 2.0 ** -20: 1.0 + 2.0 ** -7,  # above the tie
             -2.5: -2.5, 3.140625: 3.140625, 0.0: 0.0}
    for x, want in cases.items():
        assert P.bf16_round(np.float32(x))[()] == want, x


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(size=20000) * 10.0 ** rng.uniform(-30, 30, 20000),
                        np.float32(1.0) + np.arange(-300, 300) * np.float32(2.0 ** -9)])
    x = x.astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(P.bf16_round(x), want)


def test_silu_closed_forms():
    assert P.silu(0.0) == 0.0
    assert P.silu_grad(0.0) == 0.5
    assert P.silu(40.0) == pytest.approx(40.0, rel=1e-15)
    assert abs(P.silu(-40.0)) < 1e-15
    z = np.linspace(-6, 6, 25)
    h = 1e-6
    np.testing.assert_allclose(P.silu_grad(z), (P.silu(z + h) - P.silu(z - h)) / (2 * h),
                               rtol=1e-8, atol=1e-10)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    w = _params(rng, scale=1.5)
    norm = _norm(rng)
    x = rng.normal(size=(7, 12))
    t = rng.normal(size=(7, 2))
    loss, g = P.loss_and_grad(w, norm, x, t, bf16=False)
    # every bias and a spread of weights in each layer
    idx = np.unique(np.concatenate([rng.choice(P.N_PARAMS, 300, replace=False),
                                    np.arange(1536, 1664), np.arange(34944, 34946)]))
    h = 1e-6
    for k in idx:
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd = (P.loss_and_grad(wp, norm, x, t, bf16=False)[0]
              - P.loss_and_grad(wm, norm, x, t, bf16=False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g).max()), (k, fd, g[k])
    assert loss > 0


def test_bf16_gradient_is_the_gradient_at_the_rounded_weights():
    rng = np.random.default_rng(3)
    w = _params(rng).astype(np.float32).astype(np.float64)
    norm = _norm(rng)
    x, t = rng.normal(size=(5, 12)), rng.normal(size=(5, 2))
    rounded = P.pack([(P.bf16_round(W.astype(np.float32)), b) for W, b in P.unpack(w)])
    l1, g1 = P.loss_and_grad(w, norm, x, t, bf16=True)
    l2, g2 = P.loss_and_grad(rounded, norm, x, t, bf16=False)
    assert l1 == l2
    np.testing.assert_array_equal(g1, g2)
    assert not np.array_equal(rounded, w)


def test_zero_weight_network_outputs_its_last_bias():
    layers = [(np.zeros((P.DIMS[i + 1], P.DIMS[i])), np.zeros(P.DIMS[i + 1]))
              for i in range(4)]
    layers[3] = (np.zeros((2, 128)), np.array([0.25, -1.5]))
    w = P.pack(layers)
    norm = (np.zeros(12), np.ones(12), np.array([1.0, -2.0]), np.array([2.0, 4.0]))
    x = np.random.default_rng(4).normal(size=(3, 12))
    y = P.forward(w, norm, x)
    np.testing.assert_array_equal(y, np.tile([1.0 + 2 * 0.25, -2.0 + 4 * -1.5], (3, 1)))
    # targets equal to the output: zero loss and zero gradient
    loss, g = P.loss_and_grad(w, norm, x, y)
    assert loss == 0.0 and not g.any()
    # targets off by one standard deviation in output 0: loss 1/2, and the
    # last bias gradient is 2 d / (rows * outputs) summed over rows = -1
    t = y.copy()
    t[:, 0] += 2.0
    loss, g = P.loss_and_grad(w, norm, x, t)
    assert loss == pytest.approx(0.5)
    assert g[-2] == pytest.approx(-1.0) and g[-1] == 0.0


def test_adam_first_step_moves_by_lr_times_sign():
    g = np.array([3.0, -0.02, 1e-3, -7.0])
    w = np.array([0.5, 0.5, -1.0, 2.0])
    z = np.zeros(4)
    w1, m1, v1 = P.adam(w, g, z, z, 1, lr=0.01)
    # bias correction makes mhat = g and vhat = g^2 after one step
    np.testing.assert_allclose(w1, w - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(v1, 0.001 * g * g)
    # a second step with the same gradient: the corrected moments are again
    # g and g^2 (0.19 g / 0.19 and 0.001999 g^2 / 0.001999)
    w2, _, _ = P.adam(w1, g, m1, v1, 2, lr=0.01)
    np.testing.assert_allclose(w2, w1 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_oracle_training_reduces_loss():
    rng = np.random.default_rng(5)
    w = _params(rng)
    x = rng.normal(size=(64, 12))
    t = np.stack([np.sin(x[:, 0]) + 0.5 * x[:, 1] ** 2, x[:, 2] * x[:, 3]], 1)
    norm = (np.zeros(12), np.ones(12), t.mean(0), t.std(0))
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    first = None
    for step in range(1, 201):
        loss, g = P.loss_and_grad(w, norm, x, t, bf16=False)
        first = loss if first is None else first
        w, m, v = P.adam(w, g, m, v, step, lr=3e-3)
    assert loss < 0.05 * first


def test_features_of_a_hand_built_set():
    # root [-1,1]^2, L = 1: four quadrant leaves.  Leaf (0,0) holds two
    # particles (Gamma 1 and -3), leaf (1,0) one (Gamma 2), leaf (1,1) one
    # (Gamma 4), leaf (0,1) none.  n = 4, sigma = 0.25, p = 9.
    x = np.array([-0.5, -0.25, 0.5, 0.5])
    y = np.array([-0.5, -0.75, -0.5, 0.5])
    g = np.array([1.0, -3.0, 2.0, 4.0])
    f = P.features(x, y, g, 0.25, (-1.0, -1.0, 2.0), 9, 1)
    counts = np.array([2.0, 1.0, 0.0, 1.0])
    S = np.array([-2.0, 2.0, 0.0, 4.0])
    abs_total = 10.0
    A = abs_total / 4
    want = [9, 1, 0.25 / (2.0 / 2.0), 2.0, 0.0,
            math.sqrt(0.5) / 1.0,        # counts: mean 1, variance 0.5
            2.0,                         # max / mean
            8.0 / 10.0,                  # sum |S| / sum |Gamma|
            math.sqrt(5.0) / A,          # S: mean 1, variance (9+1+1+9)/4 = 5
            4.0 / A, 4.0 / 10.0, math.log10(1.0 / 0.25)]
    np.testing.assert_allclose(f, want, rtol=1e-14)
    np.testing.assert_array_equal(counts, np.bincount(
        np.array([0, 0, 1, 3]), minlength=4).astype(float))
    assert S.sum() == g.sum()


def test_features_invariances():
    rng = np.random.default_rng(6)
    n = 5000
    x, y = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    g = rng.normal(size=n)
    f = P.features(x, y, g, 0.01, (-1.0, -1.0, 2.0), 12, 4)
    perm = rng.permutation(n)
    np.testing.assert_allclose(P.features(x[perm], y[perm], g[perm], 0.01,
                                          (-1.0, -1.0, 2.0), 12, 4), f, rtol=1e-12)
    np.testing.assert_allclose(P.features(x, y, 7.5 * g, 0.01, (-1.0, -1.0, 2.0), 12, 4), f,
                               rtol=1e-12)
    # at L = 0 every particle is in the root: counts have no spread, the one
    # leaf sum is the total circulation
    f0 = P.features(x, y, g, 0.01, (-1.0, -1.0, 2.0), 12, 0)
    assert f0[5] == 0.0 and f0[6] == 1.0 and f0[8] == 0.0
    assert f0[7] == pytest.approx(abs(f0[10]), rel=1e-12)


def test_selection_rule_on_a_worked_table():
    pred = [-5.0, -6.5, -7.2, -6.9, -8.0]
    cost = [1.0, 2.0, 3.0, 1.5, 9.0]
    cp = [8, 10, 12, 14, 20]
    cL = [7, 7, 6, 6, 5]
    # tol 1e-6, margin 0.5 -> need <= -6.5: rows 1 (2.0), 2 (3.0), 3 (1.5), 4 (9.0)
    assert P.propose(pred, cost, cp, cL, 1e-6, 0.5, (20, 6)) == (3, 14, 6)
    # margin 1.0 -> need <= -7: rows 2 and 4; the cheaper is row 2
    assert P.propose(pred, cost, cp, cL, 1e-6, 1.0, (20, 6)) == (2, 12, 6)
    # nothing qualifies -> fallback
    assert P.propose(pred, cost, cp, cL, 1e-9, 0.0, (20, 6)) == (-1, 20, 6)
    # equal cost -> the first
    assert P.propose([-9, -9], [1.0, 1.0], [4, 5], [3, 3], 1e-6, 0, (20, 3)) == (0, 4, 3)


def test_cost_regressors_of_a_worked_row():
    # n = 2^20, L = 7, 64 per leaf, cv 0.5, p = 20 (padded to 32)
    # leaf / sigma = 10^0.6 = 4.0 < 5.26: the candidate runs with the cutoff
    f = np.array([20, 7, 2.0, 20, 6, 0.5, 1, 0, 0, 0, 0, 0.6])
    t = P.cost_terms(f)
    boxes = 1 + 4 + 16 + 64 + 256 + 1024 + 4096 + 16384
    np.testing.assert_allclose(t, [1, 2 ** 20, 20 * 2 ** 20, boxes * 32 * 32,
                                   9 * 16384 * 64 * 64 * 1.25, 16 * 16384 * 64 * 64 * 1.25])
    # leaves of 8 sigma: no cutoff, no ring term
    f[11] = math.log10(8.0)
    assert P.cost_terms(f)[5] == 0.0
    # the switch sits where exp(-a^2 / 2 sigma^2) = 1e-6 puts a: one leaf width
    a_over_sigma = math.sqrt(-2.0 * math.log(1e-6))
    f[11] = math.log10(a_over_sigma) - 1e-9
    assert P.cost_terms(f)[5] > 0
    f[11] = math.log10(a_over_sigma) + 1e-9
    assert P.cost_terms(f)[5] == 0.0
