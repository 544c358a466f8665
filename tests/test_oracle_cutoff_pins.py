"""Pins of the oracle's cutoff a (Sec. 4.1, Eq. 29): a pair closer than a keeps
the regularised kernel even when its leaves are not neighbours.

Each test checks the cut functions against an independent fact: the plain 3x3
rule they must reduce to, the direct sum of Eq. 9 they must reduce to when a
spans the domain, the hybrid sum the FMM converges to, and the kernel bound of
Eq. 29 (with the squared distance of Eq. 6).
"""
import math

import numpy as np
import pytest

import workloads as W


def _set(n=2500, seed=21, soh=2.0):
    # leaf / sigma = 2 at L = 4 (h = 2/50, sigma = 2h = 0.08, leaf = 0.125):
    # the 3x3 rule alone leaves a large kernel error
    return W.uniform_random(n, seed, 2.0 / 50, sigma_over_h=soh, dtype=np.float64)


def test_tiny_cutoff_is_the_plain_rule(oracle_lib):
    """A cutoff below every particle separation changes no pair: the cut
    hybrid and FMM must equal the plain ones bit for bit."""
    w = _set()
    d = np.hypot(w.x[:, None] - w.x[None, :], w.y[:, None] - w.y[None, :])
    tiny = 0.5 * d[d > 0].min()
    for L in (2, 4):
        np.testing.assert_array_equal(
            oracle_lib.hybrid(w.x, w.y, w.gamma, w.sigma, w.root, L, a=tiny),
            oracle_lib.hybrid(w.x, w.y, w.gamma, w.sigma, w.root, L))
        np.testing.assert_array_equal(
            oracle_lib.fmm(w.x, w.y, w.gamma, w.sigma, 8, L, w.root, a=tiny),
            oracle_lib.fmm(w.x, w.y, w.gamma, w.sigma, 8, L, w.root))


def test_cutoff_spanning_the_domain_is_the_direct_sum(oracle_lib):
    """With a larger than the root box's diagonal every pair keeps K_sigma:
    the cut hybrid is the direct sum of Eq. 9 exactly (same pairs, same
    order), and the cut FMM is the direct sum up to its truncation error
    (far field through singular expansions, then corrected pair by pair)."""
    w = _set(1200, 22)
    a = 3.0  # root box [-1, 1]^2: diagonal 2.83
    t = W.sample_targets(w.n, 300, 2)
    ref = oracle_lib.direct(w.x, w.y, w.gamma, w.sigma, targets=t)
    for L in (2, 3, 4):
        np.testing.assert_array_equal(
            oracle_lib.hybrid(w.x, w.y, w.gamma, w.sigma, w.root, L, targets=t, a=a), ref)
    full = oracle_lib.direct(w.x, w.y, w.gamma, w.sigma)
    m = np.abs(full).max()
    for L in (3, 4):  # leaf = 3.1 sigma, 1.6 sigma
        got = oracle_lib.fmm(w.x, w.y, w.gamma, w.sigma, 40, L, w.root, a=a)
        assert np.abs(got - full).max() / m < 1e-12, L
        plain = oracle_lib.fmm(w.x, w.y, w.gamma, w.sigma, 40, L, w.root)
        assert np.abs(plain - full).max() / m > 1e-4  # the correction did the work


@pytest.mark.parametrize("a_over_leaf", [0.6, 1.3, 1.9])
def test_cut_fmm_converges_to_the_cut_hybrid_sum(oracle_lib, a_over_leaf):
    """As p grows the cut FMM tends to the cut hybrid sum, geometrically, down
    to rounding level -- whatever ring of leaves the cutoff reaches."""
    w = _set()
    L = 4
    a = a_over_leaf * 2.0 / 2 ** L
    ref = oracle_lib.hybrid(w.x, w.y, w.gamma, w.sigma, w.root, L, a=a)
    m = np.abs(ref).max()
    errs = [np.abs(oracle_lib.fmm(w.x, w.y, w.gamma, w.sigma, p, L, w.root, a=a) - ref).max() / m
            for p in (4, 8, 16, 24, 40)]
    assert errs[-1] < 1e-13, errs
    assert all(b < a_ for a_, b in zip(errs[:3], errs[1:4])), errs


def test_cutoff_error_within_eq29_bound(oracle_lib):
    """Pairs left on the singular kernel are at r >= a, where
    |K_sigma - K'| = exp(-r^2 / 2 sigma^2) / (2 pi r) <= exp(-a^2 / 2 sigma^2) / (2 pi a),
    so |u_cut - u_sigma| <= exp(-a^2 / 2 sigma^2) sum |Gamma_j| / (2 pi a) at every
    target (Eq. 29).  The plain 3x3 rule at the same depth breaks that bound
    for a well inside the ring, so the cutoff is what keeps the error in it."""
    w = _set()
    L = 4
    t = W.sample_targets(w.n, 400, 3)
    ref = oracle_lib.direct(w.x, w.y, w.gamma, w.sigma, targets=t)
    sg = np.abs(w.gamma).sum()
    plain = np.hypot(*(oracle_lib.hybrid(w.x, w.y, w.gamma, w.sigma, w.root, L, targets=t)
                       - ref).T).max()
    for a_over_sigma in (2.5, 3.0, 3.5, 4.0):
        a = a_over_sigma * w.sigma
        bound = math.exp(-a * a / (2 * w.sigma ** 2)) * sg / (2 * math.pi * a)
        err = np.hypot(*(oracle_lib.hybrid(w.x, w.y, w.gamma, w.sigma, w.root, L, targets=t, a=a)
                         - ref).T)
        assert err.max() <= bound, (a_over_sigma, err.max(), bound)
        assert err.max() > 0
    a = 4.0 * w.sigma
    assert plain > math.exp(-a * a / (2 * w.sigma ** 2)) * sg / (2 * math.pi * a)


def test_cutoff_error_falls_as_a_grows(oracle_lib):
    """More pairs on the regularised kernel: the kernel error against the
    direct sum falls strictly as a grows through the ring of leaves."""
    w = _set(3000, 23)
    L = 4
    leaf = 2.0 / 2 ** L
    t = W.sample_targets(w.n, 300, 4)
    ref = oracle_lib.direct(w.x, w.y, w.gamma, w.sigma, targets=t)
    m = np.abs(ref).max()
    errs = [np.abs(oracle_lib.hybrid(w.x, w.y, w.gamma, w.sigma, w.root, L, targets=t, a=a)
                   - ref).max() / m for a in (0.0, 1.2 * leaf, 1.6 * leaf, 2.0 * leaf)]
    assert all(b < a_ for a_, b in zip(errs, errs[1:])), errs


def test_cutoff_rejects_negative_and_nan(oracle_lib):
    w = _set(100, 24)
    for a in (-1.0, float("nan")):
        with pytest.raises(Exception):
            oracle_lib.hybrid(w.x, w.y, w.gamma, w.sigma, w.root, 3, a=a)
        with pytest.raises(Exception):
            oracle_lib.fmm(w.x, w.y, w.gamma, w.sigma, 4, 3, w.root, a=a)
