"""Pins of the oracle's convection step (Eq. 5: dx_i/dt = u(x_i)).

Two equal regularised vortices a distance d apart turn rigidly about their
midpoint at Omega = (Gamma_1 + Gamma_2)(1 - exp(-d^2 / 2 sigma^2)) / (2 pi d^2)
(each moves with the other's Eq. 6 velocity, perpendicular to the line
between them): the exact trajectory is a circle, which pins the integrator
and its order.  A discrete velocity field from an antisymmetric kernel keeps
sum_i Gamma_i x_i fixed: any step built on it conserves that to rounding.
"""
import math

import numpy as np
import pytest

import workloads as W


def _pair_error(oracle_lib, steps, order, turns=0.25):
    sigma, d, g = 0.05, 0.1, 1.0
    x = np.array([-d / 2, d / 2])
    y = np.array([0.0, 0.0])
    gam = np.array([g, g])
    omega = 2 * g * (1 - math.exp(-d * d / (2 * sigma * sigma))) / (2 * math.pi * d * d)
    dt = turns * 2 * math.pi / omega / steps

    def vel(xx, yy):
        return oracle_lib.direct(xx, yy, gam, sigma)

    for _ in range(steps):
        x, y = oracle_lib.convect(x, y, gam, dt, vel, order=order)
    th = omega * steps * dt
    want_x = np.array([-d / 2 * math.cos(th), d / 2 * math.cos(th)])
    want_y = np.array([-d / 2 * math.sin(th), d / 2 * math.sin(th)])
    return np.hypot(x - want_x, y - want_y).max() / d


@pytest.mark.parametrize("order", [1, 2])
def test_co_rotating_pair_converges_at_the_stated_order(oracle_lib, order):
    e = [_pair_error(oracle_lib, steps, order) for steps in (20, 40, 80)]
    rates = [math.log2(a / b) for a, b in zip(e, e[1:])]
    assert all(abs(r - order) < 0.15 for r in rates), (e, rates)


def test_pair_turns_counter_clockwise(oracle_lib):
    # positive circulation: the right vortex moves up first
    x, y = np.array([-0.05, 0.05]), np.array([0.0, 0.0])
    g = np.array([1.0, 1.0])
    nx, ny = oracle_lib.convect(x, y, g, 1e-3, lambda a, b: oracle_lib.direct(a, b, g, 0.05))
    assert ny[1] > 0 > ny[0]


@pytest.mark.parametrize("order", [1, 2])
def test_circulation_weighted_centre_is_conserved(oracle_lib, order):
    w = W.uniform_random(1500, 71, 2.0 / 39, sigma_over_h=1.5, dtype=np.float64)
    x, y = w.x, w.y

    def vel(xx, yy):
        return oracle_lib.direct(xx, yy, w.gamma, w.sigma)

    c0 = np.array([np.dot(w.gamma, x), np.dot(w.gamma, y)])
    for _ in range(3):
        x, y = oracle_lib.convect(x, y, w.gamma, 0.05, vel, order=order)
    c1 = np.array([np.dot(w.gamma, x), np.dot(w.gamma, y)])
    moved = np.abs(x - w.x).max()
    assert moved > 1e-4  # the particles did move
    assert np.abs(c1 - c0).max() < 1e-12 * np.abs(w.gamma).sum()
