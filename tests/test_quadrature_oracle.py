"""Pins of the hat quadrature in y (oracle op_wall(quad=1)) and the
quadrature ablation.

The hat quadrature filters the piecewise-linear interpolant of the
wall-extended field exactly (the alternative quadrature Sec. 3 names for the
commutation error).  Pins:
  * filtering a field equals the brute-force integral (fine trapezoid) of
    the kernel against the interpolant of the Eq. 7 extension, at interior
    and wall rows, even and odd parity;
  * rows sum to one; a linear profile is reproduced exactly away from the
    walls, which the trapezoid rule on a stretched grid does not do;
Ablation (reported in the design notes): against the continuous Gaussian
filter of a smooth profile, both quadratures converge at second order; the
trapezoid rule has the smaller constant on the tanh grid.
"""
import math

import numpy as np

from oracle import oracle as O
from paper_1902_02508_gb300 import inputs as I


def gauss(s, delta):
    return math.sqrt(6.0 / (math.pi * delta * delta)) * np.exp(-6.0 * s * s / (delta * delta))


def extended_interp(s, y, f, parity):
    """Piecewise-linear interpolant of f on [-1, 1] extended by Eq. 7 mirror
    images about both walls with the given parity (period 4)."""
    t = np.mod(s + 1.0, 4.0) - 1.0            # into [-1, 3)
    sign = np.ones_like(t)
    upper = t > 1.0                            # mirror about y = +1
    t = np.where(upper, 2.0 - t, t)
    sign = np.where(upper, float(parity), sign)
    return sign * np.interp(t, y, f)


def brute_row(yi, y, f, delta, parity, n=400001):
    s = np.linspace(yi - 2.5 * delta, yi + 2.5 * delta, n)
    g = gauss(s - yi, delta)
    v = extended_interp(s, y, f, parity)
    return np.trapezoid(g * v, s) / np.trapezoid(g, s)


def test_hat_rows_equal_brute_force_integral():
    y = I.tanh_nodes(33)
    rng = np.random.default_rng(3)
    f = rng.standard_normal(33)
    delta = 0.3
    for parity in (+1, -1):
        fp = f.copy()
        if parity < 0:
            fp[0] = fp[-1] = 0.0                # an odd field vanishes at the walls
        A = O.op_wall(y, y, delta, parity, quad=1)
        for i in (0, 2, 9, 16, 30, 32):
            assert abs(A[i] @ fp - brute_row(y[i], y, fp, delta, parity)) < 1e-8, (parity, i)


def test_hat_reproduces_linear_profiles():
    y = I.tanh_nodes(65)
    delta = 0.3
    f = 0.3 + 0.7 * y
    inner = np.abs(y) < 1 - 2.5 * delta
    Ah = O.op_wall(y, y, delta, +1, quad=1)
    At = O.op_wall(y, y, delta, +1, quad=0)
    assert np.abs(Ah.sum(axis=1) - 1).max() < 1e-14
    assert np.abs((Ah @ f - f)[inner]).max() < 1e-14
    assert np.abs((At @ f - f)[inner]).max() > 1e-7      # the trapezoid rule does not, on this grid


def test_quadrature_ablation_second_order():
    delta = 0.3
    k1, k2 = 3.0, 5.0
    err = {0: [], 1: []}
    for ny in (65, 129, 257):
        y = I.tanh_nodes(ny)
        Y = I.tanh_nodes(17)
        f = 0.3 * np.cos(k1 * y) + 0.2 * np.sin(k2 * y)
        exact = (0.3 * np.cos(k1 * Y) * math.exp(-k1 * k1 * delta * delta / 24)
                 + 0.2 * np.sin(k2 * Y) * math.exp(-k2 * k2 * delta * delta / 24))
        inner = np.abs(Y) < 1 - 2.5 * delta - 0.05
        for q in (0, 1):
            A = O.op_wall(y, Y, delta, +1, quad=q)
            err[q].append(np.abs((A @ f - exact)[inner]).max())
    for q in (0, 1):
        rates = [math.log2(err[q][k] / err[q][k + 1]) for k in range(2)]
        assert min(rates) > 1.8, (q, err[q])
    assert err[0][-1] < err[1][-1]
