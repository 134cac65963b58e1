"""FP64 reference of the paper's error measures: TEST INFRASTRUCTURE ONLY.

Only the tests use this module; the CUDA library never calls it.

Sec. 4 of the paper measures how far an LES drifts from the DNS with three
normalised L2 errors, all of velocities scaled by each run's friction
velocity u_tau:
  * Eq. 13: the instantaneous field, integrated over the volume V;
  * Eq. 14: the mean profile <u_1>(x_2), averaged over the homogeneous
    directions x and z and integrated over x_2 from the wall to the channel
    centre (0 .. delta);
  * Eq. 15: the same for the turbulence intensities u_i,rms(x_2).

Quadrature (the paper does not state it): x and z are periodic with uniform
nodes, so their integrals are node sums times L/n; in y the weights are the
trapezoid rule on the given nodes.  The wall-to-centre integral of Eq. 14 and
Eq. 15 is the integral of the piecewise-linear interpolant of the integrand
over y in [-1, 0] (the lower half, x_2 = 1 + y): the trapezoid rule on the
nodes in that half plus the clipped part of the interval that contains
y = 0, if the centre is not a node.
"""
from __future__ import annotations

import numpy as np


def trapezoid_weights(y: np.ndarray) -> np.ndarray:
    """Weights w_j with sum_j w_j f(y_j) = trapezoid integral of f over [y_0, y_{n-1}]."""
    y = np.asarray(y, dtype=np.float64)
    w = np.zeros_like(y)
    h = np.diff(y)
    w[:-1] += h / 2
    w[1:] += h / 2
    return w


def half_channel_weights(y: np.ndarray) -> np.ndarray:
    """Weights of the integral over y in [-1, 0] of the linear interpolant."""
    y = np.asarray(y, dtype=np.float64)
    w = np.zeros_like(y)
    for j in range(len(y) - 1):
        a, b = y[j], y[j + 1]
        if b <= 0.0:                      # whole interval in the lower half
            w[j] += (b - a) / 2
            w[j + 1] += (b - a) / 2
        elif a < 0.0:                     # the interval containing the centre, clipped at y = 0
            h = b - a
            t = (0.0 - a) / h             # fraction of the interval below the centre
            # integral over [a, 0] of f_a + (f_b - f_a) s / h, s from 0 to t h
            w[j] += h * (t - t * t / 2)
            w[j + 1] += h * (t * t / 2)
    return w


def plane_stats(u: np.ndarray):
    """Mean and rms over x and z of each component of u [c][y][z][x]:
    <u_c>(y_j) and u_c,rms(y_j) = sqrt(<(u_c - <u_c>)^2>)."""
    u = np.asarray(u, dtype=np.float64)
    mean = u.mean(axis=(2, 3))
    rms = np.sqrt(((u - mean[:, :, None, None]) ** 2).mean(axis=(2, 3)))
    return mean, rms


def error_field(a: np.ndarray, b: np.ndarray, y: np.ndarray, Lx: float, Lz: float, utau_a: float = 1.0,
                utau_b: float = 1.0) -> float:
    """Eq. 13 for one component: a, b [y][z][x] on the same grid;
    || a/utau_a - b/utau_b ||_V / || b/utau_b ||_V."""
    a = np.asarray(a, dtype=np.float64) / utau_a
    b = np.asarray(b, dtype=np.float64) / utau_b
    ny, nz, nx = b.shape
    dV = trapezoid_weights(y)[:, None, None] * (Lx / nx) * (Lz / nz)
    num = np.sum(dV * (a - b) ** 2)
    den = np.sum(dV * b ** 2)
    return float(np.sqrt(num) / np.sqrt(den))


def error_profile(pa: np.ndarray, pb: np.ndarray, y: np.ndarray, utau_a: float = 1.0, utau_b: float = 1.0) -> float:
    """Eq. 14 (mean profiles) or Eq. 15 (rms profiles): profiles on the same
    y nodes, integrated from the wall to the centre (lower half)."""
    w = half_channel_weights(y)
    pa = np.asarray(pa, dtype=np.float64) / utau_a
    pb = np.asarray(pb, dtype=np.float64) / utau_b
    return float(np.sqrt(np.sum(w * (pa - pb) ** 2)) / np.sqrt(np.sum(w * pb ** 2)))
