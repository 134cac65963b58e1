"""Pins of the FP64 error measures of Sec. 4 (oracle/metrics.py).

Each check is a closed form or an invariant that a plausible slip (a wrong
weight, a missing square root, the wrong half of the channel, u_tau applied
to one field only) would break:
  * y quadrature: total length 2; integral of y^2 within the trapezoid bound;
  * wall-to-centre quadrature: length 1 and exact for linear integrands,
    with and without a node at the centre;
  * plane statistics: mean of U(y) + A sin(k x) is U, rms is A / sqrt(2);
  * Eq. 13: (1 + eps) b against b gives eps; b = 1 against 1 + eps cos(k x)
    gives eps / sqrt(2); scaling both fields or their u_tau consistently
    changes nothing;
  * Eq. 14 / 15: a constant offset c against a unit profile gives c;
    profiles that differ only in the upper half give 0.
"""
import math

import numpy as np

from oracle import metrics as M
from paper_1902_02508_gb300 import inputs as I


def test_trapezoid_weights():
    for ny in (9, 33, 64):
        y = I.tanh_nodes(ny)
        w = M.trapezoid_weights(y)
        assert abs(w.sum() - 2.0) < 1e-14
        h = np.diff(y).max()
        assert abs(np.sum(w * y * y) - 2.0 / 3.0) <= 2.0 * h * h * 2.0 / 12.0 + 1e-15


def test_half_channel_weights_exact_for_linear():
    for ny in (9, 32, 33, 64):                      # odd: a node at the centre; even: none
        y = I.tanh_nodes(ny)
        w = M.half_channel_weights(y)
        assert abs(w.sum() - 1.0) < 1e-14
        assert abs(np.sum(w * (3.0 + 2.0 * y)) - 2.0) < 1e-13      # int_{-1}^0 (3 + 2y) dy
        assert np.all(w[y > 0] == 0.0) or ny % 2 == 0              # only the clipped interval reaches y > 0
        assert np.all(w[np.searchsorted(y, 0.0, side="right") + 1:] == 0.0)


def test_plane_stats_single_mode():
    ny, nz, nx = 7, 12, 16
    y = I.tanh_nodes(ny)
    x = np.arange(nx) * 2 * math.pi / nx
    U = 5.0 + y * y
    A = 0.7
    u = np.zeros((3, ny, nz, nx))
    u[0] = U[:, None, None] + A * np.sin(3 * x)[None, None, :]
    u[2] = -2.0
    mean, rms = M.plane_stats(u)
    assert np.abs(mean[0] - U).max() < 1e-14
    assert np.abs(rms[0] - A / math.sqrt(2)).max() < 1e-14
    assert np.abs(mean[2] + 2.0).max() < 1e-15 and np.abs(rms[2]).max() < 1e-15


def test_error_field_closed_forms():
    rng = np.random.default_rng(4)
    ny, nz, nx = 9, 8, 12
    y = I.tanh_nodes(ny)
    b = rng.standard_normal((ny, nz, nx)) + 3.0
    eps = 0.01
    assert abs(M.error_field((1 + eps) * b, b, y, 2 * math.pi, math.pi) - eps) < 1e-14
    # u_tau divides each field: 2b with u_tau 2 is b
    assert M.error_field(2 * b, b, y, 1.0, 1.0, utau_a=2.0, utau_b=1.0) < 1e-15
    # a common scale of both fields and their u_tau leaves the error unchanged
    a = b + 0.1 * rng.standard_normal(b.shape)
    e = M.error_field(a, b, y, 1.0, 1.0)
    assert abs(M.error_field(4 * a, 4 * b, y, 3.0, 5.0, 4.0, 4.0) - e) < 1e-14
    # one x mode: || eps cos ||_V / || 1 ||_V = eps / sqrt(2)
    x = np.arange(nx) * 2 * math.pi / nx
    one = np.ones((ny, nz, nx))
    assert abs(M.error_field(one + eps * np.cos(2 * x)[None, None, :], one, y, 2 * math.pi, math.pi)
               - eps / math.sqrt(2)) < 1e-14


def test_error_profile_closed_forms():
    for ny in (33, 64):
        y = I.tanh_nodes(ny)
        pb = np.ones(ny)
        assert abs(M.error_profile(pb + 0.2, pb, y) - 0.2) < 1e-14
        upper = np.where(y > 0, 1.0, 0.0)
        if ny % 2 == 1:                              # the centre is a node: the upper half is not seen
            assert M.error_profile(pb + upper, pb, y) == 0.0
        assert abs(M.error_profile(3 * pb, 2 * pb, y, utau_a=3.0, utau_b=2.0)) < 1e-15
