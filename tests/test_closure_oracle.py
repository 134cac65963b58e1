"""Pins of the FP64 closure reference (oracle/mlp.py).

* MLP gradients against central finite differences of the loss;
* the non-uniform three-point y-derivative is exact for quadratics, and the
  mirror ghosts give the right wall derivative for even and odd profiles
  (Eq. 8 parities);
* the gradient model equals the closed form for a single x-mode.
"""
import math

import numpy as np

from oracle import mlp as M
from paper_1902_02508_gb300 import inputs as I


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    widths = (10, 7, 6, 5, 6)
    params = M.init_params(3, widths)
    params = [(W, rng.standard_normal(b.shape) * 0.1) for W, b in params]
    X = rng.standard_normal((13, 10))
    T = rng.standard_normal((13, 6))
    Y, cache = M.forward(params, X)
    grads = M.backward(params, cache, Y, T)
    eps = 1e-6
    worst = 0.0
    for l, (W, b) in enumerate(params):
        for arr, g in ((W, grads[l][0]), (b, grads[l][1])):
            for idx in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(6)]:
                old = arr[idx]
                arr[idx] = old + eps
                lp = M.mse(M.forward(params, X)[0], T)
                arr[idx] = old - eps
                lm = M.mse(M.forward(params, X)[0], T)
                arr[idx] = old
                fd = (lp - lm) / (2 * eps)
                worst = max(worst, abs(fd - g[idx]) / max(abs(fd), 1e-3))
    assert worst < 1e-6


def test_silu_prime_is_derivative():
    z = np.linspace(-6, 6, 101)
    fd = (M.silu(z + 1e-6) - M.silu(z - 1e-6)) / 2e-6
    assert np.abs(fd - M.silu_prime(z)).max() < 1e-8


def test_y_derivative_exact_for_quadratics_and_wall_parity():
    d = I.dns_grid(16, 33, 12, 2 * math.pi, math.pi)
    les = I.les_grid(d, 8, 9, 6)
    y = les.y
    ub = np.zeros((3, les.ny, les.nz, les.nx))
    ub[0] = (1 - y * y)[:, None, None] ** 1 * 1.0 + 0.3 * y[:, None, None] ** 2   # even
    ub[1] = (y * (1 - y * y))[:, None, None]                                      # odd
    ub[2] = (2.0 + y * y)[:, None, None]                                          # even
    g = M.les_gradients(ub, les)
    # interior: exact for quadratics (ub[0], ub[2]); walls: even -> 0
    exact0 = (-2 * y + 0.6 * y)[:, None, None]
    assert np.abs(g[0, 1][1:-1] - exact0[1:-1]).max() < 1e-12
    assert np.abs(g[2, 1][1:-1] - (2 * y)[1:-1, None, None]).max() < 1e-12
    assert np.abs(g[0, 1][[0, -1]]).max() < 1e-14 and np.abs(g[2, 1][[0, -1]]).max() < 1e-14
    # odd profile: the mirror ghost makes the wall derivative f(y1)/h ~ f'(wall)
    h = y[1] - y[0]
    assert abs(g[1, 1][0, 0, 0] - ub[1][1, 0, 0] / h) < 1e-14


def test_gradient_model_single_mode():
    d = I.dns_grid(64, 17, 8, 2 * math.pi, math.pi)
    les = I.les_grid(d, 32, 9, 8)
    X = np.arange(les.nx) * les.Lx / les.nx
    ub = np.zeros((3, les.ny, les.nz, les.nx))
    ub[0] = np.sin(2 * X)[None, None, :]
    gm = M.gradient_model(ub, les, 0.3)
    hx = les.Lx / les.nx
    dudx = (np.sin(2 * (X + hx)) - np.sin(2 * (X - hx))) / (2 * hx)
    assert np.abs(gm[0] - 0.09 / 12 * dudx[None, None, :] ** 2).max() < 1e-14
    assert np.abs(gm[1:]).max() == 0.0


def test_features_layout():
    d = I.dns_grid(16, 17, 12, 2 * math.pi, math.pi)
    les = I.les_grid(d, 8, 9, 6)
    ub = np.random.default_rng(1).standard_normal((3, les.ny, les.nz, les.nx))
    F = M.features(ub, les)
    assert F.shape == (les.ny * les.nz * les.nx, 10)
    assert np.allclose(F[:, 9].reshape(les.ny, les.nz, les.nx)[:, 0, 0], (1 - np.abs(les.y)) * 180)
