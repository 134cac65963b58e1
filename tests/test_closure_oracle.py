"""Pins of the FP64 closure reference (oracle/mlp.py).

* MLP gradients against central finite differences of the loss;
* the non-uniform three-point y-derivative is exact for quadratics, and the
  mirror ghosts give the right wall derivative for even and odd profiles
  (Eq. 8 parities);
* the gradient model equals the closed form for a single x-mode;
* the forward pass equals networks evaluated by hand (pre-activations 0 and
  +-ln 3, where sigma = 1/2, 3/4, 1/4), and a wrong activation or a
  transposed layer fails that evaluation;
* Adam equals the closed forms of its recursion (the sign step at t = 1, a
  constant gradient, two steps written out), and a missing bias correction or
  swapped moment rates fail them.
"""
import math

import numpy as np
import pytest

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


# --- the forward pass against a network evaluated by hand -------------------
#
# silu(z) = z sigma(z) with sigma(ln 3) = 3/4 and sigma(-ln 3) = 1/4, so a
# chain whose pre-activations are 0 and +-ln 3 has a closed-form output.

L3 = math.log(3.0)


def _chain():
    """1 -> 1 -> 1 -> 1 -> 1: z1 = ln3 x, z2 = (4/3) h1, z3 = -(4/3) h2, y = 4 h3 + 1."""
    return [(np.array([[L3]]), np.array([0.0])), (np.array([[4.0 / 3.0]]), np.array([0.0])),
            (np.array([[-4.0 / 3.0]]), np.array([0.0])), (np.array([[4.0]]), np.array([1.0]))]


def _chain_closed_form(x):
    """x = 1: h1 = (3/4) ln3, z2 = ln3, h2 = (3/4) ln3, z3 = -ln3, h3 = -(1/4) ln3,
    y = 1 - ln 3.  x = 0: every pre-activation is 0, y = 1."""
    return {1.0: 1.0 - L3, 0.0: 1.0}[x]


def _wide():
    """2 -> 2 -> 1 -> 1 -> 2 with an asymmetric first layer: for x = (1, 0),
    z1 = W x = (ln3, ln3) (W^T x would give (ln3, 0)), h1 = (3/4 ln3, 3/4 ln3),
    z2 = (2/3)(h1_0 + h1_1) = ln3, z3 = -ln3, h3 = -(1/4) ln3,
    y = (4 h3 + 1/2, -8 h3 - 1) = (1/2 - ln3, 2 ln3 - 1)."""
    W1 = np.array([[L3, 0.0], [L3, 0.0]])
    W2 = np.array([[2.0 / 3.0, 2.0 / 3.0]])          # z2 = (2/3)(3/2 ln3) = ln3
    W3 = np.array([[-4.0 / 3.0]])                    # z3 = -ln3, h3 = -(1/4) ln3
    W4 = np.array([[4.0], [-8.0]])                   # y = (-ln3 + 0.5, 2 ln3 - 1)
    return [(W1, np.zeros(2)), (W2, np.zeros(1)), (W3, np.zeros(1)), (W4, np.array([0.5, -1.0]))]


def test_forward_matches_hand_evaluation():
    for x in (1.0, 0.0):
        Y, _ = M.forward(_chain(), np.array([[x]]))
        assert abs(Y[0, 0] - _chain_closed_form(x)) < 1e-15
    Y, (Z, H) = M.forward(_wide(), np.array([[1.0, 0.0]]))
    assert np.abs(Z[0][0] - [L3, L3]).max() < 1e-15
    assert np.abs(Y[0] - [0.5 - L3, 2 * L3 - 1.0]).max() < 1e-15
    # the silu values the closed form relies on
    assert abs(M.silu(L3) - 0.75 * L3) < 4e-16 and abs(M.silu(-L3) + 0.25 * L3) < 4e-16


def _transposed_forward(params, X):
    """A plausible mistake: z = h W instead of z = h W^T (square layers only)."""
    H = np.asarray(X, dtype=np.float64)
    for l, (W, b) in enumerate(params):
        z = H @ W + b
        H = M.silu(z) if l < len(params) - 1 else z
    return H


@pytest.mark.parametrize("mistake", ["sigmoid", "tanh_gate", "no_gate", "transposed"])
def test_planted_forward_mistakes_fail(mistake, monkeypatch):
    """Each planted mistake in the forward pass breaks the hand evaluation."""
    if mistake == "transposed":
        Y = _transposed_forward(_wide()[:1] + [(np.eye(2), np.zeros(2))], np.array([[1.0, 0.0]]))
        ref, _ = M.forward(_wide()[:1] + [(np.eye(2), np.zeros(2))], np.array([[1.0, 0.0]]))
        assert np.abs(Y - ref).max() > 1e-3
        return
    wrong = {"sigmoid": lambda z: 1.0 / (1.0 + np.exp(-z)),
             "tanh_gate": lambda z: z * np.tanh(z),
             "no_gate": lambda z: z}[mistake]
    monkeypatch.setattr(M, "silu", wrong)
    Y, _ = M.forward(_chain(), np.array([[1.0]]))
    assert abs(Y[0, 0] - _chain_closed_form(1.0)) > 1e-3


# --- Adam against closed forms of its recursion ------------------------------

def _scalar(w):
    return [(np.array([[w]]), np.array([0.0]))]


def _run_adam(gs, lr=0.1, w0=1.0, **kw):
    p = _scalar(w0)
    st = M.adam_init(p)
    for g in gs:
        p = M.adam_step(p, [(np.array([[g]]), np.array([0.0]))], st, lr, **kw)
    return p[0][0][0, 0]


def test_adam_first_step_is_sign_step():
    """t = 1: m_hat = g and v_hat = g^2 exactly, so the step is lr g / (|g| + eps)."""
    for g in (0.5, -3.0, 2e-4):
        assert abs(_run_adam([g]) - (1.0 - 0.1 * g / (abs(g) + 1e-8))) < 1e-15


def test_adam_constant_gradient():
    """Bias correction makes m_hat = g and v_hat = g^2 at every step of a
    constant gradient: k steps move w by k lr g / (|g| + eps)."""
    g = -0.37
    assert abs(_run_adam([g] * 7, lr=0.01) - (1.0 - 7 * 0.01 * g / (abs(g) + 1e-8))) < 1e-14


def test_adam_two_steps_closed_form():
    """After g1, g2: m_hat = (b1 g1 + g2) / (1 + b1), v_hat = (b2 g1^2 + g2^2) / (1 + b2)
    (the moving averages divided by 1 - b^2 = (1 - b)(1 + b))."""
    b1, b2, lr, g1, g2 = 0.9, 0.999, 0.05, 0.8, -0.3
    w1 = 1.0 - lr * g1 / (abs(g1) + 1e-8)
    mh = (b1 * g1 + g2) / (1 + b1)
    vh = (b2 * g1 * g1 + g2 * g2) / (1 + b2)
    assert abs(_run_adam([g1, g2], lr=lr) - (w1 - lr * mh / (math.sqrt(vh) + 1e-8))) < 1e-14


@pytest.mark.parametrize("mistake", ["no_bias_correction", "swapped_betas"])
def test_planted_adam_mistakes_fail(mistake, monkeypatch):
    b1, b2, lr, g1, g2 = 0.9, 0.999, 0.05, 0.8, -0.3
    mh = (b1 * g1 + g2) / (1 + b1)
    vh = (b2 * g1 * g1 + g2 * g2) / (1 + b2)
    ref = 1.0 - lr * g1 / (abs(g1) + 1e-8) - lr * mh / (math.sqrt(vh) + 1e-8)
    kw = {}
    if mistake == "no_bias_correction":
        monkeypatch.setattr(M, "bias_factors", lambda t, a, b: (1.0, 1.0))
    else:
        kw = {"beta1": b2, "beta2": b1}
    assert abs(_run_adam([g1, g2], lr=lr, **kw) - ref) > 1e-3
