"""FP64 reference of the learned subgrid closure: TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the CPU-baseline leg of the benchmark use
this module; the CUDA library never calls it.

The closure is the data-driven model the paper proposes as the use of the
exact stress (Sec. 2.1 and Sec. 5: DNS data inform SGS models, e.g. by machine
learning).  Its form follows the build's configuration: inputs are the nine
filtered velocity gradients d~bar(u_i)/dx_j on the LES grid and the wall
distance y+ = (1 - |y|) Re_tau; three hidden layers of width 128 with SiLU;
six outputs T_11, T_12, T_13, T_22, T_23, T_33; mean-squared error on
standardised inputs and targets.

Functions:
  * ``les_gradients``  -- second-order central differences on the LES grid:
    periodic in x and z; three-point non-uniform stencil in y with mirror
    ghosts of parity (+, -, +) at the walls (Eq. 8);
  * ``forward`` / ``backward`` -- the MLP and its exact gradients (written out
    layer by layer, no automatic differentiation);
  * ``adam_init`` / ``adam_step`` -- one update of the Adam method (Kingma and
    Ba, 2015: exponential moving averages of the gradient and of its square,
    each divided by its bias factor 1 - beta^t, step lr m_hat / (sqrt(v_hat)
    + eps)), the optimiser the library trains with;
  * ``gradient_model`` -- the second-moment (gradient) model
    T_ij ~ (Delta^2 / 12) d~bar(u_i)/dx_k d~bar(u_j)/dx_k, the baseline the
    learned closure is compared with.
"""
from __future__ import annotations

import numpy as np

WIDTHS = (10, 128, 128, 128, 6)
PAIRS = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_prime(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def init_params(seed: int, widths=WIDTHS):
    """He-style uniform initialisation (the same recipe the library uses)."""
    rng = np.random.default_rng(seed)
    params = []
    for fan_in, fan_out in zip(widths[:-1], widths[1:]):
        bound = np.sqrt(6.0 / fan_in) * 0.5
        W = rng.uniform(-bound, bound, size=(fan_out, fan_in))
        b = np.zeros(fan_out)
        params.append((W, b))
    return params


def forward(params, X):
    """X [N, 10] -> (Y [N, 6], cache of pre-activations and activations)."""
    H = [np.asarray(X, dtype=np.float64)]
    Z = []
    for l, (W, b) in enumerate(params):
        z = H[-1] @ W.T + b
        Z.append(z)
        H.append(silu(z) if l < len(params) - 1 else z)
    return H[-1], (Z, H)


def mse(Y, T):
    return float(np.mean((Y - T) ** 2))


def backward(params, cache, Y, T):
    """Gradients of mse(Y, T) = mean over all N * 6 entries."""
    Z, H = cache
    N = Y.shape[0]
    dY = 2.0 * (Y - T) / (N * Y.shape[1])
    grads = [None] * len(params)
    d = dY
    for l in range(len(params) - 1, -1, -1):
        W, b = params[l]
        grads[l] = (d.T @ H[l], d.sum(axis=0))
        if l > 0:
            d = (d @ W) * silu_prime(Z[l - 1])
    return grads


def adam_init(params):
    """Zero first and second moments and step count 0 for ``params``."""
    return {"t": 0,
            "m": [[np.zeros_like(W), np.zeros_like(b)] for W, b in params],
            "v": [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]}


def bias_factors(t, beta1, beta2):
    """Adam's bias factors 1 - beta1^t and 1 - beta2^t after t steps."""
    return 1.0 - beta1 ** t, 1.0 - beta2 ** t


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in FP64; returns the new parameters (``state`` is
    updated in place).  With t the new step count:
      m <- beta1 m + (1 - beta1) g,   v <- beta2 v + (1 - beta2) g^2,
      w <- w - lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps)."""
    state["t"] += 1
    c1, c2 = bias_factors(state["t"], beta1, beta2)
    out = []
    for l, (wb, gb) in enumerate(zip(params, grads)):
        new = []
        for k in range(2):
            w, g = wb[k], gb[k]
            m = beta1 * state["m"][l][k] + (1.0 - beta1) * g
            v = beta2 * state["v"][l][k] + (1.0 - beta2) * g * g
            state["m"][l][k], state["v"][l][k] = m, v
            new.append(w - lr * (m / c1) / (np.sqrt(v / c2) + eps))
        out.append(tuple(new))
    return out


def les_gradients(ub, les, parity=(1, -1, 1)):
    """d ub_i / d x_j on the LES grid: [3 (i)][3 (j: x, y, z)][nly][nlz][nlx]."""
    ub = np.asarray(ub, dtype=np.float64)
    hx, hz = les.Lx / les.nx, les.Lz / les.nz
    y = les.y
    g = np.zeros((3, 3) + ub.shape[1:])
    for i in range(3):
        f = ub[i]
        g[i, 0] = (np.roll(f, -1, axis=2) - np.roll(f, 1, axis=2)) / (2 * hx)
        g[i, 2] = (np.roll(f, -1, axis=1) - np.roll(f, 1, axis=1)) / (2 * hz)
        ny = len(y)
        for J in range(ny):
            if 0 < J < ny - 1:
                hp, hm = y[J + 1] - y[J], y[J] - y[J - 1]
                fp, fm = f[J + 1], f[J - 1]
            elif J == 0:
                hp = hm = y[1] - y[0]
                fp, fm = f[1], parity[i] * f[1]
            else:
                hp = hm = y[-1] - y[-2]
                fp, fm = parity[i] * f[-2], f[-2]
            g[i, 1, J] = (hm * hm * (fp - f[J]) + hp * hp * (f[J] - fm)) / (hp * hm * (hp + hm))
    return g


def features(ub, les, re_tau=180.0):
    """[N, 10]: the nine gradients (i-major, j = x, y, z) and y+, N = nly*nlz*nlx."""
    g = les_gradients(ub, les)
    n = ub.shape[1] * ub.shape[2] * ub.shape[3]
    F = np.empty((n, 10))
    for i in range(3):
        for j in range(3):
            F[:, 3 * i + j] = g[i, j].reshape(-1)
    yp = (1.0 - np.abs(les.y)) * re_tau
    F[:, 9] = np.broadcast_to(yp[:, None, None], ub.shape[1:]).reshape(-1)
    return F


def gradient_model(ub, les, delta):
    g = les_gradients(ub, les)
    out = np.empty((6,) + ub.shape[1:])
    for q, (i, j) in enumerate(PAIRS):
        out[q] = delta * delta / 12.0 * sum(g[i, k] * g[j, k] for k in range(3))
    return out
