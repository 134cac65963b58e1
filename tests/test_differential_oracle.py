"""Pins of the FP64 differential-filter reference (oracle/differential.py).

The differential filter of Sec. 3 solves (1 - a^2 lap) ubar = u on the
extended domain.  Each check below is fixed by the mathematics, not by the
reference itself, and a plausible slip (a wrong wall row, a missing factor 2
in the non-uniform stencil, the wrong modified wavenumber, a transposed axis,
a parity not applied) breaks one of them:
  * the FFT-and-Thomas solver equals a direct sparse solve of the whole system
    (two independent implementations of the same equations), both parities,
    grids with factors 2 and 3;
  * applying the stencil operator to the result returns the input;
  * closed form on a uniform y grid: a separable mode cos(kx x) cos(kz z)
    cos(pi m j / (ny - 1)) (even) or ... sin(...) (odd) is an eigenvector and
    is damped by exactly 1 / (1 + a^2 (kx~^2 + kz~^2 + ky~^2)) with
    k~^2 = (2 - 2 cos(k h)) / h^2;
  * a constant is preserved; the filter is positive (an M-matrix inverse),
    so T_ij is positive semi-definite;
  * a = 0.1 (the paper's value) corresponds to Delta_f = sqrt(40) / 10.
"""
import math

import numpy as np
import pytest

from oracle import differential as D
from paper_1902_02508_gb300 import inputs as I

pytest.importorskip("scipy")


def _field(ny, nz, nx, seed):
    return np.random.default_rng(seed).standard_normal((ny, nz, nx))


@pytest.mark.parametrize("shape", [(9, 6, 8), (7, 4, 12), (11, 9, 6)])
@pytest.mark.parametrize("parity", [1, -1])
def test_fft_solver_equals_sparse_solve(shape, parity):
    ny, nz, nx = shape
    y = I.tanh_nodes(ny)
    u = _field(ny, nz, nx, 5 + ny)
    a = 0.3
    ref = D.filter_sparse(u, y, 2 * math.pi, math.pi, a, parity)
    got = D.filter_fft(u, y, 2 * math.pi, math.pi, a, parity)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("parity", [1, -1])
def test_operator_inverts_filter(parity):
    ny, nz, nx = 17, 12, 16
    y = I.tanh_nodes(ny)
    u = _field(ny, nz, nx, 3)
    a = 0.15
    v = D.filter_fft(u, y, 4 * math.pi, 2 * math.pi, a, parity)
    back = D.apply_operator(v, y, 4 * math.pi, 2 * math.pi, a, parity)
    if parity < 0:
        u = u.copy()
        u[0] = 0.0
        u[-1] = 0.0
        assert np.abs(v[0]).max() == 0.0 and np.abs(v[-1]).max() == 0.0
    assert np.abs(back - u).max() <= 1e-12 * np.abs(u).max()


@pytest.mark.parametrize("parity", [1, -1])
def test_separable_mode_closed_form(parity):
    ny, nz, nx = 13, 8, 12
    Lx, Lz = 2 * math.pi, math.pi
    y = np.linspace(-1.0, 1.0, ny)
    hy, hx, hz = 2.0 / (ny - 1), Lx / nx, Lz / nz
    x = np.arange(nx) * hx
    z = np.arange(nz) * hz
    jj = np.arange(ny)
    mx, mz, m = 3, 2, 5
    kx, kz = 2 * math.pi * mx / Lx, 2 * math.pi * mz / Lz
    ymode = np.cos(math.pi * m * jj / (ny - 1)) if parity > 0 else np.sin(math.pi * m * jj / (ny - 1))
    u = ymode[:, None, None] * np.cos(kz * z)[None, :, None] * np.cos(kx * x)[None, None, :]
    a = 0.2
    k2 = ((2 - 2 * math.cos(kx * hx)) / hx ** 2 + (2 - 2 * math.cos(kz * hz)) / hz ** 2
          + (2 - 2 * math.cos(math.pi * m / (ny - 1))) / hy ** 2)
    got = D.filter_fft(u, y, Lx, Lz, a, parity)
    assert np.abs(got - u / (1 + a * a * k2)).max() <= 1e-13


def test_constant_preserved_and_positive():
    ny, nz, nx = 15, 6, 12
    y = I.tanh_nodes(ny)
    c = np.full((ny, nz, nx), 2.5)
    assert np.abs(D.filter_fft(c, y, 2 * math.pi, math.pi, 0.4, 1) - 2.5).max() <= 1e-13
    pulse = np.zeros((ny, nz, nx))
    pulse[6, 2, 5] = 1.0
    for p in (1, -1):
        g = D.filter_fft(pulse, y, 2 * math.pi, math.pi, 0.4, p)
        assert g.min() >= -1e-15 and abs(g.max()) > 0


def test_tau_psd_and_filter_parameter():
    assert abs(D.filter_parameter(math.sqrt(40.0) / 10) - 0.1) < 1e-15
    dns = I.dns_grid(16, 17, 12, 2 * math.pi, math.pi)
    les = I.les_grid(dns, 8, 9, 6)
    u = I.channel_velocity(dns, 11)
    ub, tau = D.subfilter_stress(dns, les, 0.5, u)
    T = np.empty(tau.shape[1:] + (3, 3))
    for q, (i, j) in enumerate(D.PAIRS):
        T[..., i, j] = tau[q]
        T[..., j, i] = tau[q]
    assert np.linalg.eigvalsh(T.reshape(-1, 3, 3)).min() >= -1e-12 * np.abs(tau).max()
    # Eq. 8: the odd component vanishes on the walls
    assert np.abs(ub[1, 0]).max() == 0.0 and np.abs(ub[1, -1]).max() == 0.0
    # the sparse and FFT solvers give the same stress
    ub2, tau2 = D.subfilter_stress(dns, les, 0.5, u, solver=D.filter_sparse)
    assert np.abs(tau2 - tau).max() <= 1e-11 * np.abs(tau).max()
