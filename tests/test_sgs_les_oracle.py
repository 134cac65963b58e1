"""Pins of the LES-step oracle (oracle/les.py) against closed forms and the
mathematics of the projection (Sec. 3 and Fig. 2: the explicitly filtered LES
advanced with the exact T_ij of Eq. 6).

  * the projection: the per-mode form equals the dense physical-space form;
    it returns a discretely divergence-free field unchanged, annihilates
    discrete gradients of potentials that vanish on the walls, and leaves
    zero divergence (the Hodge split it must perform);
  * laminar Poiseuille flow under the mean pressure gradient is a steady
    state of the step (the stencils are exact for quadratics), and so is a
    Couette profile between wall values given by Eq. 10;
  * a single wall-bounded mode with no advection decays by the third-order
    Runge-Kutta amplification 1 + z + z^2/2 + z^3/6 (z = nu dt lambda, lambda
    the closed-form eigenvalue of the three-point operators), and by 1 + z
    for the Euler scheme;
  * the right-hand side of a two-component field equals its closed form on a
    uniform grid (advection, viscosity, forcing);
  * the subfilter term: a wall-normal gradient of T_12 (T_23) drives u_1
    (u_3) alone, by the central difference of the profile; a T_22 profile
    that vanishes on the walls is balanced by the pressure entirely; a
    constant T_ij does nothing;
  * the loop of Fig. 2: two steps are one step twice (no hidden state), each
    step takes its own snapshot's T_ij and wall values.
"""
import math

import numpy as np
import pytest

from oracle import les as L
from paper_1902_02508_gb300 import inputs as I


def grid(nx, ny, nz, Lx=2 * math.pi, Lz=math.pi, uniform=False):
    g = I.dns_grid(nx, ny, nz, Lx, Lz)
    if uniform:
        g = I.Grid(nx, ny, nz, Lx, Lz, np.linspace(-1.0, 1.0, ny))
    return g


def rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300)


def interior_y_diff(f, y):
    out = np.zeros_like(f)
    out[1:-1] = (f[2:] - f[:-2]) / (y[2:] - y[:-2])[:, None, None]
    return out


def periodic_diff(f, h, axis):
    return (np.roll(f, -1, axis) - np.roll(f, 1, axis)) / (2 * h)


def test_projection_forms_agree():
    g = grid(8, 9, 6)
    rng = np.random.default_rng(3)
    u = rng.standard_normal((3, g.ny, g.nz, g.nx))
    u[:, 0] = u[:, -1] = 0.0
    a = L.project(u, g)
    b = L.project_dense(u, g)
    assert rel(a, b) < 1e-12
    assert np.max(np.abs(L.divergence(a, g))) < 1e-11 * np.max(np.abs(u))


@pytest.mark.parametrize("shape", [(16, 13, 12), (12, 10, 9)])
def test_projection_is_the_hodge_split(shape):
    """u* = w + G phi0 with D w = 0 and phi0 = 0 on the walls: P u* = w."""
    nx, ny, nz = shape
    g = grid(nx, ny, nz)
    y = np.asarray(g.y)
    hx, hz = g.Lx / nx, g.Lz / nz
    rng = np.random.default_rng(11)
    # solenoidal part from two stream functions vanishing on the walls
    psi_a = rng.standard_normal((ny, nz, nx))
    psi_b = rng.standard_normal((ny, nz, nx))
    psi_a[0] = psi_a[-1] = 0.0
    psi_b[0] = psi_b[-1] = 0.0
    w = np.zeros((3, ny, nz, nx))
    w[0] = interior_y_diff(psi_a, y) + periodic_diff(psi_b, hz, 1)
    w[1] = -periodic_diff(psi_a, hx, 2)
    w[2] = -periodic_diff(psi_b, hx, 2)
    w[:, 0] = w[:, -1] = 0.0
    assert np.max(np.abs(L.divergence(w, g))) < 1e-12 * np.max(np.abs(w))
    # gradient part
    phi = rng.standard_normal((ny, nz, nx))
    phi[0] = phi[-1] = 0.0
    gp = np.zeros((3, ny, nz, nx))
    gp[0] = periodic_diff(phi, hx, 2)
    gp[1] = interior_y_diff(phi, y)
    gp[2] = periodic_diff(phi, hz, 1)
    gp[:, 0] = gp[:, -1] = 0.0
    assert rel(L.project(w, g), w) < 1e-12
    assert np.max(np.abs(L.project(gp, g))) < 1e-12 * np.max(np.abs(gp))
    assert rel(L.project(w + gp, g), w) < 1e-12
    # any field: zero divergence after the projection, and P P = P
    u = rng.standard_normal((3, ny, nz, nx))
    u[:, 0] = u[:, -1] = 0.0
    pu = L.project(u, g)
    assert np.max(np.abs(L.divergence(pu, g))) < 1e-11 * np.max(np.abs(u))
    assert rel(L.project(pu, g), pu) < 1e-12


@pytest.mark.parametrize("scheme", ["rk3", "euler"])
def test_couette_with_wall_values_is_steady(scheme):
    """Eq. 10: the wall rows of u_1 and u_3 come from the given field; a
    linear profile between them is steady (no forcing)."""
    g = grid(8, 13, 6)
    y = np.asarray(g.y)
    u = np.zeros((3, g.ny, g.nz, g.nx))
    u[0] = (0.4 + 1.5 * y)[:, None, None]
    u[2] = (-0.2 + 0.7 * y)[:, None, None]
    u[1, 1:-1] = 0.0
    start = np.array(u)
    start[:, 0] = start[:, -1] = 0.0           # the step sets the walls itself
    out = L.step(start, None, g, nu=0.02, dt=0.1, forcing=0.0, scheme=scheme, ubc=u)
    assert rel(out, u) < 1e-13
    # and u_2 on the walls is zero whatever the given field holds
    bc = np.array(u)
    bc[1] = 5.0
    out = L.step(start, None, g, nu=0.02, dt=0.1, forcing=0.0, scheme=scheme, ubc=bc)
    assert rel(out, u) < 1e-13


@pytest.mark.parametrize("scheme", ["rk3", "euler"])
def test_poiseuille_is_steady(scheme):
    g = grid(8, 17, 6)
    nu, Pi = 1.0 / 180.0, 1.0
    y = np.asarray(g.y)
    u = np.zeros((3, g.ny, g.nz, g.nx))
    u[0] = (Pi / (2 * nu) * (1 - y * y))[:, None, None]
    out = L.step(u, None, g, nu, dt=0.05, forcing=Pi, scheme=scheme)
    assert rel(out, u) < 1e-13


@pytest.mark.parametrize("scheme,amp", [("rk3", lambda z: 1 + z + z * z / 2 + z ** 3 / 6), ("euler", lambda z: 1 + z)])
def test_single_mode_decays_by_the_scheme_amplification(scheme, amp):
    nx, ny, nz = 8, 17, 12
    g = grid(nx, ny, nz, uniform=True)
    y = np.asarray(g.y)
    hy, hz = 2.0 / (ny - 1), g.Lz / nz
    kz, m = 2 * 2 * math.pi / g.Lz, 3
    z = np.arange(nz) * hz
    prof = np.sin(m * math.pi * (y + 1) / 2)
    prof[0] = prof[-1] = 0.0
    u = np.zeros((3, ny, nz, nx))
    u[0] = prof[:, None, None] * np.sin(kz * z)[None, :, None]
    lam = -(2 - 2 * math.cos(kz * hz)) / hz ** 2 - (2 - 2 * math.cos(m * math.pi * hy / 2)) / hy ** 2
    nu, dt = 0.05, 0.6
    zz = nu * dt * lam
    assert -2.0 < zz < -0.5          # the cubic term matters at this step size
    out = L.step(u, None, g, nu, dt, forcing=0.0, scheme=scheme)
    assert rel(out, amp(zz) * u) < 1e-12


def test_rhs_closed_form_uniform_grid():
    nx, ny, nz = 16, 21, 8
    g = grid(nx, ny, nz, uniform=True)
    y = np.asarray(g.y)[:, None, None]
    h = 2.0 / (ny - 1)
    hx = g.Lx / nx
    k = 2 * math.pi / g.Lx
    x = (np.arange(nx) * hx)[None, None, :]
    c, nu, Pi = 0.7, 0.03, 1.3
    u = np.zeros((3, ny, nz, nx))
    u[0] = np.sin(k * x) * (1 - y * y) * np.ones((1, nz, 1))
    u[1] = c * (1 - y * y) * np.ones((1, nz, nx))
    R = L.rhs(u, None, g, nu, Pi)
    q = -4 * y + 4 * y ** 3 + 4 * y * h * h            # central difference of (1 - y^2)^2 on the uniform grid
    e1 = (-(1 - y * y) ** 2 * np.sin(2 * k * x) * math.sin(2 * k * hx) / (2 * hx)
          - c * np.sin(k * x) * q
          + nu * np.sin(k * x) * ((2 * math.cos(k * hx) - 2) / hx ** 2 * (1 - y * y) - 2.0) + Pi)
    e2 = -c * (1 - y * y) ** 2 * np.cos(k * x) * math.sin(k * hx) / hx - c * c * q + nu * c * (-2.0)
    e1 = e1 * np.ones((1, nz, 1))
    e2 = e2 * np.ones((1, nz, 1))
    assert rel(R[0, 1:-1], e1[1:-1]) < 1e-13
    assert rel(R[1, 1:-1], e2[1:-1]) < 1e-13
    assert np.max(np.abs(R[2])) == 0.0
    assert np.all(R[:, 0] == 0.0) and np.all(R[:, -1] == 0.0)


def test_subfilter_term_enters_by_its_divergence():
    g = grid(8, 15, 6)
    y = np.asarray(g.y)
    shape = (g.ny, g.nz, g.nx)
    dt = 0.1
    zero = np.zeros((3,) + shape)
    f = (y ** 3 + 0.3 * y + 0.2)[:, None, None] * np.ones(shape)
    df = np.zeros(shape)
    df[1:-1] = (f[2:] - f[:-2]) / (y[2:] - y[:-2])[:, None, None]
    for pair, comp in ((1, 0), (4, 2)):           # T_12 drives u_1, T_23 drives u_3
        tau = np.zeros((6,) + shape)
        tau[pair] = f
        out = L.step(zero, tau, g, nu=0.01, dt=dt, forcing=0.0, scheme="euler")
        expect = np.zeros((3,) + shape)
        expect[comp] = -dt * df
        assert rel(out, expect) < 1e-13
    # a wall-normal stress vanishing on the walls is a pressure gradient
    tau = np.zeros((6,) + shape)
    tau[3] = ((1 - y * y) * (2 + y))[:, None, None] * np.ones(shape)
    out = L.step(zero, tau, g, nu=0.01, dt=dt, forcing=0.0, scheme="euler")
    assert np.max(np.abs(out)) < 1e-13
    # a constant stress does nothing
    rng = np.random.default_rng(5)
    u0 = rng.standard_normal((3,) + shape) * 0.1
    u0 = L.project(u0, g)
    tau = np.ones((6,) + shape) * np.array([0.3, -0.1, 0.05, 0.2, 0.4, -0.25])[:, None, None, None]
    a = L.step(u0, tau, g, nu=0.01, dt=0.01, forcing=1.0, scheme="rk3")
    b = L.step(u0, None, g, nu=0.01, dt=0.01, forcing=1.0, scheme="rk3")
    assert rel(a, b) < 1e-13


def test_loop_takes_each_snapshot_at_its_own_step():
    """Fig. 2: the loop over snapshots A, B is the loop over A followed by the
    loop over B (no state beyond the LES field), each step uses its own
    snapshot's T_ij and wall values (the order matters), and a one-snapshot
    loop is one step with that snapshot's filter output."""
    from oracle import oracle as O
    dns = I.dns_grid(32, 33, 32, 2 * math.pi, math.pi)
    les = I.les_grid(dns, 8, 9, 8)
    delta = 2 * math.pi / 16
    A, B, C = (I.channel_velocity(dns, 1000 + s) for s in range(3))
    u0, _ = O.subfilter_stress(dns, les, delta, C)
    nu, dt = 1.0 / 180.0, 0.002
    ab, taus = L.apost_run(dns, les, delta, [A, B], u0, nu, dt)
    a, _ = L.apost_run(dns, les, delta, [A], u0, nu, dt)
    a_b, _ = L.apost_run(dns, les, delta, [B], a, nu, dt)
    assert rel(ab, a_b) < 1e-15
    ba, _ = L.apost_run(dns, les, delta, [B, A], u0, nu, dt)
    assert rel(ba, ab) > 1e-6
    ubar_a, tau_a = O.subfilter_stress(dns, les, delta, A)
    assert np.array_equal(taus[0], tau_a)
    assert rel(a, L.step(u0, tau_a, les, nu, dt, ubc=ubar_a)) < 1e-15
