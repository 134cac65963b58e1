"""Pins of the CPU oracle to facts the paper and the mathematics fix.

None of these checks re-types the oracle's own formulas: each compares it with
a closed form (the Gaussian transfer function, Poisson summation), an
invariant the paper states (Eq. 7 keeps a solenoidal field solenoidal, Eq. 8
parity of the filtered field, normalisation of Eq. 2), the algebra of T_ij
(symmetry, positive semi-definiteness, Galilean invariance in x and z, the
closed form for single Fourier modes), or a brute-force third evaluation on
tiny grids with the extended field written out node by node.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1902_02508_gb300 import inputs as I


def gauss_hat(k, delta):
    return np.exp(-(k * delta) ** 2 / 24.0)


def poisson_response(k, delta, h, M=8):
    """Response of the sampled, row-normalised Gaussian at lattice nodes."""
    m = np.arange(-M, M + 1)
    return gauss_hat(k + 2 * np.pi * m / h, delta).sum() / gauss_hat(2 * np.pi * m / h, delta).sum()


def uniform_y(n):
    return np.linspace(-1.0, 1.0, n)


# ----------------------------------------------------------------- Eq. 2 ----
@pytest.mark.parametrize("n,nl,L,dfrac", [(32, 8, 2 * math.pi, 1 / 16), (64, 16, math.pi, 1 / 10),
                                          (96, 32, 4 * math.pi, 1 / 48)])
def test_periodic_rows_normalised_and_nonnegative(n, nl, L, dfrac):
    A = O.op_periodic(n, L, nl, dfrac * L)
    assert np.all(A >= 0)
    assert np.abs(A.sum(axis=1) - 1).max() < 1e-15


@pytest.mark.parametrize("n,L,delta_over_h", [(64, 2 * math.pi, 6.0), (96, math.pi, 8.0), (32, 2 * math.pi, 2.0)])
def test_periodic_transfer_function(n, L, delta_over_h):
    """cos(kx) comes out multiplied by the Poisson-summed Gaussian response;
    for delta/h >= 6 that equals exp(-k^2 delta^2 / 24) up to the first alias
    exp(-(2 pi / h - k)^2 delta^2 / 24)."""
    h = L / n
    delta = delta_over_h * h
    A = O.op_periodic(n, L, n, delta)
    x = np.arange(n) * h
    for m in (1, 3, 7, n // 4):
        k = 2 * np.pi * m / L
        got = A @ np.cos(k * x)
        R = poisson_response(k, delta, h)
        assert np.abs(got - R * np.cos(k * x)).max() < 2e-14
        if delta_over_h >= 6:
            alias = 2 * gauss_hat(2 * np.pi / h - k, delta)
            assert abs(R - gauss_hat(k, delta)) <= alias + 1e-17


def test_periodic_sampling_is_linear_interpolation():
    """Non-integer DNS/LES ratio: rows are interpolations of filtered rows."""
    n, L, nl = 40, 2 * math.pi, 12
    delta = L / 10
    F = O.op_periodic(n, L, n, delta)
    A = O.op_periodic(n, L, nl, delta)
    x = np.arange(n) * L / n
    f = np.sin(3 * x) + 0.3 * np.cos(5 * x)
    ff = F @ f
    for X in range(nl):
        pos = X * L / nl / (L / n)
        i0 = int(math.floor(pos + 1e-12))
        th = pos - i0
        want = (1 - th) * ff[i0 % n] + th * ff[(i0 + 1) % n]
        assert abs((A @ f)[X] - want) < 1e-13


# ------------------------------------------------------- Eq. 7 and Eq. 8 ----
@pytest.mark.parametrize("m", [1, 2, 5])
def test_wall_transfer_uniform_grid(m):
    """On a uniform y-grid the extended lattice is uniform: cos(m pi (y+1)) is
    even and sin(m pi (y+1)) odd about both walls, so each is an eigenfunction
    with the Gaussian response exp(-(m pi)^2 delta^2 / 24)."""
    n = 129
    y = uniform_y(n)
    h = y[1] - y[0]
    delta = 0.2
    k = m * np.pi
    R = poisson_response(k, delta, h)
    assert abs(R - gauss_hat(k, delta)) < 1e-20
    Ae = O.op_wall(y, y, delta, +1)
    Ao = O.op_wall(y, y, delta, -1)
    assert np.abs(Ae @ np.cos(k * (y + 1)) - R * np.cos(k * (y + 1))).max() < 1e-13
    assert np.abs(Ao @ np.sin(k * (y + 1)) - R * np.sin(k * (y + 1))).max() < 1e-13
    # With the wrong parity the wall rows are visibly wrong.
    assert np.abs(Ae @ np.sin(k * (y + 1)) - R * np.sin(k * (y + 1))).max() > 1e-3


def test_wall_transfer_stretched_grid_second_order():
    """On the tanh grid the trapezoid rule makes the response second order in h."""
    delta, k = 0.25, 2 * np.pi
    errs = []
    for n in (33, 65, 129, 257):
        y = I.tanh_nodes(n)
        A = O.op_wall(y, y, delta, +1)
        err = np.abs(A @ np.cos(k * (y + 1)) - gauss_hat(k, delta) * np.cos(k * (y + 1))).max()
        errs.append(err)
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(1.8 < r < 2.3 for r in rates[1:]), (errs, rates)


def test_wall_rows_even_normalised_odd_vanish_at_walls():
    y = I.tanh_nodes(65)
    Ae = O.op_wall(y, y, 0.3, +1)
    Ao = O.op_wall(y, y, 0.3, -1)
    assert np.abs(Ae.sum(axis=1) - 1).max() < 1e-15
    assert np.abs(Ao[0]).max() < 2e-15 and np.abs(Ao[-1]).max() < 2e-15   # Eq. 8 at the walls
    assert np.all(Ae >= -1e-18)
    # odd rows are even rows with the mirrored share subtracted: |odd| <= even
    assert np.all(np.abs(Ao) <= Ae + 1e-16)


def test_truncated_filter_does_not_commute():
    """Cutting the support at the wall (no extension) breaks the response."""
    n = 129
    y = uniform_y(n)
    k = np.pi
    At = O.op_wall(y, y, 0.2, +1, truncated=True)
    assert np.abs(At.sum(axis=1) - 1).max() < 1e-15
    err = np.abs(At @ np.cos(k * (y + 1)) - gauss_hat(k, 0.2) * np.cos(k * (y + 1))).max()
    assert err > 1e-3


def _central_diff_periodic(f, axis, h):
    return (np.roll(f, -1, axis=axis) - np.roll(f, 1, axis=axis)) / (2 * h)


def _central_diff_y(f, h, parity):
    """Central difference in y (axis 0) with mirror ghosts of the given parity."""
    g = np.empty_like(f)
    g[1:-1] = (f[2:] - f[:-2]) / (2 * h)
    g[0] = (f[1] - parity * f[1]) / (2 * h)
    g[-1] = (parity * f[-2] - f[-2]) / (2 * h)
    return g


@pytest.mark.parametrize("ext,expect_zero", [(O.EXT_EVEN_ODD, True), (O.EXT_ODD_EVEN, False)])
def test_divergence_preserved_uniform(ext, expect_zero):
    """The paper's consistency claim (Sec. 2.2): with Eq. 7 the filtered field
    of a discretely solenoidal field is discretely solenoidal."""
    nx, ny, nz = 24, 33, 20
    Lx, Lz = 2 * math.pi, math.pi
    hx, hz = Lx / nx, Lz / nz
    y = uniform_y(ny)
    hy = y[1] - y[0]
    rng = np.random.default_rng(5)
    psi = rng.standard_normal((3, ny, nz, nx))
    psi[0, [0, -1]] = 0.0   # psi1, psi3 odd about the walls
    psi[2, [0, -1]] = 0.0
    # u = D x psi, parities (even, odd, even) for Eq. 7
    u = np.empty_like(psi)
    u[0] = _central_diff_y(psi[2], hy, -1) - _central_diff_periodic(psi[1], 1, hz)
    u[1] = _central_diff_periodic(psi[0], 1, hz) - _central_diff_periodic(psi[2], 2, hx)
    u[2] = _central_diff_periodic(psi[1], 2, hx) - _central_diff_y(psi[0], hy, -1)
    div = (_central_diff_periodic(u[0], 2, hx) + _central_diff_y(u[1], hy, -1)
           + _central_diff_periodic(u[2], 1, hz))
    assert np.abs(div).max() < 1e-12
    delta = 0.35
    Ax = O.op_periodic(nx, Lx, nx, delta)
    Az = O.op_periodic(nz, Lz, nz, delta)
    par = (1, -1, 1) if ext == O.EXT_EVEN_ODD else (-1, 1, -1)
    ub = [O.apply_separable(u[c], Ax, O.op_wall(y, y, delta, par[c]), Az) for c in range(3)]
    divb = (_central_diff_periodic(ub[0], 2, hx) + _central_diff_y(ub[1], hy, -1)
            + _central_diff_periodic(ub[2], 1, hz))
    scale = max(np.abs(np.array(ub)).max(), 1.0)
    if expect_zero:
        assert np.abs(divb).max() < 1e-12 * scale / hx
    else:
        assert np.abs(divb).max() > 1e-4


def test_mirror_symmetric_input_gives_mirror_symmetric_output():
    """Eq. 8: filtering commutes with the reflection y -> -y of the channel."""
    d = I.dns_grid(16, 33, 12, 2 * math.pi, math.pi)
    l = I.les_grid(d, 8, 17, 6)
    u = I.channel_velocity(d, 3)
    um = u[:, ::-1].copy()
    um[1] *= -1
    ub, tau = O.subfilter_stress(d, l, 0.3, u)
    ubm, taum = O.subfilter_stress(d, l, 0.3, um)
    assert np.abs(ubm[0] - ub[0, ::-1]).max() < 1e-12
    assert np.abs(ubm[1] + ub[1, ::-1]).max() < 1e-12
    assert np.abs(taum[1] + tau[1, ::-1]).max() < 1e-11   # tau12 flips sign
    assert np.abs(taum[0] - tau[0, ::-1]).max() < 1e-11


# ------------------------------------------------------------- Eq. 6 ----
def _tiny_case(seed=11):
    d = I.dns_grid(32, 33, 32, 2 * math.pi, math.pi)
    l = I.les_grid(d, 8, 9, 8)
    return d, l, 2 * math.pi / 16, I.channel_velocity(d, seed)


def test_tau_closed_form_single_modes():
    """u1 = a sin(kx x) + b cos(kz z), u3 = c cos(kz z): every filtered
    quantity has a closed form in the Gaussian response, so T_ij does too."""
    n = 64
    d = I.Grid(n, 33, 48, 2 * math.pi, math.pi, I.tanh_nodes(33))
    l = I.les_grid(d, 16, 17, 12)
    delta = 0.6
    hx, hz = d.Lx / d.nx, d.Lz / d.nz
    kx, kz = 2 * 2 * np.pi / d.Lx, 3 * 2 * np.pi / d.Lz
    x = np.arange(d.nx) * hx
    z = np.arange(d.nz) * hz
    a, b, c = 0.7, 0.4, 0.5
    u = np.zeros((3, d.ny, d.nz, d.nx))
    u[0] = a * np.sin(kx * x)[None, None, :] + b * np.cos(kz * z)[None, :, None]
    u[2] = c * np.cos(kz * z)[None, :, None] * np.ones((d.ny, 1, 1))
    ub, tau = O.subfilter_stress(d, l, delta, u)
    Rx = lambda k: poisson_response(k, delta, hx)
    Rz = lambda k: poisson_response(k, delta, hz)
    X = np.arange(l.nx) * l.Lx / l.nx
    Z = np.arange(l.nz) * l.Lz / l.nz
    SX = np.sin(kx * X)[None, None, :]
    CZ = np.cos(kz * Z)[None, :, None]
    C2X = np.cos(2 * kx * X)[None, None, :]
    C2Z = np.cos(2 * kz * Z)[None, :, None]
    # bar(sin^2) = (1 - R(2k) cos 2kx)/2 ; bar(cos^2) = (1 + R(2k) cos 2kz)/2
    t11 = (a * a * (0.5 - 0.5 * Rx(2 * kx) * C2X - Rx(kx) ** 2 * SX ** 2)
           + b * b * (0.5 + 0.5 * Rz(2 * kz) * C2Z - Rz(kz) ** 2 * CZ ** 2))
    t33 = c * c * (0.5 + 0.5 * Rz(2 * kz) * C2Z - Rz(kz) ** 2 * CZ ** 2)
    t13 = b * c * (0.5 + 0.5 * Rz(2 * kz) * C2Z - Rz(kz) ** 2 * CZ ** 2) + 0 * SX
    assert np.abs(ub[0] - (a * Rx(kx) * SX + b * Rz(kz) * CZ)).max() < 1e-13
    assert np.abs(tau[0] - t11).max() < 1e-13
    assert np.abs(tau[2] - t13).max() < 1e-13
    assert np.abs(tau[5] - t33).max() < 1e-13
    for q in (1, 3, 4):
        assert np.abs(tau[q]).max() < 1e-15


def test_gradient_model_limit():
    """For a smooth mode with k delta << 1, T_11 -> (delta^2 / 12) (du1/dx)^2,
    the second-moment expansion of the Gaussian, with a relative error O((k delta)^2)."""
    n = 256
    d = I.Grid(n, 9, 8, 2 * math.pi, math.pi, I.tanh_nodes(9))
    l = I.Grid(n // 4, 9, 8, d.Lx, d.Lz, d.y)
    x = np.arange(n) * d.Lx / n
    errs = []
    for delta in (0.2, 0.1):
        u = np.zeros((3, d.ny, d.nz, d.nx))
        u[0] = np.sin(x)[None, None, :]
        ub, tau = O.subfilter_stress(d, l, delta, u)
        X = np.arange(l.nx) * l.Lx / l.nx
        grad = math.exp(-delta ** 2 / 24) * np.cos(X)       # d bar(u1)/dx
        model = delta ** 2 / 12 * grad ** 2
        t = tau[0, 4, 3]
        errs.append(np.abs(t - model).max() / (delta ** 2 / 12))
    assert errs[0] < 0.01 and errs[1] < errs[0] / 3.5


def test_tau_symmetric_psd_and_galilean():
    d, l, delta, u = _tiny_case()
    ub, tau = O.subfilter_stress(d, l, delta, u)
    T = np.empty(tau.shape[1:] + (3, 3))
    for q, (i, j) in enumerate(O.PAIRS):
        T[..., i, j] = tau[q]
        T[..., j, i] = tau[q]
    ev = np.linalg.eigvalsh(T.reshape(-1, 3, 3))
    assert ev.min() > -1e-11 * np.abs(tau).max()
    shifted = u.copy()
    shifted[0] += 3.0
    shifted[2] -= 1.5
    ub2, tau2 = O.subfilter_stress(d, l, delta, shifted)
    assert np.abs(tau2 - tau).max() < 1e-11 * max(1.0, np.abs(tau).max())
    assert np.abs(ub2[0] - ub[0] - 3.0).max() < 1e-12
    # a shift of u2 is not a symmetry of the extended field (it breaks parity)
    bad = u.copy()
    bad[1] += 1.0
    _, tau3 = O.subfilter_stress(d, l, delta, bad)
    assert np.abs(tau3 - tau).max() > 1e-3


def test_constant_and_mean_profile():
    """A constant u1, u3 and any profile U(y) in u1 have T = 0 away from the
    y-filter's shear term; constants pass through exactly."""
    d, l, delta, _ = _tiny_case()
    u = np.zeros((3, d.ny, d.nz, d.nx))
    u[0] = 2.5
    u[2] = -1.0
    ub, tau = O.subfilter_stress(d, l, delta, u)
    assert np.abs(ub[0] - 2.5).max() < 1e-14 and np.abs(ub[2] + 1.0).max() < 1e-14
    assert np.abs(ub[1]).max() < 1e-15
    assert np.abs(tau).max() < 1e-13


def test_separable_equals_direct3d():
    """The product kernel factorises, so the separable and the direct 3-D
    summation agree to roundoff (both are the definition)."""
    d, l, delta, u = _tiny_case(seed=4)
    ub, tau = O.subfilter_stress(d, l, delta, u)
    pts = np.array([[i, j, k] for j in range(l.ny) for k in range(l.nz) for i in range(l.nx)])
    ub3, tau3 = O.direct3d_points(d, l, delta, u, pts)
    ubs = ub.transpose(1, 2, 3, 0).reshape(-1, 3)
    taus = tau.transpose(1, 2, 3, 0).reshape(-1, 6)
    assert np.abs(ubs - ub3).max() < 1e-12
    assert np.abs(taus - tau3).max() < 1e-11


def test_separable_equals_direct3d_interpolated():
    """Non-coincident LES nodes in x, y and z exercise the interpolation."""
    d = I.dns_grid(30, 25, 20, 2 * math.pi, math.pi)
    l = I.Grid(9, 7, 6, d.Lx, d.Lz, I.tanh_nodes(7))
    delta = 0.5
    u = I.channel_velocity(d, 9)
    ub, tau = O.subfilter_stress(d, l, delta, u)
    pts = np.array([[i, j, k] for j in range(l.ny) for k in range(l.nz) for i in range(l.nx)])
    ub3, tau3 = O.direct3d_points(d, l, delta, u, pts)
    assert np.abs(ub.transpose(1, 2, 3, 0).reshape(-1, 3) - ub3).max() < 1e-12
    assert np.abs(tau.transpose(1, 2, 3, 0).reshape(-1, 6) - tau3).max() < 1e-11


def _brute_force(d, l, delta, u, ext=O.EXT_EVEN_ODD):
    """Third path: write the extended field out node by node (periodic copies
    in x and z, mirror copies in y with the parities of Eq. 7) and sum the 3-D
    product kernel over it at every DNS node, then interpolate linearly."""
    par = (1, -1, 1) if ext == O.EXT_EVEN_ODD else (-1, 1, -1)
    hx, hz = d.Lx / d.nx, d.Lz / d.nz
    xs = [(i * hx + m * d.Lx, i) for m in (-1, 0, 1) for i in range(d.nx)]
    zs = [(k * hz + m * d.Lz, k) for m in (-1, 0, 1) for k in range(d.nz)]
    ys = []
    for m in (-1, 0, 1):
        for j in range(d.ny):
            # kind 1: direct image, -1: mirror image, 0: wall node (its own mirror)
            ys.append((d.y[j] + 4 * m, j, 0 if j in (0, d.ny - 1) else 1))
            if 0 < j < d.ny - 1:
                ys.append((-2 - d.y[j] + 4 * m, j, -1))
    ys.sort()
    hy = [ys[1][0] - ys[0][0]] + [0.5 * (ys[n + 1][0] - ys[n - 1][0]) for n in range(1, len(ys) - 1)] \
        + [ys[-1][0] - ys[-2][0]]
    G = lambda s: math.exp(-6 * s * s / (delta * delta)) if abs(s) <= 2.5 * delta else 0.0
    fields = [u[0], u[1], u[2]] + [u[i] * u[j] for i, j in O.PAIRS]
    fpar = list(par) + [par[i] * par[j] for i, j in O.PAIRS]
    filt = np.zeros((9, d.ny, d.nz, d.nx))
    for jj in range(d.ny):
        wy = [(G(d.y[jj] - e) * hy[n], src, sg) for n, (e, src, sg) in enumerate(ys)]
        wy = [t for t in wy if t[0] > 0]
        for kk in range(d.nz):
            wz = [(G(kk * hz - e) * hz, src) for e, src in zs]
            wz = [t for t in wz if t[0] > 0]
            for ii in range(d.nx):
                wx = [(G(ii * hx - e) * hx, src) for e, src in xs]
                wx = [t for t in wx if t[0] > 0]
                num = np.zeros(9)
                den = 0.0
                for a, j, sg in wy:
                    for b, k in wz:
                        for c, i in wx:
                            w = a * b * c
                            den += w
                            for q in range(9):
                                s = {1: 1.0, -1: float(fpar[q]), 0: 0.5 * (1 + fpar[q])}[sg]
                                num[q] += s * w * fields[q][j, k, i]
                filt[:, jj, kk, ii] = num / den
    # discretization: LES nodes coincide with DNS nodes here
    rx, rz = d.nx // l.nx, d.nz // l.nz
    ry = (d.ny - 1) // (l.ny - 1)
    f = filt[:, ::ry, ::rz, ::rx]
    ub = f[:3]
    tau = np.array([f[3 + q] - f[i] * f[j] for q, (i, j) in enumerate(O.PAIRS)])
    return ub, tau


def test_brute_force_tiny():
    d = I.dns_grid(8, 9, 8, 2 * math.pi, math.pi)
    l = I.les_grid(d, 4, 5, 4)
    delta = 0.9
    u = I.channel_velocity(d, 21)
    ubb, taub = _brute_force(d, l, delta, u)
    ub, tau = O.subfilter_stress(d, l, delta, u)
    # the plain formula cancels bar(u1 u1) ~ 400 down to T11 ~ 20: roundoff ~1e-13
    scale = np.abs(tau).max()
    assert np.abs(ub - ubb).max() < 1e-13
    assert np.abs(tau - taub).max() < 1e-13 * scale
    pts = np.array([[i, j, k] for j in range(l.ny) for k in range(l.nz) for i in range(l.nx)])
    ub3, tau3 = O.direct3d_points(d, l, delta, u, pts)
    assert np.abs(ub.transpose(1, 2, 3, 0).reshape(-1, 3) - ub3).max() < 1e-13
    assert np.abs(tau.transpose(1, 2, 3, 0).reshape(-1, 6) - tau3).max() < 1e-13 * scale


def test_row_subset_matches_full():
    d, l, delta, u = _tiny_case(seed=8)
    ub, tau = O.subfilter_stress(d, l, delta, u)
    ub2, tau2 = O.subfilter_stress(d, l, delta, u, J0=3, J1=6)
    assert np.array_equal(ub[:, 3:6], ub2[:, 3:6]) and np.array_equal(tau[:, 3:6], tau2[:, 3:6])
    assert not tau2[:, :3].any()


def test_table1_spacing_of_grid_generator():
    """Table 1: Delta_1+ = Delta_3+ = 8.8 for the 2 pi x pi box at Re_tau 180
    with 128 x 64 nodes; the generator reproduces that arithmetic."""
    g = I.dns_grid(128, 65, 64, *I.BOX_SMALL)
    assert abs(g.Lx / g.nx * 180 - 8.8) < 0.05 and abs(g.Lz / g.nz * 180 - 8.8) < 0.05


def test_generator_solenoidal_no_slip():
    d = I.dns_grid(32, 33, 32, 2 * math.pi, math.pi)
    up = I.fluctuation(d, 3)
    assert abs(math.sqrt(np.mean(up * up)) - 0.1) < 1e-12
    assert np.abs(up[:, 0]).max() < 1e-14 and np.abs(up[:, -1]).max() < 1e-14
    assert np.abs(up.mean(axis=(2, 3))).max() < 1e-14       # zero plane means
    # spectral divergence in x, z plus a high-order y-derivative is tiny
    kx = np.fft.fftfreq(d.nx, 1.0 / d.nx) * 2 * np.pi / d.Lx
    kz = np.fft.fftfreq(d.nz, 1.0 / d.nz) * 2 * np.pi / d.Lz
    dudx = np.fft.ifft(1j * kx * np.fft.fft(up[0], axis=2), axis=2).real
    dwdz = np.fft.ifft(1j * kz[:, None] * np.fft.fft(up[2], axis=1), axis=1).real
    dvdy = np.gradient(up[1], d.y, axis=0, edge_order=2)
    res = dudx + dvdy + dwdz
    assert np.abs(res[4:-4]).max() < 0.05 * np.abs(dudx).max()


@pytest.mark.parametrize("ext", [O.EXT_EVEN_ODD, O.EXT_ODD_EVEN])
@pytest.mark.parametrize("form", ["bracket", "deviation"])
def test_decomposition_about_any_profile_matches_eq6(ext, form):
    """Eq. 6 decomposed about a profile U(y) (the form the GPU recovery uses:
    brackets of FP64 profile terms and fluctuation contractions, or the
    deviation form of the tensor-core y pass) equals the plain evaluation to
    1e-12 of max |T|, for the plane means, the mean of one z-row, and a
    profile with no relation to the field (odd components nonzero on the walls)."""
    dns = I.dns_grid(32, 33, 32, 2 * math.pi, math.pi)
    les = I.les_grid(dns, 8, 9, 8)
    u = I.channel_velocity(dns, 11)
    delta = 2 * math.pi / 16
    ub0, t0 = O.subfilter_stress(dns, les, delta, u, ext=ext)
    profiles = [u.mean(axis=(2, 3)), u[:, :, 0, :].mean(axis=2),
                np.stack([3 + 5 * dns.y ** 2, 0.3 * dns.y + 0.2, 1 - dns.y ** 4])]
    for U in profiles:
        ub, t = O.subfilter_stress_decomposed(dns, les, delta, u, U, ext=ext, form=form)
        assert np.abs(ub - ub0).max() <= 1e-12 * np.abs(ub0).max()
        assert np.abs(t - t0).max() <= 1e-12 * np.abs(t0).max()


@pytest.mark.parametrize("plant", O.PLANTS)
def test_planted_decomposition_mistakes_fail(plant):
    """Each mistake planted in the decomposed evaluation (a wrong cross-term or
    ubar parity, a dropped or doubled cross bracket, the deviation form without
    its wall term) breaks the 1e-12 agreement with the plain evaluation for at
    least one of the profiles of the test above."""
    dns = I.dns_grid(32, 33, 32, 2 * math.pi, math.pi)
    les = I.les_grid(dns, 8, 9, 8)
    u = I.channel_velocity(dns, 11)
    delta = 2 * math.pi / 16
    ub0, t0 = O.subfilter_stress(dns, les, delta, u)
    profiles = [u.mean(axis=(2, 3)), np.stack([3 + 5 * dns.y ** 2, 0.3 * dns.y + 0.2, 1 - dns.y ** 4])]
    form = "deviation" if plant == "drop_wall_term" else "bracket"
    worst = 0.0
    for U in profiles:
        ub, t = O.subfilter_stress_decomposed(dns, les, delta, u, U, form=form, plant=plant)
        worst = max(worst, np.abs(t - t0).max() / np.abs(t0).max(), np.abs(ub - ub0).max() / np.abs(ub0).max())
    assert worst > 1e-6
