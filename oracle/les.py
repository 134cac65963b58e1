"""FP64 reference of a minimal explicitly filtered LES step driven by the
exact subfilter stress: TEST INFRASTRUCTURE ONLY.

Only the tests use this module; the CUDA library never calls it.

Sec. 3 and Fig. 2 of the paper couple the two computations: at every time
step the DNS field is filtered, T_ij of Eq. 6 is formed from it (Sec. 2.1),
and the explicitly filtered LES equations (Eq. 6: Eq. 5 with
bar(u_i u_j) = ubar_i ubar_j + T_ij) are advanced with that T_ij.  The
paper's LES is a staggered second-order finite-difference code with a
fractional-step method and a third-order Runge-Kutta scheme, driven by a
constant mean pressure gradient.  This module is the minimal collocated
counterpart, on the LES nodes where the filter samples ubar and T_ij.

Readings (the paper gives no discretisation of its own beyond the above):
  * nodes: x_i = i Lx/nx, z_k = k Lz/nz (periodic), the given y nodes with
    both walls;
  * wall values (Eq. 10 and Eq. 11): ubar_2 = 0 on the walls; ubar_1 and
    ubar_3 take the filter-consistent value F(u_i) on the walls, which in the
    loop of Fig. 2 is the filtered DNS of the same step (held over the step,
    like T_ij); without a DNS field the walls are no-slip;
  * derivatives: second-order central differences,
      dx f = (f[i+1] - f[i-1]) / (2 hx)           (periodic; z alike),
      dy f = (f[j+1] - f[j-1]) / (y[j+1] - y[j-1])  (interior nodes);
    Laplacian: three-point in x and z, the three-point non-uniform stencil
      2 / (y[j+1] - y[j-1]) * ((f[j+1] - f[j]) / (y[j+1] - y[j])
                               - (f[j] - f[j-1]) / (y[j] - y[j-1])) in y;
  * right-hand side at interior nodes (Eq. 5 with the flux written through
    Eq. 6):  R_i = -sum_j d_j (ubar_i ubar_j + T_ij) + nu lap ubar_i + Pi [i = 1],
    Pi the imposed mean pressure gradient (u_tau^2 / delta = 1 in wall units);
  * projection (the pressure step of the fractional-step method): the
    orthogonal projection of the interior velocities, in the inner product
    with weight (y[j+1] - y[j-1]) / 2 per node, onto the fields whose discrete
    divergence d_x u_1 + d_y u_2 + d_z u_3 is zero at every interior node, the
    wall velocities held fixed (the divergence at the interior nodes reads
    only the wall value of u_2, which is zero);
  * time advance: the low-storage third-order Runge-Kutta scheme with
    gamma = (8/15, 5/12, 3/4), zeta = (0, -17/60, -5/12),
      u* = u_(k-1) + dt (gamma_k R(u_(k-1)) + zeta_k R(u_(k-2))),  u_k = P u*,
    and T_ij held at its value for the step; "euler" is one substep with
    gamma = 1, zeta = 0.

Functions (arrays are [c][y][z][x], T is [6][y][z][x] in the order 11, 12,
13, 22, 23, 33):
  * ``rhs``          -- R_i by the stencils above;
  * ``divergence``   -- the discrete divergence at the interior nodes;
  * ``project``      -- the projection, by the Fourier transform in x and z
    (a library FFT) and, per mode, the least-squares solution of its
    normal equations in y;
  * ``project_dense``-- the same projection as one dense least-squares
    problem in physical space (small grids; a cross-check of the first);
  * ``step``         -- one time step;
  * ``apost_run``    -- the loop of Fig. 2: per step the filter of the DNS
    snapshot (oracle.subfilter_stress) gives T_ij, then one LES step.
"""
from __future__ import annotations

import numpy as np

PAIRS = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))
RK3_GAMMA = (8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0)
RK3_ZETA = (0.0, -17.0 / 60.0, -5.0 / 12.0)


def _pair_index(i: int, j: int) -> int:
    return PAIRS.index((min(i, j), max(i, j)))


def dx(f, h: float, axis: int):
    """Periodic central difference along `axis`."""
    return (np.roll(f, -1, axis=axis) - np.roll(f, 1, axis=axis)) / (2.0 * h)


def dy(f, y):
    """Central difference in y (axis 0 of f[y][z][x]) at the interior nodes;
    the wall rows of the result are zero."""
    y = np.asarray(y, dtype=np.float64)
    out = np.zeros_like(f)
    span = (y[2:] - y[:-2])[:, None, None]
    out[1:-1] = (f[2:] - f[:-2]) / span
    return out


def lap(f, y, hx: float, hz: float):
    """Three-point Laplacian of f[y][z][x] at the interior nodes (wall rows zero)."""
    y = np.asarray(y, dtype=np.float64)
    out = np.zeros_like(f)
    fx = (np.roll(f, -1, axis=2) - 2.0 * f + np.roll(f, 1, axis=2)) / (hx * hx)
    fz = (np.roll(f, -1, axis=1) - 2.0 * f + np.roll(f, 1, axis=1)) / (hz * hz)
    hm = (y[1:-1] - y[:-2])[:, None, None]
    hp = (y[2:] - y[1:-1])[:, None, None]
    fy = 2.0 / (hm + hp) * ((f[2:] - f[1:-1]) / hp - (f[1:-1] - f[:-2]) / hm)
    out[1:-1] = fx[1:-1] + fz[1:-1] + fy
    return out


def _spacing(grid):
    return grid.Lx / grid.nx, grid.Lz / grid.nz


def rhs(u, tau, grid, nu: float, forcing: float):
    """R_i at the interior nodes (wall rows zero).  tau may be None (no
    subfilter term)."""
    u = np.asarray(u, dtype=np.float64)
    hx, hz = _spacing(grid)
    R = np.zeros_like(u)
    for i in range(3):
        acc = np.zeros_like(u[0])
        for j, d in ((0, lambda f: dx(f, hx, 2)), (1, lambda f: dy(f, grid.y)), (2, lambda f: dx(f, hz, 1))):
            flux = u[i] * u[j]
            if tau is not None:
                flux = flux + np.asarray(tau[_pair_index(i, j)], dtype=np.float64)
            acc -= d(flux)
        acc += nu * lap(u[i], grid.y, hx, hz)
        if i == 0:
            acc += forcing
        acc[0] = 0.0
        acc[-1] = 0.0
        R[i] = acc
    return R


def divergence(u, grid):
    """d_x u_1 + d_y u_2 + d_z u_3 at the interior nodes (wall rows zero)."""
    u = np.asarray(u, dtype=np.float64)
    hx, hz = _spacing(grid)
    d = dx(u[0], hx, 2) + dy(u[1], grid.y) + dx(u[2], hz, 1)
    d[0] = 0.0
    d[-1] = 0.0
    return d


def _weights(y):
    y = np.asarray(y, dtype=np.float64)
    return (y[2:] - y[:-2]) / 2.0      # interior nodes


def _symbol(n: int, h: float):
    """Fourier symbol i s(k) of the periodic central difference for the
    modes of np.fft (index m): s = sin(2 pi m / n) / h, exactly 0 at m = 0 and
    at the Nyquist index of an even n."""
    m = np.arange(n)
    s = np.sin(2.0 * np.pi * m / n) / h
    s[0] = 0.0
    if n % 2 == 0:
        s[n // 2] = 0.0
    return s


def project(u, grid):
    """The weighted orthogonal projection onto discretely divergence-free
    fields (module docstring), per Fourier mode in x and z.

    Per mode the divergence is the matrix Dh = [i s_x I | Dy | i s_z I]
    acting on the interior values (u1, u2, u3) of the y line; with W the
    diagonal of weights, u = u* - W^-1 Dh^H lam where
    (Dh W^-1 Dh^H) lam = Dh u* (least squares: the matrix is singular for the
    modes whose x and z symbols vanish)."""
    u = np.asarray(u, dtype=np.float64)
    y = np.asarray(grid.y, dtype=np.float64)
    ny, nz, nx = u.shape[1:]
    ni = ny - 2
    hx, hz = _spacing(grid)
    sx, sz = _symbol(nx, hx), _symbol(nz, hz)
    W = _weights(y)
    Winv = 1.0 / W
    # interior y-difference matrix acting on interior u2 (wall values zero)
    Dy = np.zeros((ni, ni))
    for r in range(ni):
        j = r + 1
        span = y[j + 1] - y[j - 1]
        if j + 1 <= ny - 2:
            Dy[r, r + 1] = 1.0 / span
        if j - 1 >= 1:
            Dy[r, r - 1] = -1.0 / span
    U = np.fft.fft2(u[:, 1:-1], axes=(2, 3))          # [c][ni][nz][nx]
    out = np.array(U)
    I = np.eye(ni)
    for q in range(nz):
        for m in range(nx):
            Dh = np.hstack([1j * sx[m] * I, Dy.astype(complex), 1j * sz[q] * I])   # [ni][3 ni]
            Wi = np.concatenate([Winv, Winv, Winv])
            ustar = np.concatenate([U[0, :, q, m], U[1, :, q, m], U[2, :, q, m]])
            A = (Dh * Wi[None, :]) @ Dh.conj().T
            b = Dh @ ustar
            lam = np.linalg.lstsq(A, b, rcond=1e-13)[0]
            corr = Wi * (Dh.conj().T @ lam)
            v = ustar - corr
            out[0, :, q, m] = v[:ni]
            out[1, :, q, m] = v[ni:2 * ni]
            out[2, :, q, m] = v[2 * ni:]
    res = np.array(u)
    res[:, 1:-1] = np.real(np.fft.ifft2(out, axes=(2, 3)))
    return res


def _divergence_matrix(grid):
    """The divergence at the interior nodes as a dense matrix acting on the
    interior values of (u1, u2, u3), flattened [c][j][k][i]."""
    y = np.asarray(grid.y, dtype=np.float64)
    ny, nz, nx = grid.ny, grid.nz, grid.nx
    ni = ny - 2
    hx, hz = _spacing(grid)
    npt = ni * nz * nx

    def idx(c, r, k, i):
        return ((c * ni + r) * nz + (k % nz)) * nx + (i % nx)

    D = np.zeros((npt, 3 * npt))
    for r in range(ni):
        j = r + 1
        span = y[j + 1] - y[j - 1]
        for k in range(nz):
            for i in range(nx):
                row = (r * nz + k) * nx + i
                D[row, idx(0, r, k, i + 1)] += 1.0 / (2 * hx)
                D[row, idx(0, r, k, i - 1)] -= 1.0 / (2 * hx)
                D[row, idx(2, r, k + 1, i)] += 1.0 / (2 * hz)
                D[row, idx(2, r, k - 1, i)] -= 1.0 / (2 * hz)
                if j + 1 <= ny - 2:
                    D[row, idx(1, r + 1, k, i)] += 1.0 / span
                if j - 1 >= 1:
                    D[row, idx(1, r - 1, k, i)] -= 1.0 / span
    return D


def project_dense(u, grid):
    """The same projection as one dense least-squares problem (small grids)."""
    u = np.asarray(u, dtype=np.float64)
    ny, nz, nx = u.shape[1:]
    D = _divergence_matrix(grid)
    w = np.repeat(_weights(grid.y), nz * nx)
    Wi = 1.0 / np.concatenate([w, w, w])
    ustar = u[:, 1:-1].reshape(-1)
    A = (D * Wi[None, :]) @ D.T
    lam = np.linalg.lstsq(A, D @ ustar, rcond=1e-13)[0]
    v = ustar - Wi * (D.T @ lam)
    res = np.array(u)
    res[:, 1:-1] = v.reshape(3, ny - 2, nz, nx)
    return res


def wall_values(u, ubc=None):
    """u with its wall rows set by Eq. 10 / Eq. 11: u_2 = 0, u_1 and u_3 from
    ubc (the filtered DNS) or zero."""
    u = np.asarray(u, dtype=np.float64).copy()
    for row in (0, -1):
        u[1, row] = 0.0
        for c in (0, 2):
            u[c, row] = 0.0 if ubc is None else np.asarray(ubc[c][row], dtype=np.float64)
    return u


def step(u, tau, grid, nu: float, dt: float, forcing: float = 1.0, scheme: str = "rk3", projector=project,
         ubc=None):
    """One time step of the LES (module docstring) with the wall values taken
    from ubc (None: no slip).  Returns the new field."""
    u = wall_values(u, ubc)
    if scheme == "rk3":
        coefs = list(zip(RK3_GAMMA, RK3_ZETA))
    elif scheme == "euler":
        coefs = [(1.0, 0.0)]
    else:
        raise ValueError(scheme)
    R_prev = None
    for gamma, zeta in coefs:
        R = rhs(u, tau, grid, nu, forcing)
        ustar = u + dt * gamma * R
        if zeta != 0.0:
            ustar = ustar + dt * zeta * R_prev
        u = projector(ustar, grid)
        R_prev = R
    return u


def apost_run(dns, les, delta: float, snapshots, u0, nu: float, dt: float, forcing: float = 1.0,
              ext: int = 0, scheme: str = "rk3"):
    """Fig. 2: for each DNS snapshot in turn, ubar and T_ij from the filter
    (Eq. 6, oracle.subfilter_stress) and one LES step from the current LES
    field, its wall values those of that ubar (Eq. 10).  Returns the LES field
    after the last step and the list of T_ij."""
    from . import oracle as O
    u = np.asarray(u0, dtype=np.float64)
    taus = []
    for snap in snapshots:
        ubar, tau = O.subfilter_stress(dns, les, delta, snap, ext=ext)
        taus.append(tau)
        u = step(u, tau, les, nu, dt, forcing, scheme, ubc=ubar)
    return u, taus
