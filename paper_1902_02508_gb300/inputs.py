"""Seeded synthetic channel-flow inputs: grids and velocity snapshots.

This module holds no filtering arithmetic.  It only manufactures the data the
filter consumes, in the shapes of the paper's channel experiment (Sec. 3,
Table 1): a channel of height 2 (walls at y = -1 and y = +1), periodic in x and
z, with wall-normal nodes clustered at the walls by a hyperbolic tangent
(Sec. 3).  The same arrays are handed to the CPU oracle and to the CUDA path.

Velocity recipe (units of u_tau, Re_tau = 180):
  * mean profile U(y): Reichardt's law of the wall with kappa = 0.41, C = 7.8,
    evaluated at y+ = (1 - |y|) Re_tau;
  * fluctuations u' = curl(psi) with psi built from random Fourier modes in
    (x, z) times (1 - y^2)^2 (a + b y).  Every mode is exactly solenoidal and
    vanishes with its first y-derivative at the walls (no slip).  Mode
    amplitudes fall as k^(-7/3) so the energy per shell falls as k^(-5/3);
    modes run over 1 <= |m| with |m_x| <= nx/4, |m_z| <= nz/4 (index units);
  * u' is rescaled to an rms of 0.1 over all points and components.

Layout of a snapshot: float64 array u[3][ny][nz][nx] (x fastest).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = 2.0          # tanh stretching parameter
RE_TAU = 180.0
KAPPA = 0.41
C_REICHARDT = 7.8
RMS = 0.1


@dataclass(frozen=True)
class Grid:
    """A channel grid: nx x ny x nz nodes, periodic lengths Lx, Lz, y-nodes."""
    nx: int
    ny: int
    nz: int
    Lx: float
    Lz: float
    y: np.ndarray  # (ny,) float64, ascending, y[0] = -1, y[-1] = +1

    @property
    def npts(self) -> int:
        return self.nx * self.ny * self.nz


def tanh_nodes(n: int, gamma: float = GAMMA) -> np.ndarray:
    """Wall-clustered nodes on [-1, 1]; both walls are nodes."""
    s = 2.0 * np.arange(n, dtype=np.float64) / (n - 1) - 1.0
    y = np.tanh(gamma * s) / math.tanh(gamma)
    y[0], y[-1] = -1.0, 1.0
    return y


def dns_grid(nx: int, ny: int, nz: int, Lx: float, Lz: float) -> Grid:
    return Grid(nx, ny, nz, float(Lx), float(Lz), tanh_nodes(ny))


def les_grid(dns: Grid, nlx: int, nly: int, nlz: int) -> Grid:
    """LES grid over the same box.  When (ny-1)/(nly-1) is an integer the LES
    y-nodes are taken as that subset of the DNS nodes, bit for bit."""
    if (dns.ny - 1) % (nly - 1) == 0:
        y = dns.y[:: (dns.ny - 1) // (nly - 1)].copy()
    else:
        y = tanh_nodes(nly)
    return Grid(nlx, nly, nlz, dns.Lx, dns.Lz, y)


def reichardt(y: np.ndarray, re_tau: float = RE_TAU) -> np.ndarray:
    yp = (1.0 - np.abs(y)) * re_tau
    return (np.log1p(KAPPA * yp) / KAPPA
            + C_REICHARDT * (1.0 - np.exp(-yp / 11.0) - (yp / 11.0) * np.exp(-yp / 3.0)))


def _modes(nx: int, nz: int):
    mx_max, mz_max = nx // 4, nz // 4
    mx = np.arange(0, mx_max + 1)
    mz = np.arange(-mz_max, mz_max + 1)
    MX, MZ = np.meshgrid(mx, mz, indexing="ij")
    MX, MZ = MX.ravel(), MZ.ravel()
    keep = (MX > 0) | ((MX == 0) & (MZ > 0))   # half plane: the real part covers -m
    return MX[keep], MZ[keep]


def fluctuation(grid: Grid, seed: int, rms: float = RMS) -> np.ndarray:
    """Solenoidal, no-slip random field u'[3][ny][nz][nx] with the stated rms.

    u' = curl psi with psi = sum_m (1 - y^2)^2 (a_m + b_m y) e^{i(k_x x + k_z z)}
    (real part).  Every mode has the same four y shapes, P, P y, P' and P' y
    with P = (1 - y^2)^2, so each component is four x-z fields (one inverse
    FFT each) weighted by those shapes at every y node."""
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    rng = np.random.Generator(np.random.PCG64(seed))
    MX, MZ = _modes(nx, nz)
    nm = MX.size
    kx = 2.0 * np.pi * MX / grid.Lx
    kz = 2.0 * np.pi * MZ / grid.Lz
    kmag = np.sqrt(kx * kx + kz * kz)
    amp = kmag ** (-7.0 / 3.0)
    a = (rng.standard_normal((3, nm)) + 1j * rng.standard_normal((3, nm))) * amp
    b = (rng.standard_normal((3, nm)) + 1j * rng.standard_normal((3, nm))) * amp
    ik_x, ik_z = 1j * kx, 1j * kz
    # u'_hat = sum_s f_s(y) C[c][s] with f = (P, P y, P', P' y), from
    # psi = P a + P y b and dpsi/dy = P' a + (P' y + P) b:
    #   u'_hat_0 = dpsi_2/dy - i k_z psi_1
    #   u'_hat_1 = i k_z psi_0 - i k_x psi_2
    #   u'_hat_2 = i k_x psi_1 - dpsi_0/dy
    zero = np.zeros(nm, dtype=np.complex128)
    C = [[b[2] - ik_z * a[1], -ik_z * b[1], a[2], b[2]],
         [ik_z * a[0] - ik_x * a[2], ik_z * b[0] - ik_x * b[2], zero, zero],
         [ik_x * a[1] - b[0], ik_x * b[1], -a[0], -b[0]]]
    ix, iz = np.mod(MX, nx), np.mod(MZ, nz)
    jx, jz = np.mod(-MX, nx), np.mod(-MZ, nz)
    y = grid.y
    P = (1.0 - y * y) ** 2
    dP = -4.0 * y * (1.0 - y * y)
    shapes = (P, P * y, dP, dP * y)
    out = np.zeros((3, ny, nz, nx), dtype=np.float64)
    for c in range(3):
        for sh in range(4):
            if not np.any(C[c][sh]):
                continue
            # f = Re sum_m c_m e^{i theta} = sum_m (c_m e^{i theta} + conj(c_m) e^{-i theta}) / 2
            spec = np.zeros((nz, nx), dtype=np.complex128)
            np.add.at(spec, (iz, ix), 0.5 * C[c][sh])
            np.add.at(spec, (jz, jx), 0.5 * np.conj(C[c][sh]))
            F = np.fft.ifft2(spec).real * (nx * nz)
            out[c] += shapes[sh][:, None, None] * F[None]
    scale = rms / math.sqrt(float(np.mean(out * out)))
    out *= scale
    return out


def channel_velocity(grid: Grid, seed: int, rms: float = RMS) -> np.ndarray:
    """Full velocity u = U(y) e_x + u' as float64 [3][ny][nz][nx]."""
    u = fluctuation(grid, seed, rms)
    u[0] += reichardt(grid.y)[:, None, None]
    return u


def shifted(u: np.ndarray, sx: int, sz: int) -> np.ndarray:
    """A periodic translate of a snapshot: another valid channel field."""
    return np.roll(np.roll(u, sx, axis=3), sz, axis=2)


# The paper's channel boxes.
TWO_PI = 2.0 * math.pi
BOX_SMALL = (TWO_PI, math.pi)          # 2 pi x 2 x pi (Sec. 3)
BOX_LARGE = (2.0 * TWO_PI, TWO_PI)     # 4 pi x 2 x 2 pi


# The batched configuration: snapshots of uneven channel grids, each with its
# own constant filter width, in the 4 pi x 2 x 2 pi box; LES grid = DNS / 4 in
# every direction (its y nodes are every fourth DNS node).
BATCH_GRIDS = ((128, 97, 128), (192, 129, 192), (256, 193, 256))
BATCH_WIDTHS = (16, 32, 48)          # Delta = Lx / w


def batch_draws(n: int = 64, seed: int = 7):
    """The (grid, width) of each of n snapshots: uniform draws over the three
    grids and the three widths from a seeded PCG64 stream."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = rng.integers(0, len(BATCH_GRIDS), n)
    w = rng.integers(0, len(BATCH_WIDTHS), n)
    return [(BATCH_GRIDS[a], BATCH_WIDTHS[b]) for a, b in zip(g, w)]


def batch_grids(shape):
    """(dns, les) of one batched-configuration grid."""
    nx, ny, nz = shape
    dns = dns_grid(nx, ny, nz, *BOX_LARGE)
    return dns, les_grid(dns, nx // 4, (ny - 1) // 4 + 1, nz // 4)
