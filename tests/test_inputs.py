"""Properties of the seeded synthetic channel field (the input recipe): the
stated rms, no slip at the walls, and zero divergence, checked from the field
itself (spectral x and z derivatives, a central difference in y)."""
import math

import numpy as np

from paper_1902_02508_gb300 import inputs as I


def _xz_derivative(f, L, axis):
    n = f.shape[axis]
    k = 2.0 * np.pi * np.fft.fftfreq(n, d=L / n)
    shape = [1] * f.ndim
    shape[axis] = n
    return np.fft.ifft(1j * k.reshape(shape) * np.fft.fft(f, axis=axis), axis=axis).real


def test_rms_and_no_slip():
    g = I.dns_grid(48, 33, 32, 4 * math.pi, 2 * math.pi)
    u = I.fluctuation(g, 21)
    assert abs(math.sqrt(float(np.mean(u * u))) - I.RMS) < 1e-12
    assert np.abs(u[:, 0]).max() < 1e-14 and np.abs(u[:, -1]).max() < 1e-14
    full = I.channel_velocity(g, 21)
    assert np.allclose(full[0] - u[0], I.reichardt(g.y)[:, None, None], atol=1e-13)


def test_divergence_free():
    # three y nodes y0 - e, y0, y0 + e in one call share one rms scale
    y0, e = 0.3, 1e-4
    g = I.Grid(48, 3, 32, 4 * math.pi, 2 * math.pi, np.array([y0 - e, y0, y0 + e]))
    u = I.fluctuation(g, 5)
    dudx = _xz_derivative(u[0, 1], g.Lx, 1)
    dwdz = _xz_derivative(u[2, 1], g.Lz, 0)
    dvdy = (u[1, 2] - u[1, 0]) / (2 * e)
    div = dudx + dvdy + dwdz
    assert np.abs(div).max() < 1e-6 * np.abs(dudx).max()
    # the same check fails for a field with one component perturbed
    v = u.copy()
    v[1] *= 1.01
    dvdy2 = (v[1, 2] - v[1, 0]) / (2 * e)
    assert np.abs(dudx + dvdy2 + dwdz).max() > 1e-3 * np.abs(dudx).max()


def test_seeds_differ_and_repeat():
    g = I.dns_grid(16, 9, 16, 2 * math.pi, math.pi)
    a, b, c = I.fluctuation(g, 1), I.fluctuation(g, 1), I.fluctuation(g, 2)
    assert np.array_equal(a, b)
    assert np.abs(a - c).max() > 0.1 * np.abs(a).max()
