"""FP64 reference of the differential filter: TEST INFRASTRUCTURE ONLY.

Only the tests use this module; the CUDA library never calls it.

Sec. 3 names the filter the simulations use: the kernel e^{-r/a} / (4 pi a^2 r),
the Green's function of (1 - a^2 lap), so that the filtered field solves

    (1 - a^2 lap) ubar = u                                              (D)

on the domain extended across the walls by Eq. 7 (Eq. 9 for the variant),
periodic in x and z.  Readings (the paper gives no discretisation):
  * a: the printed relation "a = Delta_f^2 / 40" is read as a^2 = Delta_f^2/40
    (the second-moment match to a top-hat sphere of radius Delta_f / 2);
    the width passed in is Delta_f.
  * lap: the second-order finite-difference Laplacian on the DNS nodes:
    three-point periodic in x and z; the three-point non-uniform stencil in y
      (D_yy v)_j = 2 / (h_- + h_+) * ((v_{j+1} - v_j) / h_+ - (v_j - v_{j-1}) / h_-)
    on the extended line, i.e. with mirror ghosts v(-1 - s) = p v(-1 + s) (and
    the same at +1) for the field's parity p.  An odd field is zero on the
    walls (its extension forces it; the input's wall value is not used), an
    even field's wall row reads (D_yy v)_0 = 2 (v_1 - v_0) / h_0^2.
  * sampling: the LES nodes are DNS nodes (every r-th in x and z, a subset of
    the y nodes); the interpolation of Sec. 3 is then the identity.
  * T_ij = bar(u_i u_j) - ubar_i ubar_j (Eq. 6) with the parity of a product
    the product of the parities.

Functions:
  * ``apply_operator``  -- the left side of (D) by its stencils (the definition);
  * ``filter_sparse``    -- (D) solved directly as one sparse system (small grids);
  * ``filter_fft``       -- (D) by the discrete Fourier transform in x and z
    (which diagonalises the periodic stencils: lap -> -(2 - 2 cos(k h)) / h^2)
    and a tridiagonal solve in y per (kx, kz);
  * ``subfilter_stress`` -- ubar_i and T_ij on the LES grid;
  * ``subfilter_stress_decomposed`` -- the same, written about a profile
    U(y) (a cross-check of the algebra of the fluctuation form).
"""
from __future__ import annotations

import math

import numpy as np

PAIRS = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))
EXT_EVEN_ODD = 0   # Eq. 7: parities (+, -, +)
EXT_ODD_EVEN = 1   # Eq. 9: parities (-, +, -)


def filter_parameter(delta_f: float) -> float:
    """a from the filter width Delta_f (reading a^2 = Delta_f^2 / 40)."""
    return delta_f / math.sqrt(40.0)


def parities(ext: int):
    if ext == EXT_EVEN_ODD:
        return (1, -1, 1)
    if ext == EXT_ODD_EVEN:
        return (-1, 1, -1)
    raise ValueError("the differential filter needs a wall extension (Eq. 7 or Eq. 9)")


def _dyy_rows(y, parity):
    """Coefficients (lower, centre, upper) of D_yy per node on the extended line."""
    ny = len(y)
    lo, ce, up = np.zeros(ny), np.zeros(ny), np.zeros(ny)
    for j in range(ny):
        if 0 < j < ny - 1:
            hm, hp = y[j] - y[j - 1], y[j + 1] - y[j]
            lo[j] = 2.0 / ((hm + hp) * hm)
            up[j] = 2.0 / ((hm + hp) * hp)
            ce[j] = -(lo[j] + up[j])
        elif parity > 0:                      # even: mirror ghost equals the inner neighbour
            h = y[1] - y[0] if j == 0 else y[-1] - y[-2]
            c = 2.0 / (h * h)
            ce[j] = -c
            if j == 0:
                up[j] = c
            else:
                lo[j] = c
        # odd: the wall value is zero; its row is handled by the callers
    return lo, ce, up


def apply_operator(v, y, Lx: float, Lz: float, a: float, parity: int):
    """(1 - a^2 lap) v for v [ny][nz][nx] of the given parity (wall rows of an
    odd field return v itself, which the extension makes zero)."""
    v = np.asarray(v, dtype=np.float64)
    ny, nz, nx = v.shape
    hx, hz = Lx / nx, Lz / nz
    lap = (np.roll(v, 1, axis=2) - 2 * v + np.roll(v, -1, axis=2)) / (hx * hx)
    lap += (np.roll(v, 1, axis=1) - 2 * v + np.roll(v, -1, axis=1)) / (hz * hz)
    lo, ce, up = _dyy_rows(y, parity)
    dyy = ce[:, None, None] * v
    dyy[1:] += lo[1:, None, None] * v[:-1]
    dyy[:-1] += up[:-1, None, None] * v[1:]
    out = v - a * a * (lap + dyy)
    if parity < 0:
        out[0] = v[0]
        out[-1] = v[-1]
    return out


def filter_sparse(u, y, Lx: float, Lz: float, a: float, parity: int):
    """(D) as one sparse linear system in all nx ny nz unknowns (direct solve)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    u = np.asarray(u, dtype=np.float64)
    ny, nz, nx = u.shape
    hx, hz = Lx / nx, Lz / nz

    def idx(j, k, i):
        return (j * nz + k) * nx + i

    rows, cols, vals = [], [], []
    lo, ce, up = _dyy_rows(y, parity)
    rhs = u.reshape(-1).copy()
    for j in range(ny):
        wall_odd = parity < 0 and (j == 0 or j == ny - 1)
        for k in range(nz):
            for i in range(nx):
                r = idx(j, k, i)
                if wall_odd:
                    rows.append(r), cols.append(r), vals.append(1.0)
                    rhs[r] = 0.0
                    continue
                diag = 1.0 + a * a * (2 / hx ** 2 + 2 / hz ** 2 - ce[j])
                rows.append(r), cols.append(r), vals.append(diag)
                for c, w in ((idx(j, k, (i + 1) % nx), hx), (idx(j, k, (i - 1) % nx), hx),
                             (idx(j, (k + 1) % nz, i), hz), (idx(j, (k - 1) % nz, i), hz)):
                    rows.append(r), cols.append(c), vals.append(-a * a / (w * w))
                if j > 0:
                    rows.append(r), cols.append(idx(j - 1, k, i)), vals.append(-a * a * lo[j])
                if j < ny - 1:
                    rows.append(r), cols.append(idx(j + 1, k, i)), vals.append(-a * a * up[j])
    n = nx * ny * nz
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    return spla.spsolve(A.tocsc(), rhs).reshape(ny, nz, nx)


def _modified_k2(n: int, L: float):
    h = L / n
    m = np.arange(n)
    return (2.0 - 2.0 * np.cos(2.0 * np.pi * m / n)) / (h * h)


def filter_fft(u, y, Lx: float, Lz: float, a: float, parity: int):
    """(D) with the DFT in x and z and the Thomas algorithm in y per mode."""
    u = np.asarray(u, dtype=np.float64).copy()
    ny, nz, nx = u.shape
    if parity < 0:
        u[0] = 0.0
        u[-1] = 0.0
    U = np.fft.fft2(u, axes=(1, 2))                          # [ny][kz][kx]
    lam = a * a * (_modified_k2(nz, Lz)[:, None] + _modified_k2(nx, Lx)[None, :])
    lo, ce, up = _dyy_rows(y, parity)
    # tridiagonal rows: sub[j] v_{j-1} + dia[j] v_j + sup[j] v_{j+1} = U_j
    sub = -a * a * lo
    sup = -a * a * up
    dia = np.empty((ny,) + lam.shape)
    for j in range(ny):
        dia[j] = 1.0 + lam - a * a * ce[j]
    if parity < 0:                                           # identity rows at the walls
        for j in (0, ny - 1):
            dia[j] = 1.0
            sub[j] = 0.0
            sup[j] = 0.0
    cp = np.empty_like(dia)
    dp = np.empty_like(U)
    cp[0] = sup[0] / dia[0]
    dp[0] = U[0] / dia[0]
    for j in range(1, ny):
        den = dia[j] - sub[j] * cp[j - 1]
        cp[j] = sup[j] / den
        dp[j] = (U[j] - sub[j] * dp[j - 1]) / den
    V = np.empty_like(U)
    V[-1] = dp[-1]
    for j in range(ny - 2, -1, -1):
        V[j] = dp[j] - cp[j] * V[j + 1]
    return np.fft.ifft2(V, axes=(1, 2)).real


def les_indices(dns, les):
    """DNS node indices of the LES nodes (x, y, z); raises if they are not DNS nodes."""
    if dns.nx % les.nx or dns.nz % les.nz:
        raise ValueError("LES x and z nodes must be DNS nodes")
    jy = np.searchsorted(dns.y, les.y)
    jy = np.clip(jy, 0, dns.ny - 1)
    if not np.array_equal(dns.y[jy], les.y):
        raise ValueError("LES y nodes must be DNS nodes")
    return dns.nx // les.nx, jy, dns.nz // les.nz


def subfilter_stress(dns, les, delta_f: float, u, ext: int = EXT_EVEN_ODD, solver=filter_fft):
    """ubar [3][nly][nlz][nlx] and T [6][...] of Eq. 6 with the differential filter."""
    u = np.asarray(u, dtype=np.float64)
    a = filter_parameter(delta_f)
    p = parities(ext)
    rx, jy, rz = les_indices(dns, les)

    def sample(f):
        return f[jy][:, ::rz, ::rx]

    ub = np.stack([sample(solver(u[c], dns.y, dns.Lx, dns.Lz, a, p[c])) for c in range(3)])
    tau = np.empty((6,) + ub.shape[1:])
    for q, (i, j) in enumerate(PAIRS):
        prod = sample(solver(u[i] * u[j], dns.y, dns.Lx, dns.Lz, a, p[i] * p[j]))
        tau[q] = prod - ub[i] * ub[j]
    return ub, tau


PLANTS = ("cross_parity", "drop_cross", "profile_parity")


def subfilter_stress_decomposed(dns, les, delta_f: float, u, U, ext: int = EXT_EVEN_ODD, solver=filter_fft,
                                plant=None):
    """ubar and T of Eq. 6 written about a profile U[3][ny] (any profile).

    With u_a = U_a(y) + u'_a and F the filter (linear; on a function of y
    alone it is the kx = kz = 0 solve):
      ubar_a = F(U_a) + F(u'_a),
      T_ab = [F(U_a U_b) - F(U_a) F(U_b)] + [F(U_a u'_b) - F(U_a) F(u'_b)]
           + [F(U_b u'_a) - F(U_b) F(u'_a)] + [F(u'_a u'_b) - F(u'_a) F(u'_b)],
    each term filtered with the parity of its product.

    ``plant`` (tests only) names one deliberate mistake, to show that the
    comparison with the plain evaluation catches it: "cross_parity" (U_a u'_b
    filtered with the parity of u'_b instead of p_a p_b), "drop_cross" (the
    [F(U_b u'_a) - F(U_b) F(u'_a)] bracket left out), "profile_parity"
    (F(U_2) with the wrong parity).
    """
    if plant is not None and plant not in PLANTS:
        raise ValueError(f"plant is one of {PLANTS}")
    u = np.asarray(u, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    assert U.shape == (3, dns.ny)
    a = filter_parameter(delta_f)
    p = parities(ext)
    rx, jy, rz = les_indices(dns, les)

    def F(f, parity):
        return solver(f, dns.y, dns.Lx, dns.Lz, a, parity)[jy][:, ::rz, ::rx]

    shape = u.shape[1:]
    prof = [np.broadcast_to(U[c][:, None, None], shape) for c in range(3)]
    up = u - U[:, :, None, None]
    FU = [F(prof[c], -p[c] if (plant == "profile_parity" and c == 1) else p[c]) for c in range(3)]
    Fu = [F(up[c], p[c]) for c in range(3)]
    ub = np.stack([FU[c] + Fu[c] for c in range(3)])
    tau = np.empty((6,) + ub.shape[1:])
    for q, (i, j) in enumerate(PAIRS):
        pij = p[i] * p[j]
        pc = (lambda d: p[d]) if plant == "cross_parity" else (lambda d: pij)
        second = 0.0 if plant == "drop_cross" else (F(prof[j] * up[i], pc(i)) - FU[j] * Fu[i])
        tau[q] = ((F(prof[i] * prof[j], pij) - FU[i] * FU[j])
                  + (F(prof[i] * up[j], pc(j)) - FU[i] * Fu[j])
                  + second
                  + (F(up[i] * up[j], pij) - Fu[i] * Fu[j]))
    return ub, tau

