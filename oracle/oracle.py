"""Python access to the CPU oracle (oracle.c): test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It shares nothing with the CUDA library
and the CUDA library never calls it.  Every function here is IEEE double
precision on the host.

Citations are to the paper's sections and equations:
  * ``op_periodic``  -- Eq. 2 on a periodic uniform line + linear interpolation
    to the LES nodes (the discretization operator of Sec. 3);
  * ``op_wall``      -- Eq. 2 on the wall-normal line extended by Eq. 7 (or
    Eq. 9, or truncated at the walls) + linear interpolation;
  * ``subfilter_stress`` -- the four steps of Sec. 2.1 / Eq. 6, separable
    evaluation of the product kernel;
  * ``direct3d_points`` -- the same quantities by direct three-dimensional
    summation of Eq. 2 at selected LES points;
  * ``subfilter_stress_decomposed`` -- Eq. 6 again, decomposed about a given
    profile U(y) (the bracket and deviation forms; a cross-check of the
    algebra, evaluated with the same 1-D operators);
  * ``mlp_*`` (oracle/mlp.py) -- the learned closure of Sec. 2.1 / Sec. 5.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
# ORACLE_LIB names a library built elsewhere from a copy of oracle.c (the
# planted-mistake tests run the pins against such copies); it is used as is.
_LIB = os.environ.get("ORACLE_LIB") or os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

EXT_EVEN_ODD = 0   # Eq. 7
EXT_ODD_EVEN = 1   # Eq. 9
EXT_NONE = 2       # filter support cut at the walls

PAIRS = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into oracle/_build/liboracle.so."""
    if os.environ.get("ORACLE_LIB"):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off",
                               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
            lib.or_op_periodic.argtypes = [i, d, i, d, p]
            lib.or_op_wall.argtypes = [i, p, i, p, d, i, i, p]
            lib.or_apply_separable.argtypes = [i, i, i, i, i, i, p, p, p, p, p, i, i]
            lib.or_subfilter_stress.argtypes = [i, i, i, d, d, p, i, i, i, p, d, i, p, p, p, i, i]
            lib.or_subfilter_stress_q.argtypes = [i, i, i, d, d, p, i, i, i, p, d, i, i, p, p, p, i, i]
            lib.or_op_wall_q.argtypes = [i, p, i, p, d, i, i, i, p]
            lib.or_direct3d_points.argtypes = [i, i, i, d, d, p, i, i, i, p, d, i, p, i, p, p, p]
            lib.or_num_threads.restype = i
            lib.or_set_threads.argtypes = [i]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return _load().or_num_threads()


def set_threads(n: int) -> None:
    _load().or_set_threads(int(n))


def op_periodic(n: int, L: float, nl: int, delta: float) -> np.ndarray:
    A = np.zeros((nl, n))
    rc = _load().or_op_periodic(n, float(L), nl, float(delta), _ptr(A))
    if rc:
        raise ValueError(f"or_op_periodic failed ({rc})")
    return A


def op_wall(y, Y, delta: float, parity: int, truncated: bool = False, quad: int = 0) -> np.ndarray:
    """quad 0: trapezoid; 1: kernel integrated exactly against the piecewise-linear interpolant."""
    y, Y = _f64(y), _f64(Y)
    A = np.zeros((Y.size, y.size))
    rc = _load().or_op_wall_q(y.size, _ptr(y), Y.size, _ptr(Y), float(delta),
                              1 if truncated else 0, int(parity), int(quad), _ptr(A))
    if rc:
        raise ValueError(f"or_op_wall failed ({rc})")
    return A


def apply_separable(f, Ax, Ay, Az, J0: int = 0, J1: int = 0) -> np.ndarray:
    f = _f64(f)
    ny, nz, nx = f.shape
    Ax, Ay, Az = _f64(Ax), _f64(Ay), _f64(Az)
    out = np.zeros((Ay.shape[0], Az.shape[0], Ax.shape[0]))
    rc = _load().or_apply_separable(nx, ny, nz, Ax.shape[0], Ay.shape[0], Az.shape[0],
                                    _ptr(Ax), _ptr(Ay), _ptr(Az), _ptr(f), _ptr(out), J0, J1)
    if rc:
        raise ValueError(f"or_apply_separable failed ({rc})")
    return out


def subfilter_stress(dns, les, delta: float, u, ext: int = EXT_EVEN_ODD,
                     J0: int = 0, J1: int = 0, quad: int = 0):
    """(ubar[3][nly][nlz][nlx], tau[6][nly][nlz][nlx]) for the whole snapshot
    (or LES rows J0 <= J < J1; other rows are zero)."""
    u = _f64(u)
    assert u.shape == (3, dns.ny, dns.nz, dns.nx)
    y, Y = _f64(dns.y), _f64(les.y)
    ubar = np.zeros((3, les.ny, les.nz, les.nx))
    tau = np.zeros((6, les.ny, les.nz, les.nx))
    rc = _load().or_subfilter_stress_q(dns.nx, dns.ny, dns.nz, dns.Lx, dns.Lz, _ptr(y),
                                       les.nx, les.ny, les.nz, _ptr(Y), float(delta), int(ext), int(quad),
                                       _ptr(u), _ptr(ubar), _ptr(tau), J0, J1)
    if rc:
        raise ValueError(f"or_subfilter_stress failed ({rc})")
    return ubar, tau


def direct3d_points(dns, les, delta: float, u, pts, ext: int = EXT_EVEN_ODD):
    """(ubar[npts][3], tau[npts][6]) by direct 3-D summation at LES points
    pts[npts][3] = (I, J, K)."""
    u = _f64(u)
    pts = np.ascontiguousarray(pts, dtype=np.int32)
    n = pts.shape[0]
    y, Y = _f64(dns.y), _f64(les.y)
    ub = np.zeros((n, 3))
    tau = np.zeros((n, 6))
    rc = _load().or_direct3d_points(dns.nx, dns.ny, dns.nz, dns.Lx, dns.Lz, _ptr(y),
                                    les.nx, les.ny, les.nz, _ptr(Y), float(delta), int(ext),
                                    _ptr(u), n, _ptr(pts), _ptr(ub), _ptr(tau))
    if rc:
        raise ValueError(f"or_direct3d_points failed ({rc})")
    return ub, tau


PLANTS = ("cross_parity", "drop_cross", "swap_cross", "drop_wall_term", "ubar_parity")


def subfilter_stress_decomposed(dns, les, delta: float, u, U, ext: int = EXT_EVEN_ODD, form: str = "bracket",
                                plant: str | None = None):
    """ubar and T of Eq. 6 written about a profile U[3][ny] (any profile).

    With u_a = U_a(y) + u'_a, h_f = A_z A_x f for f = u'_a and u'_a u'_b, and
    the wall-normal operators A^p of each parity p (Eq. 7 or Eq. 9):
      q_f = A^{p_f} h_f,  AU_a = A^{p_a} U_a,  ubar_a = AU_a + q_a,
      T_ab = [A^{p_ab}(U_a U_b) - AU_a AU_b] + [C_ab - AU_a q_b]
           + [C_ba - AU_b q_a] + [q_ab - q_a q_b],
      C_ab = A^{p_ab} (U_a h_b),  p_ab = p_a p_b,
    which holds because A_x and A_z reproduce functions of y alone (rows
    summing to one) and every operator is linear.  form="deviation" writes the
    cross brackets as
      C_ab - AU_a q_b = sum_j A^{p_ab}[J][j] (U_a(j) - AU_a(J)) h_b(j)
                        + [p_a odd] AU_a(J) ((A^{-p_b} - A^{p_b}) h_b)(J).

    ``plant`` (tests only) names one deliberate mistake, to show that the
    comparison with the plain evaluation catches it: "cross_parity" (cross
    terms filtered with the fluctuation's parity p_b instead of p_a p_b),
    "drop_cross" (the [C_ba - AU_b q_a] bracket left out), "swap_cross" (the
    [C_ab - AU_a q_b] bracket counted twice instead of once per order),
    "drop_wall_term" (deviation form without the [p_a odd] wall term),
    "ubar_parity" (AU_a of the second component with the wrong parity).
    """
    if plant is not None and plant not in PLANTS:
        raise ValueError(f"plant is one of {PLANTS}")
    if form not in ("bracket", "deviation"):
        raise ValueError("form is 'bracket' or 'deviation'")
    if ext not in (EXT_EVEN_ODD, EXT_ODD_EVEN):
        raise ValueError("the decomposition needs a wall extension (Eq. 7 or Eq. 9)")
    u, U = _f64(u), _f64(U)
    assert u.shape == (3, dns.ny, dns.nz, dns.nx) and U.shape == (3, dns.ny)
    Ax = op_periodic(dns.nx, dns.Lx, les.nx, delta)
    Az = op_periodic(dns.nz, dns.Lz, les.nz, delta)
    Ay = {p: op_wall(dns.y, les.y, delta, p) for p in (1, -1)}
    par = (1, -1, 1) if ext == EXT_EVEN_ODD else (-1, 1, -1)
    eye = np.eye(dns.ny)
    up = u - U[:, :, None, None]
    h = [apply_separable(up[a], Ax, eye, Az) for a in range(3)]                 # [ny][nlz][nlx]
    hh = [apply_separable(up[a] * up[b], Ax, eye, Az) for a, b in PAIRS]
    ycon = lambda A, f: np.einsum("Jj,jzx->Jzx", A, f)
    AU = [Ay[-par[a] if (plant == "ubar_parity" and a == 1) else par[a]] @ U[a] for a in range(3)]   # [nly]
    q = [ycon(Ay[par[a]], h[a]) for a in range(3)]
    ubar = np.stack([AU[a][:, None, None] + q[a] for a in range(3)])
    tau = np.zeros((6, les.ny, les.nz, les.nx))
    for k, (a, b) in enumerate(PAIRS):
        pab = par[a] * par[b]
        A = Ay[pab]
        qab = ycon(A, hh[k])

        def cross(c, d):                                                          # C_cd - AU_c q_d
            Ac = Ay[par[d]] if plant == "cross_parity" else A
            if form == "bracket":
                return ycon(Ac, U[c][:, None, None] * h[d]) - AU[c][:, None, None] * q[d]
            dev = np.einsum("Jj,jzx->Jzx", Ac * (U[c][None, :] - AU[c][:, None]), h[d])
            if par[c] < 0 and plant != "drop_wall_term":
                dev = dev + AU[c][:, None, None] * ycon(Ay[-par[d]] - Ay[par[d]], h[d])
            return dev

        prof = (A @ (U[a] * U[b]) - AU[a] * AU[b])[:, None, None]
        second = 0.0 if plant == "drop_cross" else cross(a, b) if plant == "swap_cross" else cross(b, a)
        tau[k] = prof + cross(a, b) + second + (qab - q[a] * q[b])
    return ubar, tau

