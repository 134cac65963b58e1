"""Thin Python binding of the C ABI in include/eles.h (ctypes).

Argument marshalling only: every step of the filter runs in the CUDA library
libeles.so.  PyTorch supplies device memory and streams.  There is no CPU or
PyTorch fallback: if the library is missing the import of a function fails
loudly.

Names follow the C ABI: ``filter_setup``, ``filter_fields``,
``subfilter_stress``, ``check_device_error``, ``plan_info``, ``plan_weights``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = (os.path.join(_HERE, "_lib_check", "libeles_check.so") if os.environ.get("ELES_CHECK") == "1"
            else os.path.join(_HERE, "_lib", "libeles.so"))

EF_OK = 0
EF_ERR_ARG, EF_ERR_SHAPE = 1, 2
STATUS = {0: "EF_OK", 1: "EF_ERR_ARG", 2: "EF_ERR_SHAPE", 3: "EF_ERR_CUDA", 4: "EF_ERR_NAN",
          5: "EF_ERR_TIMEOUT", 6: "EF_ERR_OOM", 7: "EF_ERR_UNSUPPORTED", 8: "EF_ERR_RANGE"}
KERNEL_GAUSSIAN = 0
KERNEL_GAUSSIAN_HAT = 1      # y integral exact against the piecewise-linear interpolant
KERNEL_DIFFERENTIAL = 2      # (1 - a^2 lap) ubar = u, a^2 = delta^2 / 40 (FP64)
EXT_EVEN_ODD, EXT_ODD_EVEN, EXT_NONE = 0, 1, 2
PREC_FP64, PREC_FP32, PREC_TF32X2, PREC_BF16X3 = 0, 1, 2, 3
VARIANT_CUDA_CORE_Y = 256    # or-ed into a variant choice: y contraction on CUDA cores

# every symbol include/eles.h declares
EXPORTED = ("ef_filter_setup", "ef_plan_destroy", "ef_filter_fields", "ef_subfilter_stress",
            "ef_subfilter_stress_batch", "ef_plan_reserve",
            "ef_check_device_error", "ef_plan_info", "ef_plan_weights", "ef_profile_enable",
            "ef_profile_read", "ef_last_error", "ef_version", "ef_closure_create", "ef_closure_destroy",
            "ef_closure_features", "ef_closure_fit_norm", "ef_closure_train", "ef_closure_infer",
            "ef_closure_infer_exact", "ef_plan_set_wait_limit", "ef_debug_fail_alloc",
            "ef_closure_gradients", "ef_closure_param_count", "ef_closure_get_params", "ef_closure_set_params",
            "ef_closure_save", "ef_closure_load", "ef_batch_create", "ef_batch_run", "ef_batch_destroy",
            "ef_batch_captures", "ef_plan_autotune", "ef_plan_set_variant", "ef_closure_features_static", "ef_io_create",
            "ef_closure_check_device_error", "ef_differential_unfilter", "ef_selftest_wait",
            "ef_io_destroy", "ef_subfilter_stress_host", "ef_stats_create", "ef_stats_destroy", "ef_plane_stats",
            "ef_error_field", "ef_error_profile", "ef_les_create", "ef_les_destroy", "ef_les_step",
            "ef_les_project", "ef_les_divergence", "ef_les_rhs", "ef_apost_step")


class EFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("Lx", ctypes.c_double), ("Lz", ctypes.c_double),
                ("y", ctypes.POINTER(ctypes.c_double))]


class _ClosureCfg(ctypes.Structure):
    _fields_ = [("hidden", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_float),
                ("guard_sigma", ctypes.c_float), ("seed", ctypes.c_ulonglong)]


class _LesCfg(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("forcing", ctypes.c_double), ("scheme", ctypes.c_int)]


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libeles.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise ImportError(f"libeles.so not built at {path}; run paper_1902_02508_gb300.build.build()")
            lib = ctypes.CDLL(path)
            vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
            lib.ef_filter_setup.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Grid), d, i, i, i,
                                            ctypes.POINTER(vp)]
            lib.ef_filter_setup.restype = i
            lib.ef_plan_destroy.argtypes = [vp]
            lib.ef_plan_destroy.restype = None
            lib.ef_filter_fields.argtypes = [vp, vp, vp, vp]
            lib.ef_filter_fields.restype = i
            lib.ef_subfilter_stress.argtypes = [vp, vp, vp, vp, vp, vp]
            lib.ef_subfilter_stress.restype = i
            lib.ef_subfilter_stress_batch.argtypes = [vp, i, vp, vp, vp, vp, vp]
            lib.ef_subfilter_stress_batch.restype = i
            lib.ef_plan_reserve.argtypes = [vp, i]
            lib.ef_plan_reserve.restype = i
            lib.ef_check_device_error.argtypes = [vp, vp]
            lib.ef_check_device_error.restype = i
            lib.ef_plan_info.argtypes = [vp, i, ctypes.POINTER(ctypes.c_long)]
            lib.ef_plan_info.restype = i
            lib.ef_plan_weights.argtypes = [vp, i, vp]
            lib.ef_plan_weights.restype = i
            lib.ef_profile_enable.argtypes = [vp, i]
            lib.ef_profile_enable.restype = i
            lib.ef_profile_read.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_long)]
            lib.ef_profile_read.restype = i
            L = ctypes.c_long
            lib.ef_closure_create.argtypes = [ctypes.POINTER(_ClosureCfg), ctypes.POINTER(vp)]
            lib.ef_closure_create.restype = i
            lib.ef_closure_destroy.argtypes = [vp]
            lib.ef_closure_destroy.restype = None
            lib.ef_closure_features.argtypes = [ctypes.POINTER(_Grid), vp, d, i, vp, vp]
            lib.ef_closure_features.restype = i
            lib.ef_closure_features_static.argtypes = [ctypes.POINTER(_Grid), vp, d, i, vp, vp]
            lib.ef_closure_features_static.restype = i
            lib.ef_closure_fit_norm.argtypes = [vp, vp, vp, L, vp]
            lib.ef_closure_fit_norm.restype = i
            lib.ef_closure_train.argtypes = [vp, vp, vp, L, i, vp, ctypes.POINTER(ctypes.c_float)]
            lib.ef_closure_train.restype = i
            lib.ef_closure_infer.argtypes = [vp, vp, vp, L, vp, ctypes.POINTER(L), vp]
            lib.ef_closure_infer.restype = i
            lib.ef_closure_infer_exact.argtypes = [vp, vp, vp, L, vp, vp, ctypes.POINTER(L), vp]
            lib.ef_closure_infer_exact.restype = i
            lib.ef_plan_set_wait_limit.argtypes = [vp, ctypes.c_longlong]
            lib.ef_plan_set_wait_limit.restype = i
            lib.ef_debug_fail_alloc.argtypes = [i]
            lib.ef_debug_fail_alloc.restype = i
            lib.ef_selftest_wait.argtypes = [vp, ctypes.c_longlong, i, vp]
            lib.ef_selftest_wait.restype = i
            lib.ef_differential_unfilter.argtypes = [ctypes.POINTER(_Grid), d, i, vp, vp, vp]
            lib.ef_differential_unfilter.restype = i
            lib.ef_closure_check_device_error.argtypes = [vp, vp]
            lib.ef_closure_check_device_error.restype = i
            lib.ef_closure_gradients.argtypes = [vp, vp, vp, L, vp, ctypes.POINTER(ctypes.c_float), vp]
            lib.ef_closure_gradients.restype = i
            lib.ef_closure_param_count.argtypes = [vp]
            lib.ef_closure_param_count.restype = L
            lib.ef_closure_get_params.argtypes = [vp, vp, vp]
            lib.ef_closure_get_params.restype = i
            lib.ef_closure_set_params.argtypes = [vp, vp, vp]
            lib.ef_closure_set_params.restype = i
            lib.ef_closure_save.argtypes = [vp, ctypes.c_char_p]
            lib.ef_closure_save.restype = i
            lib.ef_closure_load.argtypes = [vp, ctypes.c_char_p]
            lib.ef_closure_load.restype = i
            lib.ef_batch_create.argtypes = [vp, vp, i, ctypes.POINTER(vp)]
            lib.ef_batch_create.restype = i
            lib.ef_batch_run.argtypes = [vp, vp, vp, vp, vp]
            lib.ef_batch_run.restype = i
            lib.ef_batch_destroy.argtypes = [vp]
            lib.ef_batch_destroy.restype = None
            lib.ef_batch_captures.argtypes = [vp]
            lib.ef_batch_captures.restype = L
            lib.ef_plan_autotune.argtypes = [vp, vp, vp, vp, i, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_float)]
            lib.ef_plan_autotune.restype = i
            lib.ef_plan_set_variant.argtypes = [vp, i]
            lib.ef_plan_set_variant.restype = i
            lib.ef_io_create.argtypes = [vp, i, ctypes.POINTER(vp)]
            lib.ef_io_create.restype = i
            lib.ef_io_destroy.argtypes = [vp]
            lib.ef_io_destroy.restype = None
            lib.ef_subfilter_stress_host.argtypes = [vp, i, vp, vp, vp, vp, vp]
            lib.ef_subfilter_stress_host.restype = i
            lib.ef_stats_create.argtypes = [ctypes.POINTER(_Grid), i, ctypes.POINTER(vp)]
            lib.ef_stats_create.restype = i
            lib.ef_stats_destroy.argtypes = [vp]
            lib.ef_stats_destroy.restype = None
            lib.ef_plane_stats.argtypes = [vp, vp, vp, vp, vp]
            lib.ef_plane_stats.restype = i
            lib.ef_error_field.argtypes = [vp, vp, vp, i, ctypes.c_double, ctypes.c_double, vp, vp]
            lib.ef_error_field.restype = i
            lib.ef_error_profile.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_double, vp, vp]
            lib.ef_error_profile.restype = i
            lib.ef_les_create.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_LesCfg), ctypes.POINTER(vp)]
            lib.ef_les_create.restype = i
            lib.ef_les_destroy.argtypes = [vp]
            lib.ef_les_destroy.restype = None
            lib.ef_les_step.argtypes = [vp, vp, vp, vp, i, d, vp]
            lib.ef_les_step.restype = i
            lib.ef_les_project.argtypes = [vp, vp, vp, vp]
            lib.ef_les_project.restype = i
            lib.ef_les_divergence.argtypes = [vp, vp, vp, vp]
            lib.ef_les_divergence.restype = i
            lib.ef_les_rhs.argtypes = [vp, vp, vp, i, vp, vp]
            lib.ef_les_rhs.restype = i
            lib.ef_apost_step.argtypes = [vp, vp, vp, vp, vp, vp, d, vp]
            lib.ef_apost_step.restype = i
            lib.ef_last_error.restype = ctypes.c_char_p
            lib.ef_version.restype = ctypes.c_char_p
            _lib = lib
    return _lib


def _check(rc: int):
    if rc != EF_OK:
        raise EFError(rc, load().ef_last_error().decode())


def _grid(g):
    y = np.ascontiguousarray(g.y, dtype=np.float64)
    s = _Grid(g.nx, g.ny, g.nz, float(g.Lx), float(g.Lz), y.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return s, y


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """Owns an ef_plan*.  Created by filter_setup()."""

    def __init__(self, handle, dns, les, delta, precision):
        self.handle = handle
        self.dns, self.les, self.delta, self.precision = dns, les, delta, precision

    def close(self):
        if self.handle:
            load().ef_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == PREC_FP64 else torch.float32


def filter_setup(dns, les, delta: float, kernel: int = KERNEL_GAUSSIAN,
                 extension: int = EXT_EVEN_ODD, precision: int = PREC_FP32) -> Plan:
    lib = load()
    gd, yd = _grid(dns)
    gl, yl = _grid(les)
    h = ctypes.c_void_p()
    _check(lib.ef_filter_setup(ctypes.byref(gd), ctypes.byref(gl), float(delta), int(kernel),
                               int(extension), int(precision), ctypes.byref(h)))
    return Plan(h, dns, les, delta, precision)


def _field(t, shape, dtype, name):
    if t is None:
        return None
    if not t.is_cuda or t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name}: need a contiguous CUDA {dtype} tensor of shape {shape}, "
                         f"got {t.dtype} {tuple(t.shape)} on {t.device}")
    return ctypes.c_void_p(t.data_ptr())


def filter_fields(plan: Plan, u, ubar, stream=None) -> None:
    d, l = plan.dns, plan.les
    pu = _field(u, (3, d.ny, d.nz, d.nx), plan.dtype, "u")
    pb = _field(ubar, (3, l.ny, l.nz, l.nx), plan.dtype, "ubar")
    _check(load().ef_filter_fields(plan.handle, pu, pb, _stream(stream)))


def subfilter_stress(plan: Plan, u, ubar, tau, plane_mean=None, stream=None) -> None:
    import torch
    d, l = plan.dns, plan.les
    pu = _field(u, (3, d.ny, d.nz, d.nx), plan.dtype, "u")
    pb = _field(ubar, (3, l.ny, l.nz, l.nx), plan.dtype, "ubar")
    pt = _field(tau, (6, l.ny, l.nz, l.nx), plan.dtype, "tau")
    pm = _field(plane_mean, (3, d.ny), torch.float64, "plane_mean")
    _check(load().ef_subfilter_stress(plan.handle, pu, pb, pt, pm, _stream(stream)))


def subfilter_stress_batch(plan: Plan, u, ubar, tau, plane_mean=None, stream=None) -> None:
    """u [S][3][ny][nz][nx], ubar [S][3][..], tau [S][6][..], plane_mean [S][3][ny] or None."""
    import torch
    d, l = plan.dns, plan.les
    ns = u.shape[0]
    pu = _field(u, (ns, 3, d.ny, d.nz, d.nx), plan.dtype, "u")
    pb = _field(ubar, (ns, 3, l.ny, l.nz, l.nx), plan.dtype, "ubar")
    pt = _field(tau, (ns, 6, l.ny, l.nz, l.nx), plan.dtype, "tau")
    pm = _field(plane_mean, (ns, 3, d.ny), torch.float64, "plane_mean")
    _check(load().ef_subfilter_stress_batch(plan.handle, ns, pu, pb, pt, pm, _stream(stream)))


def plan_reserve(plan: Plan, max_snapshots: int) -> None:
    _check(load().ef_plan_reserve(plan.handle, int(max_snapshots)))


def debug_fail_alloc(n: int) -> None:
    """Make the n-th device allocation of the library from now fail (-1: off)."""
    _check(load().ef_debug_fail_alloc(int(n)))


def plan_set_wait_limit(plan: Plan, cycles: int) -> None:
    """Bound of every wait in the warp-specialised x-z kernel (0: default)."""
    _check(load().ef_plan_set_wait_limit(plan.handle, int(cycles)))


def check_device_error(plan: Plan, stream=None) -> int:
    return load().ef_check_device_error(plan.handle, _stream(stream))


def plan_info(plan: Plan, what: int) -> int:
    v = ctypes.c_long()
    _check(load().ef_plan_info(plan.handle, int(what), ctypes.byref(v)))
    return v.value


def plan_weights(plan: Plan, which: int) -> np.ndarray:
    d, l = plan.dns, plan.les
    shape = {0: (l.nx, d.nx), 1: (l.nz, d.nz), 2: (l.ny, d.ny), 3: (l.ny, d.ny)}[which]
    out = np.zeros(shape)
    _check(load().ef_plan_weights(plan.handle, int(which), out.ctypes.data_as(ctypes.c_void_p)))
    return out


def profile_enable(plan: Plan, on: bool = True) -> None:
    _check(load().ef_profile_enable(plan.handle, 1 if on else 0))


def profile_read(plan: Plan):
    """(ms per phase [x+z, 0, y + recovery, 0], calls) summed since profile_enable."""
    ms = np.zeros(4)
    n = ctypes.c_long()
    _check(load().ef_profile_read(plan.handle, ms.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n)))
    return ms, n.value


def version() -> str:
    return load().ef_version().decode()


# ----------------------------------------------------------------- closure --
class Closure:
    """Owns an ef_closure*.  Created by closure_create()."""

    def __init__(self, handle, cfg):
        self.handle, self.cfg = handle, cfg

    def close(self):
        if self.handle:
            load().ef_closure_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def closure_create(batch: int = 4096, lr: float = 1e-3, guard_sigma: float = 8.0, seed: int = 1,
                   hidden: int = 128) -> Closure:
    cfg = _ClosureCfg(hidden, batch, lr, guard_sigma, seed)
    h = ctypes.c_void_p()
    _check(load().ef_closure_create(ctypes.byref(cfg), ctypes.byref(h)))
    return Closure(h, cfg)


def closure_features(les, ubar, feats, re_tau: float = 180.0, extension: int = EXT_EVEN_ODD, stream=None):
    import torch
    g, y = _grid(les)
    n = les.nx * les.ny * les.nz
    pb = _field(ubar, (3, les.ny, les.nz, les.nx), torch.float32, "ubar")
    pf = _field(feats, (n, 10), torch.float32, "feats")
    _check(load().ef_closure_features(ctypes.byref(g), pb, float(re_tau), int(extension), pf, _stream(stream)))


def closure_features_static(les, ubar, feats, re_tau: float = 180.0, extension: int = EXT_EVEN_ODD,
                            stream=None):
    """ef_closure_features without any device allocation (static scratch)."""
    import torch
    g, y = _grid(les)
    n = les.nx * les.ny * les.nz
    pb = _field(ubar, (3, les.ny, les.nz, les.nx), torch.float32, "ubar")
    pf = _field(feats, (n, 10), torch.float32, "feats")
    _check(load().ef_closure_features_static(ctypes.byref(g), pb, float(re_tau), int(extension), pf,
                                             _stream(stream)))


def _n_feats(feats):
    if feats.dim() != 2 or feats.shape[1] != 10:
        raise ValueError("feats must be [N][10]")
    return feats.shape[0]


def closure_fit_norm(cl: Closure, feats, tau, stream=None):
    import torch
    n = _n_feats(feats)
    _check(load().ef_closure_fit_norm(cl.handle, _field(feats, (n, 10), torch.float32, "feats"),
                                      _field(tau, (6, n), torch.float32, "tau"), n, _stream(stream)))


def closure_train(cl: Closure, feats, tau, epochs: int, stream=None) -> float:
    import torch
    n = _n_feats(feats)
    loss = ctypes.c_float()
    _check(load().ef_closure_train(cl.handle, _field(feats, (n, 10), torch.float32, "feats"),
                                   _field(tau, (6, n), torch.float32, "tau"), n, int(epochs), _stream(stream),
                                   ctypes.byref(loss)))
    return loss.value


def closure_infer(cl: Closure, feats, tau_out, exact_tau=None, stream=None, count: bool = True):
    """Tensor-core inference; returns the number of guarded points (count=True,
    synchronises) or None (count=False: asynchronous on the stream)."""
    import torch
    n = _n_feats(feats)
    nf = ctypes.c_long()
    _check(load().ef_closure_infer(cl.handle, _field(feats, (n, 10), torch.float32, "feats"),
                                   _field(tau_out, (6, n), torch.float32, "tau_out"), n,
                                   _field(exact_tau, (6, n), torch.float32, "exact_tau"),
                                   ctypes.byref(nf) if count else None, _stream(stream)))
    return nf.value if count else None


def closure_infer_exact(cl: Closure, feats, tau_out, plan: Plan, u, stream=None, count: bool = True):
    """Tensor-core inference with the exact stress of `plan` on the DNS
    snapshot u [3][ny][nz][nx] at the guarded points; returns their number
    (count=True, synchronises) or None."""
    import torch
    n = _n_feats(feats)
    d = plan.dns
    nf = ctypes.c_long()
    _check(load().ef_closure_infer_exact(cl.handle, _field(feats, (n, 10), torch.float32, "feats"),
                                         _field(tau_out, (6, n), torch.float32, "tau_out"), n, plan.handle,
                                         _field(u, (3, d.ny, d.nz, d.nx), plan.dtype, "u"),
                                         ctypes.byref(nf) if count else None, _stream(stream)))
    return nf.value if count else None


def selftest_wait(plan: Plan, limit_cycles: int, complete: bool = False, stream=None):
    """Run the bounded-wait self-test on the plan's error word (asynchronous)."""
    _check(load().ef_selftest_wait(plan.handle, int(limit_cycles), 1 if complete else 0, _stream(stream)))


def differential_unfilter(grid, delta: float, u, out, extension: int = EXT_EVEN_ODD, stream=None):
    """(1 - a^2 lap) u on `grid` (the inverse of the differential filter), FP64."""
    import torch
    g, _y = _grid(grid)
    shape = (3, grid.ny, grid.nz, grid.nx)
    _check(load().ef_differential_unfilter(ctypes.byref(g), float(delta), int(extension),
                                           _field(u, shape, torch.float64, "u"), _field(out, shape, torch.float64, "out"),
                                           _stream(stream)))


def closure_check_device_error(cl: Closure, stream=None) -> int:
    """Read and clear the closure's device error word (0 = none)."""
    return load().ef_closure_check_device_error(cl.handle, _stream(stream))


def closure_param_count(cl: Closure) -> int:
    return load().ef_closure_param_count(cl.handle)


def closure_gradients(cl: Closure, feats, tau, stream=None):
    import torch
    n = _n_feats(feats)
    g = np.zeros(closure_param_count(cl), dtype=np.float32)
    loss = ctypes.c_float()
    _check(load().ef_closure_gradients(cl.handle, _field(feats, (n, 10), torch.float32, "feats"),
                                       _field(tau, (6, n), torch.float32, "tau"), n,
                                       g.ctypes.data_as(ctypes.c_void_p), ctypes.byref(loss), _stream(stream)))
    return g, loss.value


def closure_get_params(cl: Closure):
    p = np.zeros(closure_param_count(cl), dtype=np.float32)
    st = np.zeros(32)
    _check(load().ef_closure_get_params(cl.handle, p.ctypes.data_as(ctypes.c_void_p), st.ctypes.data_as(ctypes.c_void_p)))
    return p, st


def closure_set_params(cl: Closure, params=None, stats=None):
    pp = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
    ss = None if stats is None else np.ascontiguousarray(stats, dtype=np.float64)
    _check(load().ef_closure_set_params(cl.handle, None if pp is None else pp.ctypes.data_as(ctypes.c_void_p),
                                        None if ss is None else ss.ctypes.data_as(ctypes.c_void_p)))


def closure_save(cl: Closure, path: str):
    _check(load().ef_closure_save(cl.handle, path.encode()))


def closure_load(cl: Closure, path: str):
    _check(load().ef_closure_load(cl.handle, path.encode()))


CLOSURE_LAYERS = ((10, 128), (128, 128), (128, 128), (128, 6))


def closure_unpack(params):
    """Flat parameter vector -> [(W [out][in], b [out]), ...]."""
    out, off = [], 0
    for fi, fo in CLOSURE_LAYERS:
        W = params[off:off + fi * fo].reshape(fo, fi)
        off += fi * fo
        b = params[off:off + fo]
        off += fo
        out.append((W, b))
    return out


# ------------------------------------------------------------------ batches --
class Batch:
    """Owns an ef_batch*: items (plan, snapshots) replayed as one CUDA graph."""

    def __init__(self, handle, plans, nsnap):
        self.handle, self.plans, self.nsnap = handle, plans, nsnap

    def close(self):
        if self.handle:
            load().ef_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_create(plans, nsnap) -> Batch:
    hp = (ctypes.c_void_p * len(plans))(*[p.handle for p in plans])
    ns = (ctypes.c_int * len(plans))(*nsnap)
    h = ctypes.c_void_p()
    _check(load().ef_batch_create(hp, ns, len(plans), ctypes.byref(h)))
    return Batch(h, list(plans), list(nsnap))


def batch_run(batch: Batch, us, ubars, taus, stream=None) -> None:
    n = len(batch.plans)
    for k, (p, ns) in enumerate(zip(batch.plans, batch.nsnap)):
        d, l = p.dns, p.les
        _field(us[k], (ns, 3, d.ny, d.nz, d.nx), p.dtype, f"u[{k}]")
        _field(ubars[k], (ns, 3, l.ny, l.nz, l.nx), p.dtype, f"ubar[{k}]")
        _field(taus[k], (ns, 6, l.ny, l.nz, l.nx), p.dtype, f"tau[{k}]")
    pu = (ctypes.c_void_p * n)(*[t.data_ptr() for t in us])
    pb = (ctypes.c_void_p * n)(*[t.data_ptr() for t in ubars])
    pt = (ctypes.c_void_p * n)(*[t.data_ptr() for t in taus])
    _check(load().ef_batch_run(batch.handle, pu, pb, pt, _stream(stream)))


def batch_captures(batch: Batch) -> int:
    """How many times the batch has captured its CUDA graph."""
    return int(load().ef_batch_captures(batch.handle))


def plan_autotune(plan: Plan, u, ubar, tau, reps: int = 3):
    """Returns (choice, ms): choice = variant * 16 + columns per z phase."""
    d, l = plan.dns, plan.les
    pu = _field(u, (3, d.ny, d.nz, d.nx), plan.dtype, "u")
    pb = _field(ubar, (3, l.ny, l.nz, l.nx), plan.dtype, "ubar")
    pt = _field(tau, (6, l.ny, l.nz, l.nx), plan.dtype, "tau")
    ch, ms = ctypes.c_int(), ctypes.c_float()
    _check(load().ef_plan_autotune(plan.handle, pu, pb, pt, int(reps), ctypes.byref(ch), ctypes.byref(ms)))
    return ch.value, ms.value


def plan_set_variant(plan: Plan, choice: int) -> None:
    _check(load().ef_plan_set_variant(plan.handle, int(choice)))


class HostIO:
    """Owns an ef_io*: the host-buffer pipeline of one plan."""

    def __init__(self, handle, plan, chunk):
        self.handle, self.plan, self.chunk = handle, plan, chunk

    def close(self):
        if self.handle:
            load().ef_io_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def io_create(plan: Plan, chunk: int = 1) -> HostIO:
    """Set-up call: device slots of `chunk` snapshots for ef_subfilter_stress_host."""
    h = ctypes.c_void_p()
    _check(load().ef_io_create(plan.handle, int(chunk), ctypes.byref(h)))
    return HostIO(h, plan, chunk)


def _host_field(t, shape, dtype, name):
    if t is None:
        return None
    if t.is_cuda or t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name}: need a contiguous host {dtype} tensor of shape {shape}, "
                         f"got {t.dtype} {tuple(t.shape)} on {t.device}")
    return ctypes.c_void_p(t.data_ptr())


def subfilter_stress_host(io: HostIO, u, ubar, tau, plane_mean=None, stream=None) -> None:
    """Host (preferably pinned) tensors: u [S][3][ny][nz][nx], ubar [S][3][..],
    tau [S][6][..], plane_mean [S][3][ny] (float64) or None.  Asynchronous on
    `stream`; synchronise it before reading the outputs."""
    import torch
    plan = io.plan
    d, l = plan.dns, plan.les
    ns = u.shape[0]
    pu = _host_field(u, (ns, 3, d.ny, d.nz, d.nx), plan.dtype, "u")
    pb = _host_field(ubar, (ns, 3, l.ny, l.nz, l.nx), plan.dtype, "ubar")
    pt = _host_field(tau, (ns, 6, l.ny, l.nz, l.nx), plan.dtype, "tau")
    pm = _host_field(plane_mean, (ns, 3, d.ny), torch.float64, "plane_mean")
    _check(load().ef_subfilter_stress_host(io.handle, ns, pu, pb, pt, pm, _stream(stream)))


class Stats:
    """Owns an ef_stats*: the Sec. 4 error measures for fields on one grid."""

    def __init__(self, handle, grid, precision):
        self.handle, self.grid, self.precision = handle, grid, precision

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == PREC_FP64 else torch.float32

    def close(self):
        if self.handle:
            load().ef_stats_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stats_create(grid, precision: int = PREC_FP32) -> Stats:
    g, y = _grid(grid)
    h = ctypes.c_void_p()
    _check(load().ef_stats_create(ctypes.byref(g), int(precision), ctypes.byref(h)))
    return Stats(h, grid, precision)


def plane_stats(st: Stats, u, mean, rms, stream=None) -> None:
    """u [3][ny][nz][nx] (device); mean, rms device float64 [3][ny]."""
    import torch
    g = st.grid
    pu = _field(u, (3, g.ny, g.nz, g.nx), st.dtype, "u")
    pm = _field(mean, (3, g.ny), torch.float64, "mean")
    pr = _field(rms, (3, g.ny), torch.float64, "rms")
    _check(load().ef_plane_stats(st.handle, pu, pm, pr, _stream(stream)))


def error_field(st: Stats, a, b, err, component: int = 0, utau_a: float = 1.0, utau_b: float = 1.0,
                stream=None) -> None:
    """Eq. 13 of component `component`: a, b [3][ny][nz][nx] (device); err device float64 [1]."""
    import torch
    g = st.grid
    pa = _field(a, (3, g.ny, g.nz, g.nx), st.dtype, "a")
    pb = _field(b, (3, g.ny, g.nz, g.nx), st.dtype, "b")
    pe = _field(err, (1,), torch.float64, "err")
    _check(load().ef_error_field(st.handle, pa, pb, int(component), float(utau_a), float(utau_b), pe,
                                 _stream(stream)))


def error_profile(st: Stats, pa, pb, err, utau_a: float = 1.0, utau_b: float = 1.0, stream=None) -> None:
    """Eq. 14 / 15: profiles pa, pb device float64 [ny]; err device float64 [1]."""
    import torch
    g = st.grid
    a = _field(pa, (g.ny,), torch.float64, "pa")
    b = _field(pb, (g.ny,), torch.float64, "pb")
    pe = _field(err, (1,), torch.float64, "err")
    _check(load().ef_error_profile(st.handle, a, b, float(utau_a), float(utau_b), pe, _stream(stream)))


LES_RK3 = 0
LES_EULER = 1


class Les:
    """Owns an ef_les*: the minimal LES solver of the loop of Fig. 2."""

    def __init__(self, handle, grid, cfg):
        self.handle, self.grid, self.cfg = handle, grid, cfg

    def close(self):
        if self.handle:
            load().ef_les_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def les_create(grid, nu: float, forcing: float = 1.0, scheme: int = LES_RK3) -> Les:
    g, y = _grid(grid)
    cfg = _LesCfg(float(nu), float(forcing), int(scheme))
    h = ctypes.c_void_p()
    _check(load().ef_les_create(ctypes.byref(g), ctypes.byref(cfg), ctypes.byref(h)))
    return Les(h, grid, cfg)


def _les_shape(les: Les, ncomp: int):
    g = les.grid
    return (ncomp, g.ny, g.nz, g.nx)


def _prec_of(*tensors):
    import torch
    dts = {t.dtype for t in tensors if t is not None}
    if len(dts) > 1:
        raise ValueError("tau and ubar_bc must share one dtype")
    dt = dts.pop() if dts else torch.float64
    return (PREC_FP64 if dt == torch.float64 else PREC_FP32), dt


def les_step(les: Les, ubar, dt: float, tau=None, ubar_bc=None, stream=None) -> None:
    """One step in place on ubar (device float64 [3][ny][nz][nx]); tau
    [6][..] and ubar_bc [3][..] float64 or float32 (or None)."""
    import torch
    prec, tdt = _prec_of(tau, ubar_bc)
    pu = _field(ubar, _les_shape(les, 3), torch.float64, "ubar")
    pt = _field(tau, _les_shape(les, 6), tdt, "tau")
    pb = _field(ubar_bc, _les_shape(les, 3), tdt, "ubar_bc")
    _check(load().ef_les_step(les.handle, pu, pt, pb, prec, float(dt), _stream(stream)))


def les_project(les: Les, ustar, u, stream=None) -> None:
    import torch
    a = _field(ustar, _les_shape(les, 3), torch.float64, "ustar")
    b = _field(u, _les_shape(les, 3), torch.float64, "u")
    _check(load().ef_les_project(les.handle, a, b, _stream(stream)))


def les_divergence(les: Les, u, div, stream=None) -> None:
    import torch
    a = _field(u, _les_shape(les, 3), torch.float64, "u")
    b = _field(div, _les_shape(les, 1)[1:], torch.float64, "div")
    _check(load().ef_les_divergence(les.handle, a, b, _stream(stream)))


def les_rhs(les: Les, u, rhs, tau=None, stream=None) -> None:
    import torch
    prec, tdt = _prec_of(tau)
    a = _field(u, _les_shape(les, 3), torch.float64, "u")
    pt = _field(tau, _les_shape(les, 6), tdt, "tau")
    b = _field(rhs, _les_shape(les, 3), torch.float64, "rhs")
    _check(load().ef_les_rhs(les.handle, a, pt, prec, b, _stream(stream)))


def apost_step(plan: Plan, les: Les, u_dns, ubar_dns, tau, ubar_les, dt: float, stream=None) -> None:
    """Fig. 2: the filter of the DNS snapshot u_dns (T_ij into tau, ubar into
    ubar_dns; the plan's dtype), then one LES step of ubar_les (float64)."""
    import torch
    d, l = plan.dns, plan.les
    pu = _field(u_dns, (3, d.ny, d.nz, d.nx), plan.dtype, "u_dns")
    pb = _field(ubar_dns, (3, l.ny, l.nz, l.nx), plan.dtype, "ubar_dns")
    pt = _field(tau, (6, l.ny, l.nz, l.nx), plan.dtype, "tau")
    pl = _field(ubar_les, _les_shape(les, 3), torch.float64, "ubar_les")
    _check(load().ef_apost_step(plan.handle, les.handle, pu, pb, pt, pl, float(dt), _stream(stream)))
