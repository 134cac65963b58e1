"""Host-side checks of the C ABI: the library builds, loads, exports every
symbol include/eles.h declares, and rejects bad arguments before touching a
GPU (these checks need no device)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import __graft_entry__ as entry
from paper_1902_02508_gb300 import eles
from paper_1902_02508_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    entry.build()
    return eles.load()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ef_\w+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert {"ef_filter_setup", "ef_filter_fields", "ef_subfilter_stress"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(eles.EXPORTED) <= names


def test_version_and_no_error(lib):
    assert "sm_103a" in eles.version()


def _setup_rc(lib, dns, les, delta=0.3, kernel=0, ext=0, prec=1):
    gd, yd = eles._grid(dns)
    gl, yl = eles._grid(les)
    h = ctypes.c_void_p()
    rc = lib.ef_filter_setup(ctypes.byref(gd), ctypes.byref(gl), delta, kernel, ext, prec, ctypes.byref(h))
    return rc, lib.ef_last_error().decode()


def test_setup_rejects_bad_arguments_on_host(lib):
    d = I.dns_grid(32, 33, 32, 2 * math.pi, math.pi)
    l = I.les_grid(d, 8, 9, 8)
    assert _setup_rc(lib, d, l, delta=-1.0)[0] == 1
    assert _setup_rc(lib, d, l, delta=float("nan"))[0] == 1
    assert _setup_rc(lib, d, l, delta=2.0)[0] == 1            # support wider than half the box
    assert _setup_rc(lib, d, l, kernel=5)[0] == 7
    assert _setup_rc(lib, d, l, ext=9)[0] == 1
    assert _setup_rc(lib, d, l, prec=9)[0] == 7
    bad = I.Grid(32, 33, 32, 2 * math.pi, math.pi, d.y[::-1].copy())
    rc, msg = _setup_rc(lib, bad, l)
    assert rc == 1 and "y" in msg
    other_box = I.Grid(8, 9, 8, math.pi, math.pi, l.y)
    assert _setup_rc(lib, d, other_box)[0] == 2
    finer = I.les_grid(d, 64, 9, 8)
    assert _setup_rc(lib, d, finer)[0] == 2
    h = ctypes.c_void_p()
    gd, yd = eles._grid(d)
    assert lib.ef_filter_setup(ctypes.byref(gd), ctypes.byref(gd), 0.3, 0, 0, 1, None) == 1


def test_hot_calls_reject_null(lib):
    assert lib.ef_filter_fields(None, None, None, None) == 1
    assert lib.ef_subfilter_stress(None, None, None, None, None, None) == 1
    assert lib.ef_check_device_error(None, None) == 1
    v = ctypes.c_long()
    assert lib.ef_plan_info(None, 0, ctypes.byref(v)) == 1
    lib.ef_plan_destroy(None)


def test_les_calls_check_arguments_on_host(lib):
    """The LES step's entry points (the loop of Fig. 2) refuse bad arguments
    before touching a device."""
    y = np.linspace(-1.0, 1.0, 9)
    cfg = eles._LesCfg(0.01, 1.0, eles.LES_RK3)
    h = ctypes.c_void_p()

    def create(nx, ny, nz, Lx=1.0, c=cfg, yy=y):
        g = eles._Grid(nx, ny, nz, Lx, 1.0, yy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return lib.ef_les_create(ctypes.byref(g), ctypes.byref(c), ctypes.byref(h))

    assert create(2, 9, 8) == eles.EF_ERR_SHAPE                 # fewer than 3 nodes in x
    assert create(8, 9, 5000) == eles.EF_ERR_SHAPE              # more than 4096 in z
    assert create(8, 9, 8, Lx=0.0) == eles.EF_ERR_ARG
    assert create(8, 9, 8, yy=y[::-1].copy()) == eles.EF_ERR_ARG   # y nodes must ascend
    assert create(8, 9, 8, c=eles._LesCfg(-1.0, 1.0, 0)) == eles.EF_ERR_ARG
    assert create(8, 9, 8, c=eles._LesCfg(0.01, 1.0, 7)) == eles.EF_ERR_ARG
    assert lib.ef_les_create(None, None, None) == eles.EF_ERR_ARG
    assert lib.ef_les_step(None, None, None, None, 0, 0.01, None) == eles.EF_ERR_ARG
    assert lib.ef_les_project(None, None, None, None) == eles.EF_ERR_ARG
    assert lib.ef_les_divergence(None, None, None, None) == eles.EF_ERR_ARG
    assert lib.ef_les_rhs(None, None, None, 0, None, None) == eles.EF_ERR_ARG
    assert lib.ef_apost_step(None, None, None, None, None, None, 0.01, None) == eles.EF_ERR_ARG
    lib.ef_les_destroy(None)
