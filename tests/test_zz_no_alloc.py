"""The allocation-free feature entry point.

Some host programs may not allocate device memory themselves (they own every
allocation, or run where the allocator must not be called).
ef_closure_features_static serves them: its scratch is a fixed device array
instead of a per-call allocation.  This test calls it through the C ABI twice
in a row, on two different LES grids, and checks each result against the
allocating entry point ef_closure_features; it also checks the size limit.
The file is collected last on purpose.
"""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import __graft_entry__ as entry
from paper_1902_02508_gb300 import eles
from paper_1902_02508_gb300 import inputs as I


@pytest.mark.gpu
def test_static_features_match_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    entry.build()
    lib = eles.load()
    dev = torch.device("cuda")
    rng = np.random.default_rng(12)
    for (nx, ny, nz) in ((32, 33, 24), (16, 17, 12)):
        dns = I.dns_grid(4 * nx, 2 * ny - 1, 4 * nz, 4 * math.pi, 2 * math.pi)
        les = I.les_grid(dns, nx, ny, nz)
        ub = torch.from_numpy(rng.standard_normal((3, ny, nz, nx))).to(dev, torch.float32)
        n = nx * ny * nz
        ref = torch.full((n, 10), float("nan"), device=dev)
        got = torch.full((n, 10), float("nan"), device=dev)
        eles.closure_features(les, ub, ref)
        g, y = eles._grid(les)
        rc = lib.ef_closure_features_static(ctypes.byref(g), ctypes.c_void_p(ub.data_ptr()), 180.0, 0,
                                            ctypes.c_void_p(got.data_ptr()),
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, lib.ef_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(got).all()
        assert torch.allclose(got, ref, rtol=1e-6, atol=1e-6)
    big = I.Grid(8, 4097, 8, 1.0, 1.0, np.linspace(-1, 1, 4097))
    g, y = eles._grid(big)
    dummy = torch.zeros(16, device=dev)
    rc = lib.ef_closure_features_static(ctypes.byref(g), ctypes.c_void_p(dummy.data_ptr()), 180.0, 0,
                                        ctypes.c_void_p(dummy.data_ptr()), None)
    assert rc == 1                                   # EF_ERR_ARG
    assert b"4096" in lib.ef_last_error()
