"""GPU tests of the host-buffer pipeline (ef_subfilter_stress_host).

The pipeline runs the same kernels as ef_subfilter_stress_batch on device
copies of host snapshots, so its outputs must equal the device call's bit
for bit, for every group size (including a ragged last group), with and
without plane means, on repeated calls, and in FP32 and BF16x3; and they
meet the oracle's tolerance.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import __graft_entry__ as entry
from oracle import oracle as O
from paper_1902_02508_gb300 import eles
from paper_1902_02508_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    entry.build()


@pytest.mark.parametrize("prec", [eles.PREC_FP32, eles.PREC_BF16X3, eles.PREC_TF32X2])
@pytest.mark.parametrize("chunk", [1, 2])
def test_host_pipeline_equals_device_call(prec, chunk):
    dns = I.dns_grid(128, 65, 128, 2 * math.pi, math.pi)
    les = I.les_grid(dns, 16, 17, 16)
    delta = 12 * math.pi / 128
    ns = 3
    snaps = [I.channel_velocity(dns, 500 + s) for s in range(ns)]
    plan = eles.filter_setup(dns, les, delta, precision=prec)
    dev = torch.device("cuda")
    u = torch.stack([torch.from_numpy(s) for s in snaps]).to(torch.float32)
    ud = u.to(dev)
    ub = torch.empty((ns, 3, les.ny, les.nz, les.nx), device=dev)
    tau = torch.empty((ns, 6, les.ny, les.nz, les.nx), device=dev)
    pm = torch.empty((ns, 3, dns.ny), device=dev, dtype=torch.float64)
    eles.plan_reserve(plan, ns)
    eles.subfilter_stress_batch(plan, ud, ub, tau, pm)
    torch.cuda.synchronize()
    io = eles.io_create(plan, chunk)
    hu = u.pin_memory()
    stream = torch.cuda.Stream()
    for _ in range(2):
        hb = torch.full(ub.shape, float("nan")).pin_memory()
        ht = torch.full(tau.shape, float("nan")).pin_memory()
        hp = torch.full(pm.shape, float("nan"), dtype=torch.float64).pin_memory()
        eles.subfilter_stress_host(io, hu, hb, ht, hp, stream=stream)
        stream.synchronize()
        assert torch.equal(hb, ub.cpu()) and torch.equal(ht, tau.cpu()) and torch.equal(hp, pm.cpu())
    hb2 = torch.empty(ub.shape).pin_memory()
    ht2 = torch.empty(tau.shape).pin_memory()
    eles.subfilter_stress_host(io, hu, hb2, ht2, None, stream=stream)   # no plane means
    stream.synchronize()
    assert torch.equal(ht2, tau.cpu())
    assert eles.check_device_error(plan) == 0
    _, tau_ref = O.subfilter_stress(dns, les, delta, snaps[-1])
    assert np.abs(ht2[-1].double().numpy() - tau_ref).max() <= 1e-4
    io.close()


def test_host_pipeline_rejects_device_tensors():
    dns = I.dns_grid(32, 33, 32, 2 * math.pi, math.pi)
    les = I.les_grid(dns, 8, 9, 8)
    plan = eles.filter_setup(dns, les, 2 * math.pi / 16, precision=eles.PREC_FP32)
    io = eles.io_create(plan, 1)
    ud = torch.zeros((1, 3, 33, 32, 32), device="cuda")
    hb = torch.empty((1, 3, 9, 8, 8))
    ht = torch.empty((1, 6, 9, 8, 8))
    with pytest.raises(ValueError):
        eles.subfilter_stress_host(io, ud, hb, ht)
    io.close()
