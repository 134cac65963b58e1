"""Failure detection without a GPU fault.

* A bounded device wait that nothing completes gives up and records
  EF_ERR_TIMEOUT in the plan's error word; the read clears it, and the same
  plan and context then compute a correct stress (the context stays usable).
* A completed wait records nothing.
* A non-finite input is reported as EF_ERR_NAN by the device scan (the check
  lives in test_parity_gpu.py); host-side argument errors come back as status
  codes (test_abi.py, test_differential_gpu.py).
No test here traps, faults or hangs the GPU: the wait limit is a few thousand
SM clocks and the barrier lives in the self-test kernel's own shared memory.
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


def test_wait_timeout_is_reported_and_recovered():
    dns = I.dns_grid(32, 33, 32, 2 * math.pi, math.pi)
    les = I.les_grid(dns, 8, 9, 8)
    delta = 2 * math.pi / 16
    plan = eles.filter_setup(dns, les, delta, precision=eles.PREC_FP64)
    eles.selftest_wait(plan, 2000, complete=False)
    assert eles.check_device_error(plan) == 5                     # EF_ERR_TIMEOUT
    assert eles.check_device_error(plan) == 0                     # cleared by the read
    eles.selftest_wait(plan, 2000, complete=True)
    assert eles.check_device_error(plan) == 0
    # the same plan still computes the right answer
    u = I.channel_velocity(dns, 3)
    dev = torch.device("cuda")
    ub = torch.empty((3, les.ny, les.nz, les.nx), device=dev, dtype=torch.float64)
    tau = torch.empty((6, les.ny, les.nz, les.nx), device=dev, dtype=torch.float64)
    eles.subfilter_stress(plan, torch.from_numpy(u).to(dev), ub, tau)
    assert eles.check_device_error(plan) == 0
    ub_ref, tau_ref = O.subfilter_stress(dns, les, delta, u)
    assert np.abs(tau.cpu().numpy() - tau_ref).max() <= 1e-12 * np.abs(tau_ref).max()


def test_selftest_argument_errors():
    dns = I.dns_grid(32, 33, 32, 2 * math.pi, math.pi)
    plan = eles.filter_setup(dns, I.les_grid(dns, 8, 9, 8), 2 * math.pi / 16, precision=eles.PREC_FP32)
    with pytest.raises(eles.EFError) as e:
        eles.selftest_wait(plan, 0)
    assert e.value.code == 1


def test_xz_kernel_wait_limit_one_times_out_and_recovers():
    """The warp-specialised x-z kernel with every wait bounded by 1 SM clock:
    the first wait that is not already complete runs out, EF_ERR_TIMEOUT is
    recorded, the roles stop (the producer still waits for its copies in
    flight), and with the default bound restored the same plan computes the
    stress to the oracle's tolerance.  Also through a batch graph."""
    dns = I.dns_grid(128, 65, 128, 2 * math.pi, math.pi)
    les = I.les_grid(dns, 16, 17, 16)
    delta = 12 * math.pi / 128
    u = I.channel_velocity(dns, 41)
    plan = eles.filter_setup(dns, les, delta, precision=eles.PREC_BF16X3)
    assert eles.plan_info(plan, 10) == 3
    dev = torch.device("cuda")
    ud = torch.from_numpy(u).to(dev, torch.float32)
    ub = torch.empty((3, les.ny, les.nz, les.nx), device=dev)
    tau = torch.empty((6, les.ny, les.nz, les.nx), device=dev)
    eles.plan_set_wait_limit(plan, 1)
    eles.subfilter_stress(plan, ud, ub, tau)
    torch.cuda.synchronize()
    assert eles.check_device_error(plan) == 5                  # EF_ERR_TIMEOUT
    eles.plan_set_wait_limit(plan, 0)
    eles.subfilter_stress(plan, ud, ub, tau)
    torch.cuda.synchronize()
    assert eles.check_device_error(plan) == 0
    _, tau_ref = O.subfilter_stress(dns, les, delta, u)
    assert np.abs(tau.double().cpu().numpy() - tau_ref).max() <= 1e-4
    # the same through a batch: the limit reaches the graph's launch arguments
    batch = eles.batch_create([plan], [1])
    us, ubs, taus = [ud[None]], [ub[None]], [tau[None]]
    eles.batch_run(batch, us, ubs, taus)
    eles.plan_set_wait_limit(plan, 1)
    eles.batch_run(batch, us, ubs, taus)
    torch.cuda.synchronize()
    assert eles.batch_captures(batch) == 2
    assert eles.check_device_error(plan) == 5
    eles.plan_set_wait_limit(plan, 0)
    eles.batch_run(batch, us, ubs, taus)
    torch.cuda.synchronize()
    assert eles.check_device_error(plan) == 0
    assert np.abs(taus[0][0].double().cpu().numpy() - tau_ref).max() <= 1e-4
