"""GPU tests of the two debug aids (no GPU fault is provoked by either).

* The allocation hook (ef_debug_fail_alloc): for every device allocation a
  set-up call makes, making exactly that one fail returns EF_ERR_OOM, frees
  what the call had allocated, and leaves the library usable.
* The range-checked build (ELES_CHECK=1 selects _lib_check/libeles_check.so,
  compiled with -DELES_CHECK): the hot-path kernels check their global
  indices; on the tensor-core geometries (one and several output phases,
  x strides 8 and 4, a batch) no check fires and the results equal the
  normal build's bit for bit.
"""
import math
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import __graft_entry__ as entry
from paper_1902_02508_gb300 import eles
from paper_1902_02508_gb300 import inputs as I

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    entry.build()


def _fail_each_allocation(make):
    """Fail allocation k = 0, 1, ... of make() until it succeeds; returns the
    number of allocations it makes."""
    k = 0
    while True:
        eles.debug_fail_alloc(k)
        try:
            obj = make()
        except eles.EFError as e:
            assert e.code == 6, f"allocation {k}: {e}"          # EF_ERR_OOM
            k += 1
            assert k < 200
            continue
        eles.debug_fail_alloc(-1)
        obj.close()
        return k


def test_allocation_failures_are_reported_and_released():
    dns = I.dns_grid(128, 65, 128, 2 * math.pi, math.pi)
    les = I.les_grid(dns, 16, 17, 16)
    delta = 12 * math.pi / 128
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    makers = {
        "plan bf16x3": lambda: eles.filter_setup(dns, les, delta, precision=eles.PREC_BF16X3),
        "plan fp64": lambda: eles.filter_setup(dns, les, delta, precision=eles.PREC_FP64),
        "plan differential": lambda: eles.filter_setup(dns, les, 0.3, kernel=eles.KERNEL_DIFFERENTIAL,
                                                       precision=eles.PREC_FP32),
        "closure": lambda: eles.closure_create(batch=1024, seed=2),
        "stats": lambda: eles.stats_create(dns),
    }
    counts = {name: _fail_each_allocation(make) for name, make in makers.items()}
    assert all(n >= 1 for n in counts.values()), counts
    # the library still works, and the failed set-ups left nothing allocated
    plan = eles.filter_setup(dns, les, delta, precision=eles.PREC_FP32)
    u = torch.from_numpy(I.channel_velocity(dns, 5)).to("cuda", torch.float32)
    ub = torch.empty((3, les.ny, les.nz, les.nx), device="cuda")
    tau = torch.empty((6, les.ny, les.nz, les.nx), device="cuda")
    eles.subfilter_stress(plan, u, ub, tau)
    torch.cuda.synchronize()
    assert eles.check_device_error(plan) == 0
    plan.close()
    del u, ub, tau
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < 64 << 20, (free0 - free1, counts)


_CHECK_RUN = r"""
import math, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
from paper_1902_02508_gb300 import build, eles, inputs as I
build.build(check=True)
assert "range-checked" in eles.version(), eles.version()
cases = [(128, 65, 128, 2 * math.pi, math.pi, 16, 17, 16, 12 * math.pi / 128),
         (128, 65, 128, 2 * math.pi, math.pi, 16, 17, 16, 24 * math.pi / 128),
         (128, 65, 128, 4 * math.pi, 2 * math.pi, 32, 17, 32, 4 * math.pi / 20),
         (192, 33, 256, 2 * math.pi, math.pi, 24, 17, 32, 10 * math.pi / 192)]
for prec in (eles.PREC_BF16X3, eles.PREC_TF32X2):
    plans, us, ubs, taus = [], [], [], []
    for nx, ny, nz, Lx, Lz, nlx, nly, nlz, delta in cases:
        dns = I.dns_grid(nx, ny, nz, Lx, Lz)
        les = I.les_grid(dns, nlx, nly, nlz)
        plan = eles.filter_setup(dns, les, delta, precision=prec)
        u = torch.from_numpy(np.stack([I.channel_velocity(dns, 3), I.channel_velocity(dns, 4)])).to("cuda", torch.float32)
        ub = torch.empty((2, 3, les.ny, les.nz, les.nx), device="cuda")
        tau = torch.empty((2, 6, les.ny, les.nz, les.nx), device="cuda")
        pm = torch.empty((2, 3, dns.ny), device="cuda", dtype=torch.float64)
        eles.plan_reserve(plan, 2)
        eles.subfilter_stress_batch(plan, u, ub, tau, pm)
        torch.cuda.synchronize()
        assert eles.check_device_error(plan) == 0, "range check fired"
        np.save(OUT + f"/tau_{prec}_{len(plans)}.npy", tau.cpu().numpy())
        plans.append(plan); us.append(u); ubs.append(ub); taus.append(tau)
    batch = eles.batch_create(plans, [2] * len(plans))
    eles.batch_run(batch, us, ubs, taus)
    torch.cuda.synchronize()
    for p in plans:
        assert eles.check_device_error(p) == 0, "range check fired in the batch"
print("check-build ok")
"""


def test_range_checked_build_matches_and_stays_silent(tmp_path):
    env = dict(os.environ, ELES_CHECK="1")
    code = _CHECK_RUN.replace("ROOT", repr(ROOT)).replace("OUT", repr(str(tmp_path)))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "check-build ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
    # the normal build gives the same bits
    cases = [(128, 65, 128, 2 * math.pi, math.pi, 16, 17, 16, 12 * math.pi / 128),
             (128, 65, 128, 2 * math.pi, math.pi, 16, 17, 16, 24 * math.pi / 128),
             (128, 65, 128, 4 * math.pi, 2 * math.pi, 32, 17, 32, 4 * math.pi / 20),
             (192, 33, 256, 2 * math.pi, math.pi, 24, 17, 32, 10 * math.pi / 192)]
    for prec in (eles.PREC_BF16X3, eles.PREC_TF32X2):
        for k, (nx, ny, nz, Lx, Lz, nlx, nly, nlz, delta) in enumerate(cases):
            dns = I.dns_grid(nx, ny, nz, Lx, Lz)
            les = I.les_grid(dns, nlx, nly, nlz)
            plan = eles.filter_setup(dns, les, delta, precision=prec)
            u = torch.from_numpy(np.stack([I.channel_velocity(dns, 3), I.channel_velocity(dns, 4)])).to("cuda",
                                                                                                      torch.float32)
            ub = torch.empty((2, 3, les.ny, les.nz, les.nx), device="cuda")
            tau = torch.empty((2, 6, les.ny, les.nz, les.nx), device="cuda")
            eles.plan_reserve(plan, 2)
            eles.subfilter_stress_batch(plan, u, ub, tau)
            torch.cuda.synchronize()
            assert np.array_equal(tau.cpu().numpy(), np.load(tmp_path / f"tau_{prec}_{k}.npy")), (prec, k)
