"""GPU tests of batches over several plans (one CUDA graph) and of the
autotuner: every variant it can pick meets the oracle tolerance, and a batch
gives the same bits as the plans called one by one."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import __graft_entry__ as entry
from oracle import oracle as O
from paper_1902_02508_gb300 import autotune
from paper_1902_02508_gb300 import eles
from paper_1902_02508_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    entry.build()


# (nx, ny, nz, nlx, nly, nlz, delta fraction of Lx) in the 4 pi x 2 x 2 pi box
ITEMS = [(64, 49, 64, 16, 13, 16, 1 / 16), (192, 49, 128, 48, 13, 32, 1 / 32), (128, 65, 128, 32, 17, 32, 1 / 48)]


def make(item, prec):
    nx, ny, nz, nlx, nly, nlz, f = item
    dns = I.dns_grid(nx, ny, nz, 4 * math.pi, 2 * math.pi)
    les = I.les_grid(dns, nlx, nly, nlz)
    return dns, les, f * dns.Lx, eles.filter_setup(dns, les, f * dns.Lx, precision=prec)


@pytest.mark.parametrize("prec", [eles.PREC_FP32, eles.PREC_BF16X3, eles.PREC_TF32X2])
def test_batch_graph_equals_single_calls(prec):
    dev = torch.device("cuda")
    nsnap = [2, 1, 3]
    plans, us, ubs, taus, cases = [], [], [], [], []
    for k, (item, ns) in enumerate(zip(ITEMS, nsnap)):
        dns, les, delta, plan = make(item, prec)
        u = np.stack([I.channel_velocity(dns, 100 * k + s) for s in range(ns)])
        plans.append(plan)
        cases.append((dns, les, delta, u))
        us.append(torch.from_numpy(u).to(dev, torch.float32))
        ubs.append(torch.empty((ns, 3, les.ny, les.nz, les.nx), device=dev))
        taus.append(torch.empty((ns, 6, les.ny, les.nz, les.nx), device=dev))
    batch = eles.batch_create(plans, nsnap)
    for _ in range(2):                      # capture, then replay
        eles.batch_run(batch, us, ubs, taus)
    torch.cuda.synchronize()
    for k, (plan, ns) in enumerate(zip(plans, nsnap)):
        dns, les, delta, u = cases[k]
        ub1 = torch.empty_like(ubs[k])
        t1 = torch.empty_like(taus[k])
        eles.subfilter_stress_batch(plan, us[k], ub1, t1)
        torch.cuda.synchronize()
        assert torch.equal(ub1, ubs[k]) and torch.equal(t1, taus[k])
        _, tau_ref = O.subfilter_stress(dns, les, delta, u[-1])
        assert np.abs(taus[k][-1].double().cpu().numpy() - tau_ref).max() <= 1e-4


def test_autotune_choices_all_meet_tolerance(tmp_path):
    dev = torch.device("cuda")
    item = (128, 65, 128, 16, 17, 16, 6 / 128)   # stride 8, short ring: every variant exists
    nx, ny, nz, nlx, nly, nlz, f = item
    dns = I.dns_grid(nx, ny, nz, 2 * math.pi, math.pi)
    les = I.les_grid(dns, nlx, nly, nlz)
    delta = 12 * math.pi / 128
    u = I.channel_velocity(dns, 77)
    _, tau_ref = O.subfilter_stress(dns, les, delta, u)
    plan = eles.filter_setup(dns, les, delta, precision=eles.PREC_BF16X3)
    ud = torch.from_numpy(u).to(dev, torch.float32)
    ub = torch.empty((3, les.ny, les.nz, les.nx), device=dev)
    tau = torch.empty((6, les.ny, les.nz, les.nx), device=dev)
    res = autotune.tune(plan, ud, ub, tau, cache_path=str(tmp_path / "tune.json"))
    assert not res["cached"] and res["ms"] > 0
    again = autotune.tune(plan, ud, ub, tau, cache_path=str(tmp_path / "tune.json"))
    assert again["cached"] and again["choice"] == res["choice"]
    for choice in (0 * 16 + 8, 1 * 16 + 4, 2 * 16 + 2, 2 * 16 + 8, 3 * 16 + 2, res["choice"]):
        eles.plan_set_variant(plan, choice)
        eles.subfilter_stress(plan, ud, ub, tau)
        torch.cuda.synchronize()
        assert np.abs(tau.double().cpu().numpy() - tau_ref).max() <= 1e-4, choice


def test_batch_recaptures_after_scratch_or_variant_change():
    """A batch graph holds each plan's scratch pointers and kernel choice: after
    ef_plan_reserve grows a plan's scratch (freeing the old buffers) or
    ef_plan_set_variant changes its kernel, the next run captures again and
    the results still match the oracle."""
    dev = torch.device("cuda")
    plans, us, ubs, taus, cases = [], [], [], [], []
    for k, item in enumerate(ITEMS[:2]):
        dns, les, delta, plan = make(item, eles.PREC_BF16X3)
        u = I.channel_velocity(dns, 300 + k)[None]
        plans.append(plan)
        cases.append((dns, les, delta, u))
        us.append(torch.from_numpy(u).to(dev, torch.float32))
        ubs.append(torch.empty((1, 3, les.ny, les.nz, les.nx), device=dev))
        taus.append(torch.empty((1, 6, les.ny, les.nz, les.nx), device=dev))
    batch = eles.batch_create(plans, [1, 1])
    eles.batch_run(batch, us, ubs, taus)
    eles.batch_run(batch, us, ubs, taus)
    assert eles.batch_captures(batch) == 1
    eles.plan_reserve(plans[0], 4)                 # frees and reallocates plan 0's scratch
    for t in taus:
        t.fill_(float("nan"))
    eles.batch_run(batch, us, ubs, taus)
    assert eles.batch_captures(batch) == 2
    eles.plan_set_variant(plans[1], 0 * 16 + 8)    # unfused CUDA-core kernels
    eles.batch_run(batch, us, ubs, taus)
    assert eles.batch_captures(batch) == 3
    torch.cuda.synchronize()
    for k, (dns, les, delta, u) in enumerate(cases):
        _, tau_ref = O.subfilter_stress(dns, les, delta, u[0])
        assert np.abs(taus[k][0].double().cpu().numpy() - tau_ref).max() <= 1e-4


@pytest.mark.parametrize("prec", [eles.PREC_BF16X3, eles.PREC_TF32X2])
def test_mixed_batch_of_the_batched_configuration(prec):
    """Six items of the batched configuration (its three grids, LES = DNS / 4,
    and its three filter widths; one snapshot each) in one batch: the x-z
    stages share persistent launches per kernel class, every item matches
    the oracle, and the result equals the plans called one by one bit for bit."""
    dev = torch.device("cuda")
    items = [((128, 97, 128), 16), ((128, 97, 128), 48), ((192, 129, 192), 32), ((192, 129, 192), 16),
             ((256, 193, 256), 48), ((256, 193, 256), 32)]
    plans, us, ubs, taus, cases = [], [], [], [], []
    for k, (shape, w) in enumerate(items):
        dns, les = I.batch_grids(shape)
        delta = dns.Lx / w
        plan = eles.filter_setup(dns, les, delta, precision=prec)
        assert eles.plan_info(plan, 10) == 3
        u = I.channel_velocity(dns, 700 + k)
        plans.append(plan)
        cases.append((dns, les, delta, u))
        us.append(torch.from_numpy(u[None]).to(dev, torch.float32))
        ubs.append(torch.full((1, 3, les.ny, les.nz, les.nx), float("nan"), device=dev))
        taus.append(torch.full((1, 6, les.ny, les.nz, les.nx), float("nan"), device=dev))
    batch = eles.batch_create(plans, [1] * len(items))
    eles.batch_run(batch, us, ubs, taus)
    eles.batch_run(batch, us, ubs, taus)
    torch.cuda.synchronize()
    for k, (dns, les, delta, u) in enumerate(cases):
        assert eles.check_device_error(plans[k]) == 0
        ub_ref, tau_ref = O.subfilter_stress(dns, les, delta, u)
        assert np.abs(ubs[k][0].double().cpu().numpy() - ub_ref).max() <= 1e-4, k
        assert np.abs(taus[k][0].double().cpu().numpy() - tau_ref).max() <= 1e-4, k
        ub1 = torch.empty_like(ubs[k])
        t1 = torch.empty_like(taus[k])
        eles.subfilter_stress_batch(plans[k], us[k], ub1, t1)
        torch.cuda.synchronize()
        assert torch.equal(ub1, ubs[k]) and torch.equal(t1, taus[k]), k
