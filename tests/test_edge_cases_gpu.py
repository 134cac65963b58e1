"""GPU edge cases of the filter and stress calls (through the C ABI):

  * an empty batch (no snapshot) is refused with EF_ERR_ARG and leaves the
    plan usable;
  * a field constant in each component (u1 = c1, u2 = 0, u3 = c3; the odd
    component zero as Eq. 7 requires): a normalised filter returns the
    constants and the stress vanishes (Eq. 6 with bar(c c) = c c), in every
    precision, the split forms included;
  * the degenerate filter: a width so small that the cut-off 2.5 Delta is
    below the grid spacing in every direction leaves one tap per row, so on
    an LES grid equal to the DNS grid the filter is the identity and T is
    zero (the FP32 and FP64 plans; the split forms need a stride of 4, 8 or
    16 and refuse it);
  * the same small filter on a coarser LES grid is plain sampling at the LES
    nodes (LES nodes that are DNS nodes).
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


def _run(plan, dns, les, u):
    dev = torch.device("cuda")
    ud = torch.from_numpy(np.ascontiguousarray(u)).to(dev, plan.dtype)
    ub = torch.full((3, les.ny, les.nz, les.nx), float("nan"), device=dev, dtype=plan.dtype)
    tau = torch.full((6, les.ny, les.nz, les.nx), float("nan"), device=dev, dtype=plan.dtype)
    eles.subfilter_stress(plan, ud, ub, tau)
    torch.cuda.synchronize()
    assert eles.check_device_error(plan) == 0
    return ub.double().cpu().numpy(), tau.double().cpu().numpy()


def test_empty_batch_is_refused_and_plan_stays_usable():
    dns = I.dns_grid(32, 33, 32, 2 * math.pi, math.pi)
    les = I.les_grid(dns, 8, 9, 8)
    delta = 2 * math.pi / 16
    plan = eles.filter_setup(dns, les, delta, precision=eles.PREC_FP64)
    dev = torch.device("cuda")
    u0 = torch.empty((0, 3, dns.ny, dns.nz, dns.nx), device=dev, dtype=torch.float64)
    b0 = torch.empty((0, 3, les.ny, les.nz, les.nx), device=dev, dtype=torch.float64)
    t0 = torch.empty((0, 6, les.ny, les.nz, les.nx), device=dev, dtype=torch.float64)
    with pytest.raises(eles.EFError) as e:
        eles.subfilter_stress_batch(plan, u0, b0, t0)
    assert e.value.code == 1                                   # EF_ERR_ARG
    u = I.channel_velocity(dns, 3)
    ub, tau = _run(plan, dns, les, u)
    ub_ref, tau_ref = O.subfilter_stress(dns, les, delta, u)
    assert np.abs(tau - tau_ref).max() <= 1e-12 * max(np.abs(tau_ref).max(), 1.0)
    assert np.abs(ub - ub_ref).max() <= 1e-12 * max(np.abs(ub_ref).max(), 1.0)


# (name, nx, ny, nz, Lx, Lz, nlx, nly, nlz, delta, precisions)
CONST_CASES = [
    ("tiny", 32, 33, 32, 2 * math.pi, math.pi, 8, 9, 8, 2 * math.pi / 16, (eles.PREC_FP64, eles.PREC_FP32)),
    ("tc", 128, 65, 128, 2 * math.pi, math.pi, 16, 17, 16, 12 * math.pi / 128,
     (eles.PREC_FP64, eles.PREC_FP32, eles.PREC_BF16X3, eles.PREC_TF32X2)),
]


@pytest.mark.parametrize("case", CONST_CASES, ids=[c[0] for c in CONST_CASES])
def test_constant_field_gives_constants_and_zero_stress(case):
    _, nx, ny, nz, Lx, Lz, nlx, nly, nlz, delta, precs = case
    dns = I.dns_grid(nx, ny, nz, Lx, Lz)
    les = I.les_grid(dns, nlx, nly, nlz)
    c1, c3 = 17.25, -3.5
    u = np.zeros((3, ny, nz, nx))
    u[0] = c1
    u[2] = c3
    for prec in precs:
        plan = eles.filter_setup(dns, les, delta, precision=prec)
        ub, tau = _run(plan, dns, les, u)
        # FP64: the plain formula cancels c^2 ~ 300 to zero; the reduced
        # precisions contract zero fluctuations about U = c
        tol_u, tol_t = (1e-12 * c1, 1e-12 * c1 * c1) if prec == eles.PREC_FP64 else (1e-5, 1e-6)
        assert np.abs(ub[0] - c1).max() <= tol_u
        assert np.abs(ub[1]).max() <= tol_u
        assert np.abs(ub[2] - c3).max() <= tol_u
        assert np.abs(tau).max() <= tol_t, (prec, np.abs(tau).max())


def _tiny_delta_grids(nlx, nly, nlz):
    dns = I.dns_grid(64, 65, 48, 2 * math.pi, math.pi)
    les = I.les_grid(dns, nlx, nly, nlz)
    hy = float(np.diff(dns.y).min())
    delta = 0.3 * min(dns.Lx / dns.nx, dns.Lz / dns.nz, hy)   # 2.5 delta below every spacing
    return dns, les, delta


@pytest.mark.parametrize("prec", [eles.PREC_FP64, eles.PREC_FP32])
def test_degenerate_filter_is_the_identity(prec):
    dns, les, delta = _tiny_delta_grids(64, 65, 48)
    u = I.channel_velocity(dns, 11)
    plan = eles.filter_setup(dns, les, delta, precision=prec)
    ub, tau = _run(plan, dns, les, u)
    tol_u, tol_t = (1e-13, 1e-12) if prec == eles.PREC_FP64 else (1e-5, 1e-5)
    assert np.abs(ub - u).max() <= tol_u * max(np.abs(u).max(), 1.0)
    assert np.abs(tau).max() <= tol_t
    ub_ref, tau_ref = O.subfilter_stress(dns, les, delta, u)
    assert np.abs(ub_ref - u).max() <= 1e-13 * np.abs(u).max()     # the oracle agrees: identity


@pytest.mark.parametrize("prec", [eles.PREC_BF16X3, eles.PREC_TF32X2])
def test_degenerate_filter_refused_by_split_forms(prec):
    dns, les, delta = _tiny_delta_grids(64, 65, 48)
    with pytest.raises(eles.EFError) as e:
        eles.filter_setup(dns, les, delta, precision=prec)
    assert e.value.code == 7                                   # EF_ERR_UNSUPPORTED


@pytest.mark.parametrize("prec", [eles.PREC_FP64, eles.PREC_FP32])
def test_degenerate_filter_on_coarser_les_is_sampling(prec):
    dns, les, delta = _tiny_delta_grids(16, 17, 12)
    u = I.channel_velocity(dns, 12)
    plan = eles.filter_setup(dns, les, delta, precision=prec)
    ub, tau = _run(plan, dns, les, u)
    sy = (dns.ny - 1) // (les.ny - 1)
    sampled = u[:, ::sy, :: dns.nz // les.nz, :: dns.nx // les.nx]
    tol = 1e-13 if prec == eles.PREC_FP64 else 1e-5
    assert np.abs(ub - sampled).max() <= tol * max(np.abs(u).max(), 1.0)
    assert np.abs(tau).max() <= (1e-12 if prec == eles.PREC_FP64 else 1e-5)
