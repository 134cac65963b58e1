"""GPU parity of the differential filter (EF_KERNEL_DIFFERENTIAL, FP64).

The CUDA path (FFTs in x and z, a tridiagonal solve in y per mode, inverse
transforms at the LES nodes) is compared with the pinned FP64 reference
oracle/differential.py on the same seeded channel fields:
  * ubar_i, T_ij and the plane means on grids with factors 2 and 3, both wall
    extensions (Eq. 7, Eq. 9), several LES ratios, and the 192 x 129 x 192
    channel with the paper's filter parameter a = 0.1;
  * a batch of snapshots equals single calls bit for bit; ef_filter_fields
    equals the ubar of ef_subfilter_stress;
  * requests outside its domain are refused at setup.
Tolerance: both sides are FP64 with different summation orders (FFT versus
numpy's FFT, the same Thomas recurrence); 1e-12 of the largest value of each
component.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import __graft_entry__ as entry
from oracle import differential as D
from paper_1902_02508_gb300 import eles
from paper_1902_02508_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12
A_PAPER = 0.1                                    # Sec. 3: a = 0.1
DELTA_PAPER = A_PAPER * math.sqrt(40.0)          # the width it corresponds to (a^2 = Delta_f^2 / 40)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    entry.build()


def run(dns, les, delta, u, ext=eles.EXT_EVEN_ODD):
    plan = eles.filter_setup(dns, les, delta, kernel=eles.KERNEL_DIFFERENTIAL, extension=ext,
                             precision=eles.PREC_FP64)
    assert eles.plan_info(plan, 14) == 1
    dev = torch.device("cuda")
    ud = torch.from_numpy(np.ascontiguousarray(u)).to(dev, torch.float64)
    ub = torch.full((3, les.ny, les.nz, les.nx), float("nan"), device=dev, dtype=torch.float64)
    tau = torch.full((6, les.ny, les.nz, les.nx), float("nan"), device=dev, dtype=torch.float64)
    pm = torch.zeros((3, dns.ny), device=dev, dtype=torch.float64)
    eles.subfilter_stress(plan, ud, ub, tau, pm)
    torch.cuda.synchronize()
    assert eles.check_device_error(plan) == 0
    return plan, ub.cpu().numpy(), tau.cpu().numpy(), pm.cpu().numpy()


def close(got, ref, what):
    for c in range(ref.shape[0]):
        err = np.abs(got[c] - ref[c]).max()
        scale = max(np.abs(ref[c]).max(), 1e-300)
        assert err <= TOL * scale, f"{what}[{c}]: {err:.3e} > {TOL * scale:.3e}"


CASES = {
    # (nx, ny, nz, Lx, Lz, nlx, nly, nlz, delta_f)
    "small": (16, 17, 12, 2 * math.pi, math.pi, 8, 9, 6, 0.5),
    "radix3": (24, 33, 18, 4 * math.pi, 2 * math.pi, 8, 17, 6, 0.8),
    "ragged": (36, 21, 32, 2 * math.pi, math.pi, 12, 11, 16, DELTA_PAPER),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("ext", [eles.EXT_EVEN_ODD, eles.EXT_ODD_EVEN])
def test_matches_reference(name, ext):
    nx, ny, nz, Lx, Lz, nlx, nly, nlz, delta = CASES[name]
    dns = I.dns_grid(nx, ny, nz, Lx, Lz)
    les = I.les_grid(dns, nlx, nly, nlz)
    u = I.channel_velocity(dns, 77)
    _, ub, tau, pm = run(dns, les, delta, u, ext)
    ub_ref, tau_ref = D.subfilter_stress(dns, les, delta, u, ext=ext)
    close(ub, ub_ref, "ubar")
    close(tau, tau_ref, "tau")
    assert np.abs(pm - u.mean(axis=(2, 3))).max() <= 1e-12 * np.abs(u).max()


def test_channel_192_paper_filter():
    """The 192 x 129 x 192 channel (4 pi x 2 x 2 pi) -> 32 x 33 x 32 with a = 0.1."""
    dns = I.dns_grid(192, 129, 192, 4 * math.pi, 2 * math.pi)
    les = I.les_grid(dns, 32, 33, 32)
    u = I.channel_velocity(dns, 1000)
    _, ub, tau, pm = run(dns, les, DELTA_PAPER, u)
    ub_ref, tau_ref = D.subfilter_stress(dns, les, DELTA_PAPER, u)
    close(ub, ub_ref, "ubar")
    close(tau, tau_ref, "tau")
    T = np.empty(tau.shape[1:] + (3, 3))
    for q, (i, j) in enumerate(D.PAIRS):
        T[..., i, j] = tau[q]
        T[..., j, i] = tau[q]
    assert np.linalg.eigvalsh(T.reshape(-1, 3, 3)).min() >= -1e-10
    assert np.abs(ub[1, 0]).max() == 0.0 and np.abs(ub[1, -1]).max() == 0.0


TOL32 = 1e-4                     # u_tau^2, the bar of the FP32 and tensor-core paths


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("ext", [eles.EXT_EVEN_ODD, eles.EXT_ODD_EVEN])
def test_fp32_matches_reference(name, ext):
    """FP32 transforms of the fluctuations about the plane means, FP64 profile
    terms and recovery, against the FP64 reference."""
    nx, ny, nz, Lx, Lz, nlx, nly, nlz, delta = CASES[name]
    dns = I.dns_grid(nx, ny, nz, Lx, Lz)
    les = I.les_grid(dns, nlx, nly, nlz)
    u = I.channel_velocity(dns, 78)
    plan = eles.filter_setup(dns, les, delta, kernel=eles.KERNEL_DIFFERENTIAL, extension=ext,
                             precision=eles.PREC_FP32)
    dev = torch.device("cuda")
    ub = torch.empty((3, nly, nlz, nlx), device=dev)
    tau = torch.empty((6, nly, nlz, nlx), device=dev)
    pm = torch.zeros((3, ny), device=dev, dtype=torch.float64)
    uf = torch.from_numpy(u).to(dev, torch.float32)
    eles.subfilter_stress(plan, uf, ub, tau, pm)
    torch.cuda.synchronize()
    ub_ref, tau_ref = D.subfilter_stress(dns, les, delta, uf.double().cpu().numpy(), ext=ext)
    eu = np.abs(ub.double().cpu().numpy() - ub_ref).max(axis=(1, 2, 3))
    et = np.abs(tau.double().cpu().numpy() - tau_ref).max(axis=(1, 2, 3))
    print(f"{name} ext {ext}: max |ubar err| {eu.max():.2e}, max |T err| per component {et}")
    assert eu.max() <= TOL32 and et.max() <= TOL32
    assert np.abs(pm.cpu().numpy() - uf.double().cpu().numpy().mean(axis=(2, 3))).max() <= 1e-12 * np.abs(u).max()


def test_fp32_channel_192():
    dns = I.dns_grid(192, 129, 192, 4 * math.pi, 2 * math.pi)
    les = I.les_grid(dns, 32, 33, 32)
    u = I.channel_velocity(dns, 1000)
    plan = eles.filter_setup(dns, les, DELTA_PAPER, kernel=eles.KERNEL_DIFFERENTIAL, precision=eles.PREC_FP32)
    dev = torch.device("cuda")
    uf = torch.from_numpy(u).to(dev, torch.float32)
    ub = torch.empty((3, 33, 32, 32), device=dev)
    tau = torch.empty((6, 33, 32, 32), device=dev)
    eles.subfilter_stress(plan, uf, ub, tau)
    torch.cuda.synchronize()
    ub_ref, tau_ref = D.subfilter_stress(dns, les, DELTA_PAPER, uf.double().cpu().numpy())
    et = np.abs(tau.double().cpu().numpy() - tau_ref).max(axis=(1, 2, 3))
    print(f"192 channel FP32: max |T err| per component {et}")
    assert np.abs(ub.double().cpu().numpy() - ub_ref).max() <= TOL32 and et.max() <= TOL32


def test_batch_and_filter_fields():
    nx, ny, nz, Lx, Lz, nlx, nly, nlz, delta = CASES["radix3"]
    dns = I.dns_grid(nx, ny, nz, Lx, Lz)
    les = I.les_grid(dns, nlx, nly, nlz)
    us = np.stack([I.channel_velocity(dns, 5), I.channel_velocity(dns, 6)])
    plan = eles.filter_setup(dns, les, delta, kernel=eles.KERNEL_DIFFERENTIAL, precision=eles.PREC_FP64)
    dev = torch.device("cuda")
    ud = torch.from_numpy(us).to(dev)
    ub = torch.empty((2, 3, nly, nlz, nlx), device=dev, dtype=torch.float64)
    tau = torch.empty((2, 6, nly, nlz, nlx), device=dev, dtype=torch.float64)
    eles.subfilter_stress_batch(plan, ud, ub, tau)
    for s in range(2):
        ub1 = torch.empty((3, nly, nlz, nlx), device=dev, dtype=torch.float64)
        tau1 = torch.empty((6, nly, nlz, nlx), device=dev, dtype=torch.float64)
        eles.subfilter_stress(plan, ud[s].contiguous(), ub1, tau1)
        ubf = torch.empty_like(ub1)
        eles.filter_fields(plan, ud[s].contiguous(), ubf)
        torch.cuda.synchronize()
        assert torch.equal(ub1, ub[s]) and torch.equal(tau1, tau[s])
        assert torch.equal(ubf, ub1)


def test_setup_refusals():
    dns = I.dns_grid(16, 17, 12, 2 * math.pi, math.pi)
    les = I.les_grid(dns, 8, 9, 6)
    K = eles.KERNEL_DIFFERENTIAL
    with pytest.raises(eles.EFError) as e:
        eles.filter_setup(dns, les, 0.5, kernel=K, precision=eles.PREC_BF16X3)
    assert e.value.code == 7                                   # EF_ERR_UNSUPPORTED
    with pytest.raises(eles.EFError) as e:
        eles.filter_setup(dns, les, 0.5, kernel=K, extension=eles.EXT_NONE, precision=eles.PREC_FP64)
    assert e.value.code == 1                                   # EF_ERR_ARG
    d5 = I.dns_grid(20, 17, 12, 2 * math.pi, math.pi)             # 20 = 2^2 * 5
    with pytest.raises(eles.EFError) as e:
        eles.filter_setup(d5, I.les_grid(d5, 10, 9, 6), 0.5, kernel=K, precision=eles.PREC_FP64)
    assert e.value.code == 2                                   # EF_ERR_SHAPE
    off = I.Grid(8, 9, 6, dns.Lx, dns.Lz, I.tanh_nodes(9, 1.5))   # LES y nodes off the DNS nodes
    with pytest.raises(eles.EFError) as e:
        eles.filter_setup(dns, off, 0.5, kernel=K, precision=eles.PREC_FP64)
    assert e.value.code == 2


def test_unfilter_inverts_filter_and_matches_operator():
    """ef_differential_unfilter is (1 - a^2 lap): it undoes the filter on the
    DNS grid (the LES grid taken equal to it) and equals the reference
    operator on an arbitrary field."""
    dns = I.dns_grid(24, 33, 18, 2 * math.pi, math.pi)
    delta = 0.8
    dev = torch.device("cuda")
    u = I.channel_velocity(dns, 9)
    plan = eles.filter_setup(dns, dns, delta, kernel=eles.KERNEL_DIFFERENTIAL, precision=eles.PREC_FP64)
    ud = torch.from_numpy(u).to(dev)
    ub = torch.empty_like(ud)
    eles.filter_fields(plan, ud, ub)
    back = torch.empty_like(ud)
    eles.differential_unfilter(dns, delta, ub, back)
    torch.cuda.synchronize()
    assert np.abs(back.cpu().numpy() - u).max() <= 1e-11 * np.abs(u).max()
    v = np.random.default_rng(4).standard_normal(u.shape)
    v[1, 0] = 0.0
    v[1, -1] = 0.0
    out = torch.empty_like(ud)
    eles.differential_unfilter(dns, delta, torch.from_numpy(v).to(dev), out)
    a = D.filter_parameter(delta)
    p = D.parities(D.EXT_EVEN_ODD)
    ref = np.stack([D.apply_operator(v[c], dns.y, dns.Lx, dns.Lz, a, p[c]) for c in range(3)])
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
