"""GPU parity of the Sec. 4 error measures (ef_plane_stats, ef_error_field,
ef_error_profile) against the FP64 reference of oracle/metrics.py, on DNS
and LES shaped channel fields (odd and even y node counts), FP32 and FP64
inputs; and the a-priori use: the filtered LES field against the DNS field
sampled at the LES nodes.

Tolerances: the reductions run in FP64 on the same values, so they agree to
1e-12 relative; FP32 inputs are compared with the oracle on the same
FP32-rounded values.  Repeat calls agree bit for bit (fixed-order sums).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import __graft_entry__ as entry
from oracle import metrics as M
from paper_1902_02508_gb300 import eles
from paper_1902_02508_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    entry.build()


@pytest.mark.parametrize("shape", [(96, 65, 64), (64, 48, 40)])
@pytest.mark.parametrize("prec", [eles.PREC_FP64, eles.PREC_FP32])
def test_measures_match_reference(shape, prec):
    nx, ny, nz = shape
    g = I.dns_grid(nx, ny, nz, 2 * math.pi, math.pi)
    a = I.channel_velocity(g, 41)
    b = I.channel_velocity(g, 42)
    dt = torch.float64 if prec == eles.PREC_FP64 else torch.float32
    a = torch.from_numpy(a).to(dt)
    b = torch.from_numpy(b).to(dt)
    an, bn = a.double().numpy(), b.double().numpy()
    st = eles.stats_create(g, prec)
    dev = torch.device("cuda")
    ad, bd = a.to(dev), b.to(dev)
    mean = torch.empty((3, ny), device=dev, dtype=torch.float64)
    rms = torch.empty_like(mean)
    eles.plane_stats(st, ad, mean, rms)
    m_ref, r_ref = M.plane_stats(an)
    assert np.abs(mean.cpu().numpy() - m_ref).max() <= 1e-12 * np.abs(m_ref).max()
    assert np.abs(rms.cpu().numpy() - r_ref).max() <= 1e-10 * np.abs(r_ref).max()
    err = torch.empty(1, device=dev, dtype=torch.float64)
    for c in range(3):
        vals = []
        for _ in range(2):
            eles.error_field(st, ad, bd, err, component=c, utau_a=1.1, utau_b=0.9)
            vals.append(float(err.item()))
        assert vals[0] == vals[1]
        ref = M.error_field(an[c], bn[c], g.y, g.Lx, g.Lz, 1.1, 0.9)
        assert abs(vals[0] - ref) <= 1e-12 * ref
    mb = torch.empty_like(mean)
    rb = torch.empty_like(rms)
    eles.plane_stats(st, bd, mb, rb)
    eles.error_profile(st, mean[0], mb[0], err, 1.1, 0.9)
    ref = M.error_profile(m_ref[0], M.plane_stats(bn)[0][0], g.y, 1.1, 0.9)
    assert abs(float(err.item()) - ref) <= 1e-12 * ref
    eles.error_profile(st, rms[0], rb[0], err)
    ref = M.error_profile(r_ref[0], M.plane_stats(bn)[1][0], g.y)
    assert abs(float(err.item()) - ref) <= 1e-9 * ref
    st.close()


def test_a_priori_filtered_against_dns():
    """The filtered field at the LES nodes against the DNS field at the same
    nodes: Eq. 13 of u_1 is the relative energy the filter removes, positive
    and below one; the mean-profile error (Eq. 14) is far smaller, because
    the filter keeps functions of y up to the y operator's commutation."""
    dns = I.dns_grid(128, 65, 128, 2 * math.pi, math.pi)
    les = I.les_grid(dns, 16, 17, 16)
    u = I.channel_velocity(dns, 9)
    plan = eles.filter_setup(dns, les, 12 * math.pi / 128, precision=eles.PREC_FP64)
    dev = torch.device("cuda")
    ud = torch.from_numpy(u).to(dev, torch.float64)
    ub = torch.empty((3, les.ny, les.nz, les.nx), device=dev, dtype=torch.float64)
    tau = torch.empty((6, les.ny, les.nz, les.nx), device=dev, dtype=torch.float64)
    eles.subfilter_stress(plan, ud, ub, tau)
    ry, rz, rx = (dns.ny - 1) // (les.ny - 1), dns.nz // les.nz, dns.nx // les.nx
    us = ud[:, ::ry, ::rz, ::rx].contiguous()          # DNS at the LES nodes
    st = eles.stats_create(les, eles.PREC_FP64)
    err = torch.empty(1, device=dev, dtype=torch.float64)
    eles.error_field(st, ub, us, err, component=0)
    e13 = float(err.item())
    ref = M.error_field(ub[0].cpu().numpy(), us[0].cpu().numpy(), les.y, les.Lx, les.Lz)
    assert abs(e13 - ref) <= 1e-12 * ref and 0.0 < e13 < 1.0
    mean_b = torch.empty((3, les.ny), device=dev, dtype=torch.float64)
    rms_b = torch.empty_like(mean_b)
    mean_s, rms_s = torch.empty_like(mean_b), torch.empty_like(mean_b)
    eles.plane_stats(st, ub, mean_b, rms_b)
    eles.plane_stats(st, us, mean_s, rms_s)
    eles.error_profile(st, mean_b[0], mean_s[0], err)
    assert float(err.item()) < e13
