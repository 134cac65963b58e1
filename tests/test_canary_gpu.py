"""Guard bands around every output buffer (the out-of-bounds check that
stands in for a memory sanitizer).

Each output is a view into the middle of a larger buffer whose margins hold a
canary bit pattern; after the call (and a synchronise) the margins must be
untouched and the view must hold no canary.  Covered: the stress on every
precision and on the warp-specialised tensor-core plan (single and batched),
ef_filter_fields, the differential filter and its inverse, the closure
features and tensor-core inference, the error measures, and the host-buffer
entry point.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import __graft_entry__ as entry
from paper_1902_02508_gb300 import eles
from paper_1902_02508_gb300 import inputs as I

pytestmark = pytest.mark.gpu

PAD = 256                  # elements on each side (a multiple of 16 bytes for every dtype)
CANARY = -1.2345e30


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    entry.build()


class Guarded:
    def __init__(self, shape, dtype, device="cuda", pin=False):
        n = int(np.prod(shape))
        self.n = n
        self.buf = torch.full((PAD + n + PAD,), CANARY, dtype=dtype, device=device)
        if pin:
            self.buf = self.buf.pin_memory()
        self.view = self.buf[PAD:PAD + n].view(*shape)

    def check(self, what):
        torch.cuda.synchronize()
        b = self.buf.cpu()
        assert torch.all(b[:PAD] == CANARY) and torch.all(b[PAD + self.n:] == CANARY), f"{what}: guard band written"
        assert not torch.any(b[PAD:PAD + self.n] == CANARY), f"{what}: output not fully written"


def grids(nx, ny, nz, Lx, Lz, nlx, nly, nlz):
    dns = I.dns_grid(nx, ny, nz, Lx, Lz)
    return dns, I.les_grid(dns, nlx, nly, nlz)


@pytest.mark.parametrize("prec", [eles.PREC_FP64, eles.PREC_FP32, eles.PREC_BF16X3, eles.PREC_TF32X2])
@pytest.mark.parametrize("geom", ["tiny", "tc2"])
def test_stress_outputs(prec, geom):
    if geom == "tiny" and prec in (eles.PREC_BF16X3, eles.PREC_TF32X2):
        pytest.skip("split precision needs a tensor-core geometry")
    if geom == "tiny":
        dns, les = grids(32, 33, 32, 2 * math.pi, math.pi, 8, 9, 8)
        delta = 2 * math.pi / 16
    else:
        dns, les = grids(192, 33, 256, 2 * math.pi, math.pi, 24, 17, 32)
        delta = 10 * math.pi / 192
    plan = eles.filter_setup(dns, les, delta, precision=prec)
    dt = plan.dtype
    ns = 2
    eles.plan_reserve(plan, ns)
    u = torch.from_numpy(np.stack([I.channel_velocity(dns, 1 + s) for s in range(ns)])).to("cuda", dt)
    lshape = (les.ny, les.nz, les.nx)
    ub = Guarded((ns, 3) + lshape, dt)
    tau = Guarded((ns, 6) + lshape, dt)
    pm = Guarded((ns, 3, dns.ny), torch.float64)
    eles.subfilter_stress_batch(plan, u, ub.view, tau.view, pm.view)
    ub.check("ubar (batch)"), tau.check("tau (batch)"), pm.check("plane means (batch)")
    ub1 = Guarded((3,) + lshape, dt)
    eles.filter_fields(plan, u[0].contiguous(), ub1.view)
    ub1.check("ubar (filter_fields)")
    assert eles.check_device_error(plan) == 0


@pytest.mark.parametrize("prec", [eles.PREC_FP64, eles.PREC_FP32])
def test_differential_outputs(prec):
    dns, les = grids(24, 33, 18, 4 * math.pi, 2 * math.pi, 8, 17, 6)
    plan = eles.filter_setup(dns, les, 0.8, kernel=eles.KERNEL_DIFFERENTIAL, precision=prec)
    dt = plan.dtype
    u = torch.from_numpy(I.channel_velocity(dns, 4)).to("cuda", dt)
    lshape = (les.ny, les.nz, les.nx)
    ub, tau, pm = Guarded((3,) + lshape, dt), Guarded((6,) + lshape, dt), Guarded((3, dns.ny), torch.float64)
    eles.subfilter_stress(plan, u, ub.view, tau.view, pm.view)
    ub.check("ubar"), tau.check("tau"), pm.check("plane means")
    ub1 = Guarded((3,) + lshape, dt)
    eles.filter_fields(plan, u, ub1.view)
    ub1.check("ubar (filter_fields)")
    if prec == eles.PREC_FP64:
        out = Guarded((3, dns.ny, dns.nz, dns.nx), torch.float64)
        eles.differential_unfilter(dns, 0.8, u, out.view)
        out.check("unfilter")


def test_closure_outputs():
    dns, les = grids(64, 33, 48, 2 * math.pi, math.pi, 16, 17, 12)
    plan = eles.filter_setup(dns, les, 2 * math.pi / 16, precision=eles.PREC_FP32)
    u = torch.from_numpy(I.channel_velocity(dns, 5)).to("cuda", torch.float32)
    lshape = (les.ny, les.nz, les.nx)
    ub = torch.empty((3,) + lshape, device="cuda")
    tau = torch.empty((6,) + lshape, device="cuda")
    eles.subfilter_stress(plan, u, ub, tau)
    n = les.nx * les.ny * les.nz
    feats = Guarded((n, 10), torch.float32)
    eles.closure_features(les, ub, feats.view)
    feats.check("features")
    feats_s = Guarded((n, 10), torch.float32)
    eles.closure_features_static(les, ub, feats_s.view)
    feats_s.check("features (static)")
    cl = eles.closure_create(batch=1024, seed=2)
    eles.closure_fit_norm(cl, feats.view, tau.reshape(6, n).contiguous())
    out = Guarded((6, n), torch.float32)
    eles.closure_infer(cl, feats.view, out.view, exact_tau=tau.reshape(6, n).contiguous())
    out.check("closure inference")


def test_stats_and_host_outputs():
    dns, les = grids(32, 33, 32, 2 * math.pi, math.pi, 8, 9, 8)
    st = eles.stats_create(dns, eles.PREC_FP32)
    u = torch.from_numpy(I.channel_velocity(dns, 6)).to("cuda", torch.float32)
    mean, rms, err = Guarded((3, dns.ny), torch.float64), Guarded((3, dns.ny), torch.float64), \
        Guarded((1,), torch.float64)
    eles.plane_stats(st, u, mean.view, rms.view)
    mean.check("plane mean"), rms.check("plane rms")
    eles.error_field(st, u, u * 1.01, err.view)
    err.check("Eq. 13")
    err2 = Guarded((1,), torch.float64)
    eles.error_profile(st, mean.view[0].contiguous(), rms.view[0].contiguous() + 1.0, err2.view)
    err2.check("Eq. 14/15")
    plan = eles.filter_setup(dns, les, 2 * math.pi / 16, precision=eles.PREC_FP32)
    io = eles.io_create(plan, 1)
    ns = 3
    hu = torch.from_numpy(np.stack([I.channel_velocity(dns, 7 + s) for s in range(ns)])).float().pin_memory()
    lshape = (les.ny, les.nz, les.nx)
    hb = Guarded((ns, 3) + lshape, torch.float32, device="cpu", pin=True)
    ht = Guarded((ns, 6) + lshape, torch.float32, device="cpu", pin=True)
    hp = Guarded((ns, 3, dns.ny), torch.float64, device="cpu", pin=True)
    stream = torch.cuda.current_stream()
    eles.subfilter_stress_host(io, hu, hb.view, ht.view, hp.view, stream=stream)
    stream.synchronize()
    hb.check("host ubar"), ht.check("host tau"), hp.check("host plane means")
    io.close()
