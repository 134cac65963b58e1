"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances:
  * FP64 path: per component, max |GPU - oracle| <= 1e-12 max(|oracle|, 1)
    (the plain formula cancels bar(u1 u1) ~ 400 to T11 ~ 1..20, so the
    oracle itself carries ~1e-14 relative roundoff);
  * FP32 and split-precision paths (BF16X3, TF32X2): max |GPU - oracle|
    <= 1e-4 u_tau^2 for every T_ij component (velocities in units of u_tau)
    and <= 1e-4 for ~bar(u_i).
Operator weights are compared entry by entry with the oracle's FP64 operators.
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

TOL64 = 1e-12
TOL32 = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    entry.build()


def run_gpu(dns, les, delta, u, prec, ext=eles.EXT_EVEN_ODD, plane_mean=False):
    plan = eles.filter_setup(dns, les, delta, extension=ext, precision=prec)
    dev = torch.device("cuda")
    ud = torch.from_numpy(np.ascontiguousarray(u)).to(dev, plan.dtype)
    ub = torch.full((3, les.ny, les.nz, les.nx), float("nan"), device=dev, dtype=plan.dtype)
    tau = torch.full((6, les.ny, les.nz, les.nx), float("nan"), device=dev, dtype=plan.dtype)
    pm = torch.zeros((3, dns.ny), device=dev, dtype=torch.float64) if plane_mean else None
    eles.subfilter_stress(plan, ud, ub, tau, pm)
    torch.cuda.synchronize()
    assert eles.check_device_error(plan) == 0
    out = (ub.double().cpu().numpy(), tau.double().cpu().numpy())
    if plane_mean:
        out = out + (pm.cpu().numpy(),)
    return plan, out


def assert_close(got, ref, tol, what):
    for c in range(ref.shape[0]):
        err = np.abs(got[c] - ref[c]).max()
        scale = max(np.abs(ref[c]).max(), 1.0) if tol == TOL64 else 1.0
        assert err <= tol * scale, f"{what}[{c}]: max err {err:.3e} > {tol * scale:.3e}"


CASES = {
    # name: (nx, ny, nz, Lx, Lz, nlx, nly, nlz, delta)
    "tiny": (32, 33, 32, 2 * math.pi, math.pi, 8, 9, 8, 2 * math.pi / 16),
    # several 128-row tiles in z with a ragged tail (160 = 128 + 32)
    "tiles": (96, 65, 160, 2 * math.pi, math.pi, 24, 17, 40, 2 * math.pi / 24),
    # stride 6 in x and z (channel box 4 pi x 2 x 2 pi)
    "stride6": (96, 49, 96, 4 * math.pi, 2 * math.pi, 16, 13, 16, 4 * math.pi / 16),
    # non-integer DNS/LES ratios in x, y and z: generic banded path + interpolation
    "interp": (30, 25, 20, 2 * math.pi, math.pi, 9, 8, 6, 0.5),
    # stride 8 in x and z with a short x ring: the tensor-core x-contraction
    "tc": (128, 65, 128, 2 * math.pi, math.pi, 16, 17, 16, 12 * math.pi / 128),
    # stride 8, 8 x warps, odd first output of the x stream, 24 outputs per row
    # (not a multiple of the four B rotations): warp-specialised tensor-core kernel
    "tc2": (192, 33, 256, 2 * math.pi, math.pi, 24, 17, 32, 10 * math.pi / 192),
    # stride 8 with a wide x filter (2.5 Delta = 30 x cells): two output phases
    "wide": (128, 65, 128, 2 * math.pi, math.pi, 16, 17, 16, 24 * math.pi / 128),
    # stride 4 in x and z (the batched configuration's LES = DNS / 4)
    "s4": (128, 65, 128, 4 * math.pi, 2 * math.pi, 32, 17, 32, 4 * math.pi / 20),
    # stride 4 with a wide filter (2.5 Delta = 35 x cells): four output phases
    "s4w": (256, 49, 128, 4 * math.pi, 2 * math.pi, 64, 13, 32, 0.7),
}
SPLIT = (eles.PREC_BF16X3, eles.PREC_TF32X2)
TC_CASES = ("tc", "tc2", "wide", "s4", "s4w")


def case(name, seed=1000):
    nx, ny, nz, Lx, Lz, nlx, nly, nlz, delta = CASES[name]
    dns = I.dns_grid(nx, ny, nz, Lx, Lz)
    les = I.les_grid(dns, nlx, nly, nlz) if (ny - 1) % (nly - 1) == 0 else \
        I.Grid(nlx, nly, nlz, Lx, Lz, I.tanh_nodes(nly))
    return dns, les, delta, I.channel_velocity(dns, seed)


@pytest.mark.parametrize("name", sorted(CASES))
def test_weights_match_oracle(name):
    dns, les, delta, _ = case(name)
    plan = eles.filter_setup(dns, les, delta, precision=eles.PREC_FP64)
    assert np.abs(eles.plan_weights(plan, 0) - O.op_periodic(dns.nx, dns.Lx, les.nx, delta)).max() < 1e-14
    assert np.abs(eles.plan_weights(plan, 1) - O.op_periodic(dns.nz, dns.Lz, les.nz, delta)).max() < 1e-14
    assert np.abs(eles.plan_weights(plan, 2) - O.op_wall(dns.y, les.y, delta, +1)).max() < 1e-14
    assert np.abs(eles.plan_weights(plan, 3) - O.op_wall(dns.y, les.y, delta, -1)).max() < 1e-14


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("prec", [eles.PREC_FP64, eles.PREC_FP32, eles.PREC_BF16X3, eles.PREC_TF32X2])
def test_subfilter_stress_matches_oracle(name, prec):
    if prec in SPLIT and name not in TC_CASES:
        pytest.skip("split precision runs on tensor-core geometries only (refusal tested below)")
    dns, les, delta, u = case(name)
    ub_ref, tau_ref = O.subfilter_stress(dns, les, delta, u)
    plan, (ub, tau) = run_gpu(dns, les, delta, u, prec)
    tol = TOL64 if prec == eles.PREC_FP64 else TOL32
    assert_close(ub, ub_ref, tol, "ubar")
    assert_close(tau, tau_ref, tol, "tau")


@pytest.mark.parametrize("ext", [eles.EXT_ODD_EVEN, eles.EXT_NONE])
@pytest.mark.parametrize("prec", [eles.PREC_FP64, eles.PREC_FP32])
def test_other_wall_treatments(ext, prec):
    dns, les, delta, u = case("tiny", seed=7)
    ub_ref, tau_ref = O.subfilter_stress(dns, les, delta, u, ext=ext)
    _, (ub, tau) = run_gpu(dns, les, delta, u, prec, ext=ext)
    tol = TOL64 if prec == eles.PREC_FP64 else TOL32
    assert_close(ub, ub_ref, tol, "ubar")
    assert_close(tau, tau_ref, tol, "tau")


def test_channel_shape_re180_fp32_and_fp64():
    """192 x 129 x 192 -> 32 x 33 x 32, Delta = Lx / 32 (Re_tau ~ 180 shape)."""
    dns = I.dns_grid(192, 129, 192, 4 * math.pi, 2 * math.pi)
    les = I.les_grid(dns, 32, 33, 32)
    delta = dns.Lx / 32
    u = I.channel_velocity(dns, 1001)
    ub_ref, tau_ref = O.subfilter_stress(dns, les, delta, u)
    for prec, tol in ((eles.PREC_FP64, TOL64), (eles.PREC_FP32, TOL32)):
        _, (ub, tau) = run_gpu(dns, les, delta, u, prec)
        assert_close(ub, ub_ref, tol, "ubar")
        assert_close(tau, tau_ref, tol, "tau")


_BIG = {}


def big_field():
    if not _BIG:
        dns = I.dns_grid(512, 257, 384, 2 * math.pi, math.pi)
        _BIG["v"] = (dns, I.les_grid(dns, 64, 65, 48), I.channel_velocity(dns, 1002))
    return _BIG["v"]


@pytest.mark.parametrize("dfrac,prec", [(64, eles.PREC_FP32), (32, eles.PREC_FP32), (64, eles.PREC_BF16X3),
                                        (32, eles.PREC_BF16X3), (64, eles.PREC_TF32X2), (32, eles.PREC_TF32X2)])
def test_full_size_sampled_points(dfrac, prec):
    """512 x 257 x 384 -> 64 x 65 x 48 at full size, checked at seeded LES
    points (wall rows included) by the oracle's direct 3-D summation."""
    dns, les, u = big_field()
    delta = dns.Lx / dfrac
    plan, (ub, tau) = run_gpu(dns, les, delta, u, prec)
    if prec in SPLIT:
        assert eles.plan_info(plan, 10) == 3          # warp-specialised tensor-core x-z kernel
        assert eles.plan_info(plan, 15) == (1 if dfrac == 64 else 2)   # output phases
    rng = np.random.default_rng(3)
    pts = np.stack([rng.integers(0, les.nx, 12), rng.integers(0, les.ny, 12),
                    rng.integers(0, les.nz, 12)], axis=1)
    pts[:2, 1] = [0, les.ny - 1]
    ub3, tau3 = O.direct3d_points(dns, les, delta, u, pts)
    got_ub = ub[:, pts[:, 1], pts[:, 2], pts[:, 0]].T
    got_tau = tau[:, pts[:, 1], pts[:, 2], pts[:, 0]].T
    assert np.abs(got_ub - ub3).max() <= TOL32
    assert np.abs(got_tau - tau3).max() <= TOL32


def test_plane_mean_and_filter_fields():
    dns, les, delta, u = case("tiles", seed=5)
    plan, (ub, tau, pm) = run_gpu(dns, les, delta, u, eles.PREC_FP32, plane_mean=True)
    assert np.abs(pm - u.mean(axis=(2, 3))).max() < 1e-6
    dev = torch.device("cuda")
    ud = torch.from_numpy(u).to(dev, torch.float32)
    ub2 = torch.empty((3, les.ny, les.nz, les.nx), device=dev)
    eles.filter_fields(plan, ud, ub2)
    torch.cuda.synchronize()
    assert np.array_equal(ub2.double().cpu().numpy(), ub)


def test_invariants_on_gpu():
    """Eq. 8 parity at the walls, symmetric PSD T_ij, Galilean shift in x, z."""
    dns, les, delta, u = case("tiles", seed=9)
    _, (ub, tau) = run_gpu(dns, les, delta, u, eles.PREC_FP64)
    assert np.abs(ub[1, 0]).max() < 1e-14 and np.abs(ub[1, -1]).max() < 1e-14
    T = np.empty(tau.shape[1:] + (3, 3))
    for q, (i, j) in enumerate(O.PAIRS):
        T[..., i, j] = tau[q]
        T[..., j, i] = tau[q]
    assert np.linalg.eigvalsh(T.reshape(-1, 3, 3)).min() > -1e-11
    u2 = u.copy()
    u2[0] += 2.0
    u2[2] -= 0.5
    _, (ubs, taus) = run_gpu(dns, les, delta, u2, eles.PREC_FP32)
    _, (ub32, tau32) = run_gpu(dns, les, delta, u, eles.PREC_FP32)
    assert np.abs(taus - tau32).max() < 1e-5


def test_nan_input_sets_device_error():
    dns, les, delta, u = case("tiny")
    u = u.copy()
    u[0, 5, 3, 7] = np.nan
    plan = eles.filter_setup(dns, les, delta, precision=eles.PREC_FP32)
    dev = torch.device("cuda")
    ud = torch.from_numpy(u).to(dev, torch.float32)
    ub = torch.empty((3, les.ny, les.nz, les.nx), device=dev)
    tau = torch.empty((6, les.ny, les.nz, les.nx), device=dev)
    eles.subfilter_stress(plan, ud, ub, tau)
    assert eles.check_device_error(plan) == 4
    assert eles.check_device_error(plan) == 0      # the word is cleared by the read


@pytest.mark.parametrize("name", ["tiny", "tiles"])
def test_batch_equals_single_calls(name):
    """Three snapshots in one batched call (two groups: reserve 2) give the
    same bits as three single calls."""
    dns, les, delta, u0 = case(name, seed=31)
    us = np.stack([u0, I.shifted(u0, 3, 1), I.channel_velocity(dns, 32)])
    plan = eles.filter_setup(dns, les, delta, precision=eles.PREC_FP32)
    eles.plan_reserve(plan, 2)
    dev = torch.device("cuda")
    ud = torch.from_numpy(us).to(dev, torch.float32)
    ub = torch.empty((3, 3, les.ny, les.nz, les.nx), device=dev)
    tau = torch.empty((3, 6, les.ny, les.nz, les.nx), device=dev)
    pm = torch.empty((3, 3, dns.ny), device=dev, dtype=torch.float64)
    eles.subfilter_stress_batch(plan, ud, ub, tau, pm)
    for k in range(3):
        ub1 = torch.empty((3, les.ny, les.nz, les.nx), device=dev)
        t1 = torch.empty((6, les.ny, les.nz, les.nx), device=dev)
        pm1 = torch.empty((3, dns.ny), device=dev, dtype=torch.float64)
        eles.subfilter_stress(plan, ud[k].contiguous(), ub1, t1, pm1)
        torch.cuda.synchronize()
        assert torch.equal(ub1, ub[k]) and torch.equal(t1, tau[k]) and torch.equal(pm1, pm[k])
    _, tau_ref = O.subfilter_stress(dns, les, delta, us[2])
    assert np.abs(tau[2].double().cpu().numpy() - tau_ref).max() <= TOL32


def test_fused_path_is_used_for_channel_shapes():
    for (nx, ny, nz, Lx, Lz, nlx, nly, nlz, dfrac) in [(192, 129, 192, 4 * math.pi, 2 * math.pi, 32, 33, 32, 32),
                                                        (512, 257, 384, 2 * math.pi, math.pi, 64, 65, 48, 64),
                                                        (512, 257, 384, 2 * math.pi, math.pi, 64, 65, 48, 32)]:
        dns = I.dns_grid(nx, ny, nz, Lx, Lz)
        plan = eles.filter_setup(dns, I.les_grid(dns, nlx, nly, nlz), Lx / dfrac, precision=eles.PREC_FP32)
        assert eles.plan_info(plan, 11) == 1


def test_tensor_core_variant_selected():
    dns, les, delta, _ = case("tc")
    plan = eles.filter_setup(dns, les, delta, precision=eles.PREC_BF16X3)
    assert eles.plan_info(plan, 10) == 3 and eles.plan_info(plan, 11) == 1
    assert eles.plan_info(plan, 13) == 1                  # tensor-core y contraction
    plan32 = eles.filter_setup(dns, les, delta, precision=eles.PREC_FP32)
    assert eles.plan_info(plan32, 10) == 1 and eles.plan_info(plan32, 13) == 0
    with pytest.raises(eles.EFError):
        eles.plan_set_variant(plan32, 3 * 16 + 2)     # no tensor cores for an FP32 plan


@pytest.mark.parametrize("name,variant,prec", [("tc", 2, eles.PREC_BF16X3), ("tc2", 2, eles.PREC_BF16X3)] +
                         [(n, 3, pr) for n in TC_CASES for pr in SPLIT])
def test_tensor_core_variants_match_oracle(name, variant, prec):
    """Both tensor-core x-z kernels (slide and warp-specialised; one, two or
    four output phases; x stride 8 and 4), with and without plane means,
    against the oracle; the plane means against the FP64 mean of the field."""
    dns, les, delta, u = case(name, seed=31)
    ub_ref, tau_ref = O.subfilter_stress(dns, les, delta, u)
    plan = eles.filter_setup(dns, les, delta, precision=prec)
    eles.plan_set_variant(plan, variant * 16 + 2)
    assert eles.plan_info(plan, 10) == variant
    if variant == 3:
        assert eles.plan_info(plan, 15) == {"wide": 2, "s4": 2, "s4w": 4}.get(name, 1)
    dev = torch.device("cuda")
    ud = torch.from_numpy(u).to(dev, torch.float32)
    for with_mean in (False, True):
        ub = torch.full((3, les.ny, les.nz, les.nx), float("nan"), device=dev)
        tau = torch.full((6, les.ny, les.nz, les.nx), float("nan"), device=dev)
        pm = torch.zeros((3, dns.ny), device=dev, dtype=torch.float64) if with_mean else None
        eles.subfilter_stress(plan, ud, ub, tau, pm)
        torch.cuda.synchronize()
        assert eles.check_device_error(plan) == 0
        assert_close(ub.double().cpu().numpy(), ub_ref, TOL32, "ubar")
        assert_close(tau.double().cpu().numpy(), tau_ref, TOL32, "tau")
        if with_mean:
            ref = u.mean(axis=(2, 3))
            assert np.abs(pm.cpu().numpy() - ref).max() <= 1e-5


def test_repeat_calls_are_bitwise_stable():
    dns, les, delta, u = case("tiles", seed=2)
    plan = eles.filter_setup(dns, les, delta, precision=eles.PREC_FP32)
    dev = torch.device("cuda")
    ud = torch.from_numpy(u).to(dev, torch.float32)
    outs = []
    for _ in range(2):
        ub = torch.empty((3, les.ny, les.nz, les.nx), device=dev)
        tau = torch.empty((6, les.ny, les.nz, les.nx), device=dev)
        eles.subfilter_stress(plan, ud, ub, tau)
        outs.append(tau.cpu())
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("name,prec", [("tiny", eles.PREC_FP64), ("tiny", eles.PREC_FP32), ("tc", eles.PREC_FP64),
                                       ("tc", eles.PREC_FP32), ("tc", eles.PREC_BF16X3), ("tc", eles.PREC_TF32X2)])
def test_hat_quadrature_matches_oracle(name, prec):
    """EF_KERNEL_GAUSSIAN_HAT: the y operators built on the device equal the
    oracle's hat-quadrature operators, and the whole path matches the
    oracle evaluated with them."""
    dns, les, delta, u = case(name, seed=77)
    plan = eles.filter_setup(dns, les, delta, kernel=eles.KERNEL_GAUSSIAN_HAT, precision=prec)
    # 1e-13, not 1e-14: the weights are differences of erf values (device and
    # host erf differ in the last ulps) divided by the node gaps
    assert np.abs(eles.plan_weights(plan, 2) - O.op_wall(dns.y, les.y, delta, +1, quad=1)).max() < 1e-13
    assert np.abs(eles.plan_weights(plan, 3) - O.op_wall(dns.y, les.y, delta, -1, quad=1)).max() < 1e-13
    ub_ref, tau_ref = O.subfilter_stress(dns, les, delta, u, quad=1)
    dev = torch.device("cuda")
    ud = torch.from_numpy(u).to(dev, plan.dtype)
    ub = torch.empty((3, les.ny, les.nz, les.nx), device=dev, dtype=plan.dtype)
    tau = torch.empty((6, les.ny, les.nz, les.nx), device=dev, dtype=plan.dtype)
    eles.subfilter_stress(plan, ud, ub, tau)
    torch.cuda.synchronize()
    tol = TOL64 if prec == eles.PREC_FP64 else TOL32
    assert_close(ub.double().cpu().numpy(), ub_ref, tol, "ubar")
    assert_close(tau.double().cpu().numpy(), tau_ref, tol, "tau")
    # the trapezoid operator differs (the quadrature really changed)
    assert np.abs(eles.plan_weights(plan, 2) - O.op_wall(dns.y, les.y, delta, +1)).max() > 1e-8


@pytest.mark.parametrize("name", ["tiny", "tiles", "stride6", "interp"])
@pytest.mark.parametrize("prec", [eles.PREC_BF16X3, eles.PREC_TF32X2])
def test_split_precision_refused_off_tensor_cores(name, prec):
    """A split-precision plan on a geometry the tensor-core x-z kernels do not
    cover is refused (EF_ERR_UNSUPPORTED) rather than run on CUDA cores."""
    dns, les, delta, _ = case(name)
    with pytest.raises(eles.EFError) as e:
        eles.filter_setup(dns, les, delta, precision=prec)
    assert e.value.code == 7


@pytest.mark.parametrize("name", ["tc", "tc2"])
def test_cuda_core_y_after_tensor_core_xz(name):
    """A split-precision plan whose y tiling does not fit runs the CUDA-core y
    pass after the tensor-core x-z kernel; the same combination, selected with
    EF_VARIANT_CUDA_CORE_Y on grids where it would fit, meets the FP32 bar."""
    dns, les, delta, u = case(name, seed=21)
    ub_ref, tau_ref = O.subfilter_stress(dns, les, delta, u)
    plan = eles.filter_setup(dns, les, delta, precision=eles.PREC_BF16X3)
    xv = eles.plan_info(plan, 10)
    assert xv in (2, 3)
    eles.plan_set_variant(plan, xv * 16 + 2 | eles.VARIANT_CUDA_CORE_Y)
    assert eles.plan_info(plan, 13) == 0 and eles.plan_info(plan, 10) == xv
    dev = torch.device("cuda")
    ud = torch.from_numpy(u).to(dev, torch.float32)
    ub = torch.full((3, les.ny, les.nz, les.nx), float("nan"), device=dev)
    tau = torch.full((6, les.ny, les.nz, les.nx), float("nan"), device=dev)
    eles.subfilter_stress(plan, ud, ub, tau)
    torch.cuda.synchronize()
    assert eles.check_device_error(plan) == 0
    assert_close(ub.double().cpu().numpy(), ub_ref, TOL32, "ubar")
    assert_close(tau.double().cpu().numpy(), tau_ref, TOL32, "tau")
    eles.plan_set_variant(plan, xv * 16 + 2)      # back on the tensor-core y pass
    assert eles.plan_info(plan, 13) == 1


@pytest.mark.parametrize("dfrac", [64, 32])
@pytest.mark.parametrize("prec", [eles.PREC_BF16X3, eles.PREC_TF32X2])
def test_full_size_whole_grid_split_precision(prec, dfrac):
    """512 x 257 x 384 -> 64 x 65 x 48, Delta = Lx / 64 and Lx / 32, split
    precision on the tensor cores: every LES point of ubar and T against the
    oracle's separable FP64 evaluation (the bench's workloads and launch
    configuration)."""
    dns, les, u = big_field()
    delta = dns.Lx / dfrac
    plan, (ub, tau) = run_gpu(dns, les, delta, u, prec)
    assert eles.plan_info(plan, 10) == 3 and eles.plan_info(plan, 13) == 1
    ub_ref, tau_ref = O.subfilter_stress(dns, les, delta, u)
    assert_close(ub, ub_ref, TOL32, "ubar")
    assert_close(tau, tau_ref, TOL32, "tau")
