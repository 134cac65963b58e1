"""GPU parity of the tensor-core closure inference (through the C ABI).

The inference kernel runs the whole MLP on the tcgen05 tensor cores with the
BF16 working weights and activations split into two BF16 parts.  It is
compared with the FP64 reference forward pass (oracle/mlp.py) at the same
BF16-rounded weights and the same standardisation:

* outputs, in standardised units, on ragged point counts from one point to
  several passes of the persistent grid, and on sampled points of a
  1M-point call (the size the closure's inference is quoted on);
* the guard: the count of points with a standardised input beyond it, and
  the exact stress returned at exactly those points.

Tolerance (standardised units, relative to max |Y|): each activation keeps
16 significant bits (|a - a_hi - a_lo| <= 2^-16 |a|), sums of 128 products
accumulate in FP32 (<= 128 * 2^-24 relative to the sum of magnitudes), and
SiLU uses the fast exponential and division (a few ulp); four layers of
that stay below 1e-5 of the output scale for weights of unit gain, so the
bound 1e-4 leaves a factor of ten.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import __graft_entry__ as entry
from oracle import mlp as M
from paper_1902_02508_gb300 import eles

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    entry.build()


def bf16(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def make_closure(seed, guard=8.0):
    """A closure with He-uniform weights (gain ~1 per layer, so the SiLU sees
    both signs), uniform biases and fixed standardisation statistics."""
    rng = np.random.default_rng(seed)
    cl = eles.closure_create(batch=256, guard_sigma=guard, seed=seed)
    flat = []
    for fi, fo in eles.CLOSURE_LAYERS:
        b = np.sqrt(6.0 / fi)
        flat.append(rng.uniform(-b, b, size=(fo, fi)).ravel())
        flat.append(rng.uniform(-0.5, 0.5, size=fo))
    p = np.concatenate(flat).astype(np.float32)
    st = np.zeros(32)
    st[:10] = rng.normal(0.0, 0.3, 10)             # feature means
    st[10:20] = rng.uniform(0.5, 2.0, 10)          # feature sd
    st[20:26] = rng.normal(0.0, 0.5, 6)            # target means
    st[26:32] = rng.uniform(0.2, 1.5, 6)           # target sd
    eles.closure_set_params(cl, p, st)
    params = [(bf16(W), bf16(bb)) for W, bb in eles.closure_unpack(p)]
    return cl, params, st


def features(n, st, seed, spread=1.0):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 10)) * spread
    X[:, 9] = rng.uniform(-1.7, 1.7, n)            # the wall distance is bounded
    return (st[:10] + X * st[10:20]).astype(np.float32)


def reference(params, st, F):
    X = (F.astype(np.float64) - st[:10]) / st[10:20]
    Y, _ = M.forward(params, X)
    return X, Y


def standardised(out, st):
    return (out.double().cpu().numpy().T - st[20:26]) / st[26:32]


@pytest.mark.parametrize("n", [1, 127, 128, 129, 677, 2 * 152 * 128 * 2 + 300])
def test_matches_reference(n):
    cl, params, st = make_closure(11)
    F = features(n, st, 100 + n)
    _, Y = reference(params, st, F)
    out = torch.full((6, n), float("nan"), device="cuda")
    nf = eles.closure_infer(cl, torch.from_numpy(F).cuda(), out)
    assert nf == 0
    got = standardised(out, st)
    err = np.abs(got - Y).max()
    scale = max(1.0, np.abs(Y).max())
    print(f"n={n}: max |Y| {np.abs(Y).max():.3f}, max error {err:.3e} ({err / scale:.2e} of scale)")
    assert err <= TOL * scale
    assert eles.closure_check_device_error(cl) == 0


def test_million_points_sampled():
    n = 1 << 20
    cl, params, st = make_closure(5)
    F = features(n, st, 7)
    out = torch.empty((6, n), device="cuda")
    eles.closure_infer(cl, torch.from_numpy(F).cuda(), out, count=False)
    torch.cuda.synchronize()
    assert eles.closure_check_device_error(cl) == 0
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.choice(n, 4000, replace=False), np.arange(n - 200, n)])
    _, Y = reference(params, st, F[idx])
    got = standardised(out, st)[idx]
    assert np.isfinite(got).all()
    assert np.abs(got - Y).max() <= TOL * max(1.0, np.abs(Y).max())


def test_guard_and_fallback():
    n = 5000
    guard = 1.5
    cl, params, st = make_closure(9, guard=guard)
    F = features(n, st, 21, spread=0.8)
    X32 = (F - st[:10].astype(np.float32)) * (1.0 / st[10:20]).astype(np.float32)
    beyond = np.abs(X32) > guard
    near = np.abs(np.abs(X32) - guard) < 1e-5       # decisions too close to call across roundings
    fell_ref = beyond.any(axis=1)
    undecided = near.any(axis=1)
    assert 0 < fell_ref.sum() < n
    Fd = torch.from_numpy(F).cuda()
    exact = torch.from_numpy(np.random.default_rng(2).standard_normal((6, n)).astype(np.float32) + 50.0).cuda()
    out = torch.empty((6, n), device="cuda")
    nf = eles.closure_infer(cl, Fd, out, exact_tau=exact)
    fell = (out == exact).all(dim=0).cpu().numpy()
    assert nf == int(fell.sum())
    assert np.array_equal(fell[~undecided], fell_ref[~undecided])
    # the model outputs elsewhere, within the parity bound
    _, Y = reference(params, st, F)
    got = standardised(out, st)
    keep = ~fell
    assert np.abs(got[keep] - Y[keep]).max() <= TOL * max(1.0, np.abs(Y).max())
    # without an exact stress: the count is reported, every output is the model's
    out2 = torch.empty_like(out)
    nf2 = eles.closure_infer(cl, Fd, out2)
    assert nf2 == nf
    assert np.abs(standardised(out2, st) - Y).max() <= TOL * max(1.0, np.abs(Y).max())
