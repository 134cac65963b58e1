"""GPU tests of the learned closure (through the C ABI).

* features against the FP64 reference (oracle/mlp.py);
* one forward + backward pass against the FP64 reference gradients at the
  same (BF16-rounded) weights and standardisation, per layer;
* training lowers the loss; resuming from a checkpoint reproduces an
  uninterrupted run bit for bit;
* the gain: on a held-out snapshot the trained network's error against the
  exact T_ij is well below that of the model-free LES (T = 0) and below that
  of the gradient model (oracle/mlp.gradient_model), and the
  guarded inference falls back to the exact stress where asked.
"""
import math
import os
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import __graft_entry__ as entry
from oracle import mlp as M
from oracle import oracle as O
from paper_1902_02508_gb300 import eles
from paper_1902_02508_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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


_DATA = {}


def dataset(nsnap=5):
    """Exact (ubar, tau, features) of channel snapshots: DNS 128 x 65 x 128 in
    4 pi x 2 x 2 pi -> LES 32 x 33 x 32, Delta = Lx / 32."""
    if "v" not in _DATA:
        dns = I.dns_grid(128, 65, 128, 4 * math.pi, 2 * math.pi)
        les = I.les_grid(dns, 32, 33, 32)
        delta = dns.Lx / 32
        plan = eles.filter_setup(dns, les, delta, precision=eles.PREC_FP32)
        dev = torch.device("cuda")
        ubs, taus, feats = [], [], []
        n = les.nx * les.ny * les.nz
        for s in range(nsnap):
            u = torch.from_numpy(I.channel_velocity(dns, 2000 + s)).to(dev, torch.float32)
            ub = torch.empty((3, les.ny, les.nz, les.nx), device=dev)
            tau = torch.empty((6, les.ny, les.nz, les.nx), device=dev)
            eles.subfilter_stress(plan, u, ub, tau)
            f = torch.empty((n, 10), device=dev)
            eles.closure_features(les, ub, f)
            ubs.append(ub), taus.append(tau.reshape(6, n)), feats.append(f)
        torch.cuda.synchronize()
        _DATA["v"] = (dns, les, delta, ubs, taus, feats)
    return _DATA["v"]


def test_features_match_reference():
    dns, les, delta, ubs, taus, feats = dataset()
    ref = M.features(ubs[0].double().cpu().numpy(), les)
    got = feats[0].double().cpu().numpy()
    scale = np.abs(ref).max(axis=0)
    assert np.all(np.abs(got - ref).max(axis=0) <= 2e-5 * np.maximum(scale, 1.0))


def test_gradients_match_reference():
    dns, les, delta, ubs, taus, feats = dataset()
    cl = eles.closure_create(batch=512, seed=7)
    f, t = feats[0][:512].contiguous(), taus[0][:, :512].contiguous()
    eles.closure_fit_norm(cl, f, t)
    g, loss = eles.closure_gradients(cl, f, t)
    p, st = eles.closure_get_params(cl)
    params = [(bf16(W), bf16(b)) for W, b in eles.closure_unpack(p)]
    X = (f.double().cpu().numpy() - st[:10]) / st[10:20]
    T = ((t.double().cpu().numpy().T) - st[20:26]) / st[26:32]
    X = X.astype(np.float32).astype(np.float64)
    T = T.astype(np.float32).astype(np.float64)
    Y, cache = M.forward(params, X)
    ref = M.backward(params, cache, Y, T)
    assert abs(loss - M.mse(Y, T)) <= 1e-4 * M.mse(Y, T)
    gl = eles.closure_unpack(g)
    for l, ((gW, gb), (rW, rb)) in enumerate(zip(gl, ref)):
        assert np.abs(gW - rW).max() <= 2e-3 * np.abs(rW).max(), f"layer {l} W"
        assert np.abs(gb - rb).max() <= 2e-3 * np.abs(rb).max(), f"layer {l} b"


def _concat(xs, axis):
    return torch.cat(xs, dim=axis).contiguous()


def test_training_gain_and_fallback():
    dns, les, delta, ubs, taus, feats = dataset()
    ftr, ttr = _concat(feats[:4], 0), _concat(taus[:4], 1)
    cl = eles.closure_create(batch=4096, lr=2e-3, seed=3)
    l0 = eles.closure_train(cl, ftr, ttr, epochs=1)
    l1 = eles.closure_train(cl, ftr, ttr, epochs=40)
    assert l1 < 0.5 * l0
    # held-out snapshot
    n = feats[4].shape[0]
    out = torch.empty((6, n), device="cuda")
    eles.closure_infer(cl, feats[4], out)
    exact = taus[4].double().cpu().numpy()
    pred = out.double().cpu().numpy()
    err_mlp = np.linalg.norm(pred - exact) / np.linalg.norm(exact)
    gm = M.gradient_model(ubs[4].double().cpu().numpy(), les, delta).reshape(6, -1)
    err_grad = np.linalg.norm(gm - exact) / np.linalg.norm(exact)
    per = [np.linalg.norm(pred[q] - exact[q]) / np.linalg.norm(exact[q]) for q in range(6)]
    per_g = [np.linalg.norm(gm[q] - exact[q]) / np.linalg.norm(exact[q]) for q in range(6)]
    print(f"relative error: MLP {err_mlp:.3f}, gradient model {err_grad:.3f}, no model 1.000; per component "
          f"MLP {np.round(per, 3)}, gradient model {np.round(per_g, 3)}")
    # the gain over the model-free LES (T = 0, error 1) and over the gradient model
    assert err_mlp < 0.5
    assert err_mlp < err_grad
    assert max(per) < 1.0
    # guard: a tiny threshold sends (almost) every point to the exact stress
    cl2 = eles.closure_create(batch=4096, lr=2e-3, seed=3, guard_sigma=1e-3)
    p, st = eles.closure_get_params(cl)
    eles.closure_set_params(cl2, p, st)
    out2 = torch.empty_like(out)
    nfall = eles.closure_infer(cl2, feats[4], out2, exact_tau=taus[4])
    assert nfall >= n - 100
    fell = (out2 == taus[4]).all(dim=0)
    assert int(fell.sum()) == nfall


def test_checkpoint_resume_is_bitwise():
    dns, les, delta, ubs, taus, feats = dataset()
    ftr, ttr = _concat(feats[:2], 0), _concat(taus[:2], 1)
    a = eles.closure_create(batch=2048, seed=11)
    eles.closure_train(a, ftr, ttr, epochs=2)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        eles.closure_save(a, path)
        eles.closure_train(a, ftr, ttr, epochs=2)
        pa, _ = eles.closure_get_params(a)
        b = eles.closure_create(batch=2048, seed=11)
        eles.closure_load(b, path)
        eles.closure_train(b, ftr, ttr, epochs=2)
        pb, _ = eles.closure_get_params(b)
        assert np.array_equal(pa, pb)
        # a corrupted file is refused
        raw = bytearray(open(path, "rb").read())
        raw[100] ^= 0xFF
        open(path, "wb").write(bytes(raw))
        with pytest.raises(eles.EFError):
            eles.closure_load(b, path)


def test_adam_steps_match_reference():
    """Two ef_closure_train steps on one mini-batch against the FP64 Adam of the
    reference (oracle/mlp.adam_step) fed with the library's own gradients at the
    same weights (ef_closure_gradients, checked against the reference gradients
    above): every parameter whose gradient is not lost in FP32 rounding within
    1e-3 of the step size lr; the rest (|g| below 1e-5 of its layer's largest,
    where Adam's sign-like first step is undetermined) within one step."""
    dns, les, delta, ubs, taus, feats = dataset()
    n = 256
    lr = 1e-3
    cl = eles.closure_create(batch=n, lr=lr, seed=5)
    f, t = feats[1][:n].contiguous(), taus[1][:, :n].contiguous()
    eles.closure_fit_norm(cl, f, t)
    p0, _ = eles.closure_get_params(cl)
    ref = [(W.astype(np.float64), b.astype(np.float64)) for W, b in eles.closure_unpack(p0)]
    state = M.adam_init(ref)
    small_total = 0
    for step in range(2):
        g, _ = eles.closure_gradients(cl, f, t)     # at the current weights
        grads = [(gW.astype(np.float64), gb.astype(np.float64)) for gW, gb in eles.closure_unpack(g)]
        eles.closure_train(cl, f, t, epochs=1)      # n == batch: one Adam step per epoch
        ref = M.adam_step(ref, grads, state, lr)
        got = eles.closure_unpack(eles.closure_get_params(cl)[0])
        for l, (gl, rl, gr) in enumerate(zip(got, ref, grads)):
            gmax = max(np.abs(gr[0]).max(), np.abs(gr[1]).max())
            for k in range(2):
                d = np.abs(gl[k] - rl[k])
                small = np.abs(gr[k]) < 1e-5 * gmax
                small_total += int(small.sum())
                assert d[~small].max(initial=0.0) <= 1e-3 * lr, f"step {step + 1} layer {l} part {k}"
                assert d[small].max(initial=0.0) <= 2.1 * lr, f"step {step + 1} layer {l} part {k}"
    assert small_total < 0.05 * 2 * p0.size       # the tight bound covers almost every parameter
    # the steps moved the weights by about lr each (the comparison is not vacuous)
    moved = np.abs(eles.closure_get_params(cl)[0] - p0)
    assert np.median(moved) > 0.5 * lr


def test_exact_fallback_through_a_plan():
    """ef_closure_infer_exact: at the guarded points the output is the exact
    stress, computed from the DNS snapshot through the plan, and equals the
    oracle's direct 3-D summation at that LES point within 1e-4 u_tau^2; at
    the other points it is the network's output, bit for bit."""
    dns, les, delta, ubs, taus, feats = dataset()
    ftr, ttr = _concat(feats[:2], 0), _concat(taus[:2], 1)
    cl = eles.closure_create(batch=4096, lr=2e-3, seed=3, guard_sigma=3.0)
    eles.closure_train(cl, ftr, ttr, epochs=3)
    plan = eles.filter_setup(dns, les, delta, precision=eles.PREC_FP32)
    u = torch.from_numpy(I.channel_velocity(dns, 2004)).to("cuda", torch.float32)   # snapshot 4 of the dataset
    n = feats[4].shape[0]
    plain = torch.empty((6, n), device="cuda")
    nplain = eles.closure_infer(cl, feats[4], plain)
    out = torch.full((6, n), float("nan"), device="cuda")
    nfall = eles.closure_infer_exact(cl, feats[4], out, plan, u)
    assert nfall == nplain and 0 < nfall < n // 2
    differs = (out != plain).any(dim=0).cpu().numpy()
    idx = np.nonzero(differs)[0]
    assert len(idx) == nfall                       # exactly the guarded points changed
    sample = idx[np.linspace(0, len(idx) - 1, min(24, len(idx))).astype(int)]
    X, Z, J = sample % les.nx, (sample // les.nx) % les.nz, sample // (les.nx * les.nz)
    pts = np.stack([X, J, Z], axis=1)
    _, tau3 = O.direct3d_points(dns, les, delta, I.channel_velocity(dns, 2004), pts)
    got = out[:, sample].double().cpu().numpy().T
    assert np.abs(got - tau3).max() <= 1e-4
