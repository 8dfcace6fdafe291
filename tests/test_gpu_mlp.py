"""GPU parity of the pruning network and the retrieval helpers against the
FP64 numpy oracle (oracle/mlp.py), through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp as omlp
from paper_2501_17779_gb300 import api, synth

from _mlp_bounds import forward_bounds, pair_grad_bounds

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _params(seed):
    rng = np.random.default_rng(seed)
    out = {}
    for name, shp in omlp.SHAPES:
        out[name] = (rng.normal(size=shp) * np.sqrt(2.0 / shp[1]) if len(shp) == 2
                     else rng.normal(size=shp) * 0.1)
    return omlp.pack(out).astype(np.float32)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def test_forward_matches_oracle():
    net = api.Mlp(seed=1)
    p = _params(2)
    net.set_params(p)
    np.testing.assert_array_equal(net.get_params(), p)
    X = np.random.default_rng(3).normal(size=(333, 64)).astype(np.float32)
    Y = net.forward(torch.from_numpy(X).to(DEV)).cpu().numpy()
    Yo, _, _ = omlp.forward(p, X)
    bound = forward_bounds(p, X)["bound_y"]
    err = np.abs(Y.astype(np.float64) - Yo)
    print(f"forward: max err/bound {np.max(err / bound):.3g}, relative norm {_rel(Y, Yo):.3g}")
    assert (err <= bound).all()


def test_pair_gradient_matches_oracle():
    """float32 accumulation against the float64 oracle on the same bfloat16
    weights, element by element within the probabilistic float32 bound of
    tests/_mlp_bounds.py (the relative norm per block is printed only)."""
    net = api.Mlp(seed=1)
    p = _params(4)
    net.set_params(p)
    rng = np.random.default_rng(5)
    rows, P = 517, 701
    X = rng.normal(size=(rows, 64)).astype(np.float32)
    pi = rng.integers(0, rows, P)
    pj = rng.integers(0, rows, P)
    d = rng.uniform(0.02, 0.5, P).astype(np.float32)
    loss, g = net.pair_grad(torch.from_numpy(X).to(DEV), torch.from_numpy(pi).to(DEV),
                            torch.from_numpy(pj).to(DEV), torch.from_numpy(d).to(DEV), grad=True)
    lo, go = omlp.pair_loss_grad(p, X, pi, pj, d)
    assert abs(loss.item() - lo) <= 1e-5 * lo
    g = g.cpu().numpy()
    bound = pair_grad_bounds(p, X, pi, pj, d)
    err = np.abs(g.astype(np.float64) - go)
    gu, gou, eu, bu = (omlp.unpack(a) for a in (g, go, err, bound))
    for name, _ in omlp.SHAPES:
        print(f"{name}: max err/bound {np.max(eu[name] / bu[name]):.3g}, "
              f"relative norm {_rel(gu[name], gou[name]):.3g}")
    assert (err <= bound).all()
    # the pair loss depends on y_i - y_j only: dL/db3 = 0 exactly in the oracle
    assert np.linalg.norm(gou["b3"]) < 1e-12 * np.linalg.norm(gou["W3"])


def test_adam_step_matches_oracle():
    net = api.Mlp(seed=1)
    p = _params(6)
    net.set_params(p)
    rng = np.random.default_rng(7)
    X = rng.normal(size=(64, 64)).astype(np.float32)
    pi, pj = rng.integers(0, 64, 128), rng.integers(0, 64, 128)
    d = rng.uniform(0.05, 0.3, 128).astype(np.float32)
    po, m, v = p.astype(np.float64), np.zeros(p.size), np.zeros(p.size)
    # a small rate keeps both sides on the same gradients step after step (the
    # float32 and float64 gradients then share their signs where they matter)
    lr = 1e-5
    for t in (1, 2, 3):
        net.pair_grad(torch.from_numpy(X).to(DEV), torch.from_numpy(pi).to(DEV),
                      torch.from_numpy(pj).to(DEV), torch.from_numpy(d).to(DEV))
        net.adam_step(lr)
        _, go = omlp.pair_loss_grad(po.astype(np.float32), X, pi, pj, d)
        po, m, v = omlp.adam_step(po, go, m, v, t, lr)
    got = net.get_params()
    # where the gradient is not tiny its sign is shared, so each step moves alike
    big = np.abs(go) > 1e-2 * np.abs(go).max()
    assert big.sum() > 1000
    assert np.abs(got - po)[big].max() < 3e-2 * lr
    assert np.abs(got - p).max() <= 3.0 * lr * 1.01


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_select_k_matches_oracle(dtype):
    rng = np.random.default_rng(8)
    keys = rng.integers(0, 50, (37, 1500)).astype(np.float64) * 0.01 - 0.1  # ties, negatives
    keys[3, 10] = np.nan
    for k in (1, 10, 200, 256):
        pos = api.select_k(torch.from_numpy(keys).to(DEV, dtype), k).cpu().numpy()
        ref = omlp.select_k(keys.astype(np.float32 if dtype == torch.float32 else np.float64), k)
        np.testing.assert_array_equal(pos, ref)


def test_embed_sqdist_and_stats():
    rng = np.random.default_rng(9)
    A = rng.normal(size=(70, 64)).astype(np.float32)
    B = rng.normal(size=(130, 64)).astype(np.float32)
    D = api.embed_sqdist(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)).cpu().numpy()
    ref = ((A[:, None, :].astype(np.float64) - B[None]) ** 2).sum(-1)
    assert np.abs(D - ref).max() < 1e-5 * ref.max()
    X = torch.from_numpy((rng.normal(size=(999, 5)) * [1, 2, 3, 4, 5] + 7).astype(np.float32)).to(DEV)
    mu, inv = api.column_stats(X)
    x = X.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(mu.cpu().numpy(), x.mean(0), rtol=1e-6)
    np.testing.assert_allclose(inv.cpu().numpy(), 1 / x.std(0), rtol=1e-6)
    Z = api.standardize_(X.clone(), mu, inv).cpu().numpy()
    np.testing.assert_allclose(Z, (x - x.mean(0)) / x.std(0), atol=1e-5)


def test_descriptors_match_oracle():
    g = synth.shape_gallery(12, 20, 128)
    pts = g.curves.reshape(-1)
    offs = np.arange(0, 20 * 128 + 1, 128, dtype=np.int64)
    zo, _ = oracle.resample(pts, offs, 128)
    z, st = api.resample_arclength(torch.from_numpy(pts).to(DEV), torch.from_numpy(offs).to(DEV), 128)
    F = 32
    d = api.fourier_descriptors(z.reshape(20, 128), F).cpu().numpy()
    do = omlp.fourier_descriptors(zo, F)
    mag, mago = np.exp(d.astype(np.float64)), np.exp(do)
    assert np.abs(mag - mago).max() < 1e-6 * mago.max()
    big = mago > 1e-6 * mago.max()
    assert np.abs(d - do)[big].max() < 1e-4


def test_training_lowers_the_loss():
    rng = np.random.default_rng(13)
    X = torch.from_numpy(rng.normal(size=(400, 64)).astype(np.float32)).to(DEV)
    # targets: a fixed random projection's distances (learnable)
    Pm = rng.normal(size=(64, 8)) / 8
    xp = X.cpu().numpy() @ Pm
    pi = rng.integers(0, 400, 2000)
    pj = rng.integers(0, 400, 2000)
    d = np.linalg.norm(xp[pi] - xp[pj], axis=1).astype(np.float32)
    net = api.Mlp(seed=3)
    args = [torch.from_numpy(a).to(DEV) for a in (pi, pj, d)]
    first = net.pair_grad(X, *args).item()
    for _ in range(150):
        net.pair_grad(X, *args)
        net.adam_step(1e-3)
    last = net.pair_grad(X, *args).item()
    assert last < 0.2 * first, (first, last)
