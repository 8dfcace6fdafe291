"""Pins of the pruning-network oracle (oracle/mlp.py): bfloat16 rounding and
Adam against torch's own routines, backpropagation against finite
differences, k-selection against a stable sort, descriptor invariances."""
import numpy as np
import pytest
import torch

from oracle import mlp
from paper_2501_17779_gb300 import synth


def _params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    p = mlp.unpack(np.zeros(mlp.N_PARAMS, np.float32))
    out = {}
    for name, shp in mlp.SHAPES:
        fan_in = shp[1] if len(shp) == 2 else 1
        out[name] = (rng.normal(size=shp) * scale * np.sqrt(2.0 / fan_in) if len(shp) == 2
                     else rng.normal(size=shp) * 0.1)
    assert set(out) == set(p)
    return mlp.pack(out).astype(np.float32)


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.normal(size=5000).astype(np.float32) * 10.0 ** rng.integers(-30, 30, 5000),
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.01171875, 65504.0, 3.4e38,
                                  1e-40, np.inf, -np.inf], np.float32)])
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(mlp.bf16_round(a), ref)


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(1)
    flat = _params(2)
    x = rng.normal(size=(12, 64))
    pi = rng.integers(0, 12, 9)
    pj = (pi + rng.integers(1, 12, 9)) % 12
    d = rng.uniform(0.02, 0.4, 9)
    loss, g = mlp.pair_loss_grad(flat, x, pi, pj, d, round_bf16=False)
    assert loss > 0
    base = flat.astype(np.float64)
    for idx in rng.choice(mlp.N_PARAMS, 40, replace=False):
        h = 1e-6
        e = np.zeros(mlp.N_PARAMS)
        e[idx] = h
        lp = _loss64(base + e, x, pi, pj, d)
        lm = _loss64(base - e, x, pi, pj, d)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(g[idx])), (idx, fd, g[idx])


def _loss64(flat64, x, pi, pj, d):
    """The loss with float64 parameters (no float32 round trip)."""
    w = mlp.unpack(flat64)
    xs = np.concatenate([x[pi], x[pj]])
    h1 = np.maximum(xs @ w["W1"].T + w["b1"], 0.0)
    h2 = np.maximum(h1 @ w["W2"].T + w["b2"], 0.0)
    y = h2 @ w["W3"].T + w["b3"]
    P = len(pi)
    r = np.sqrt(((y[:P] - y[P:]) ** 2).sum(axis=1) + mlp.LOSS_EPS)
    return float(np.mean((r - d) ** 2 / (d + mlp.LOSS_C) ** 2))


def test_adam_matches_torch():
    rng = np.random.default_rng(3)
    p0 = rng.normal(size=50)
    tp = torch.nn.Parameter(torch.from_numpy(p0.copy()))
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(mlp.ADAM_B1, mlp.ADAM_B2), eps=mlp.ADAM_EPS)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, 4):
        g = rng.normal(size=50)
        tp.grad = torch.from_numpy(g.copy())
        opt.step()
        p, m, v = mlp.adam_step(p, g, m, v, t, 1e-2)
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=0, atol=1e-14)


def test_select_k_ties_and_order():
    rng = np.random.default_rng(4)
    keys = rng.integers(0, 20, (7, 300)).astype(np.float64)
    k = 25
    got = mlp.select_k(keys, k)
    for r in range(7):
        ref = np.argsort(keys[r], kind="stable")[:k]
        np.testing.assert_array_equal(got[r], ref)


def test_descriptors_invariant_and_circle():
    z = np.stack([synth.uniform_arclength_nodes(synth.random_harmonics(np.random.default_rng(s), 8), 128)
                  for s in range(3)])
    d = mlp.fourier_descriptors(z)
    d2 = mlp.fourier_descriptors(np.exp(0.7j) * np.roll(z, 17, axis=1) + 0.3)
    np.testing.assert_allclose(d, d2, atol=1e-9)
    c = 0.2 * np.exp(2j * np.pi * np.arange(64) / 64)
    dc = mlp.fourier_descriptors(c[None])[0]
    assert abs(np.exp(dc[0]) - 0.2) < 1e-15 and (dc[1:] < np.log(1e-14)).all()
