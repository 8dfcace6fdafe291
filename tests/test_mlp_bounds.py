"""The element-wise float32 bounds of tests/_mlp_bounds.py, checked on the
CPU: a float32 computation of the same network (numpy, float32 matrix
products) stays inside them, and they are far from vacuous (well below the
values they bound)."""
import numpy as np

from oracle import mlp as omlp

from _mlp_bounds import forward_bounds, pair_grad_bounds


def _params(seed):
    rng = np.random.default_rng(seed)
    out = {}
    for name, shp in omlp.SHAPES:
        out[name] = (rng.normal(size=shp) * np.sqrt(2.0 / shp[1]) if len(shp) == 2
                     else rng.normal(size=shp) * 0.1)
    return omlp.pack(out).astype(np.float32)


def _f32_net(flat, X, pi, pj, d):
    w = {n: (omlp.bf16_round(v) if n.startswith("W") else v).astype(np.float32)
         for n, v in omlp.unpack(flat).items()}
    xs = np.concatenate([X[pi], X[pj]]).astype(np.float32)
    P = len(pi)
    h1 = np.maximum(xs @ w["W1"].T + w["b1"], 0)
    h2 = np.maximum(h1 @ w["W2"].T + w["b2"], 0)
    y = h2 @ w["W3"].T + w["b3"]
    diff = y[:P] - y[P:]
    r = np.sqrt((diff ** 2).sum(1) + np.float32(omlp.LOSS_EPS))
    wgt = np.float32(1) / (d + np.float32(omlp.LOSS_C)) ** 2
    gd = (np.float32(2.0 / P) * wgt * (r - d) / r)[:, None] * diff
    gy = np.concatenate([gd, -gd])
    g = {"W3": gy.T @ h2, "b3": gy.sum(0)}
    gh2 = (gy @ w["W3"]) * (h2 > 0)
    g["W2"], g["b2"] = gh2.T @ h1, gh2.sum(0)
    gh1 = (gh2 @ w["W2"]) * (h1 > 0)
    g["W1"], g["b1"] = gh1.T @ xs, gh1.sum(0)
    return y, omlp.pack(g)


def test_float32_network_stays_inside_the_bounds():
    p = _params(4)
    rng = np.random.default_rng(5)
    rows, P = 517, 701
    X = rng.normal(size=(rows, 64)).astype(np.float32)
    pi, pj = rng.integers(0, rows, P), rng.integers(0, rows, P)
    d = rng.uniform(0.02, 0.5, P).astype(np.float32)
    y32, g32 = _f32_net(p, X, pi, pj, d)
    _, g64 = omlp.pair_loss_grad(p, X, pi, pj, d)
    bound = pair_grad_bounds(p, X, pi, pj, d)
    assert (np.abs(g32 - g64) <= bound).all()
    xs = np.concatenate([X[pi], X[pj]])
    fb = forward_bounds(p, xs)
    assert (np.abs(y32 - fb["y"]) <= fb["bound_y"]).all()
    # not vacuous: the bounds sit orders of magnitude below the values
    assert np.median(fb["bound_y"] / np.abs(fb["y"])) < 1e-2
    big = np.abs(g64) > 1e-3 * np.abs(g64).max()
    assert np.median(bound[big] / np.abs(g64[big])) < 1e-2
