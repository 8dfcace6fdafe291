"""Element-wise error bounds of the pruning network computed in float32
against the float64 oracle (oracle/mlp.py) on the same bfloat16 weights.

To first order the float32 result differs from the exact one by a linear
combination sum_i c_i delta_i of the individual rounding errors, each
|delta_i| <= u |v_i| (v_i the rounded partial result).  The worst case, every
delta_i of the same sign, overstates real errors by orders of magnitude over
three layers and a backward pass.  These bounds use the probabilistic model of
rounding errors (Higham and Mary, "A New Approach to Probabilistic Rounding
Error Analysis", SIAM J. Sci. Comput. 2019): the delta_i independent with mean
zero, so that |sum_i c_i delta_i| <= lambda sqrt(sum_i c_i^2 u^2 v_i^2) with
probability at least 1 - 2 exp(-lambda^2 (1 - u)^2 / 2); lambda = 8 puts that
below 3e-14 per element.  The code carries the square-root term s (a standard
deviation proxy) through the computation and multiplies by lambda once:

  a K-term sum adds sqrt(K) u sum |a_k b_k| (every partial sum is at most
      sum |a_k b_k|); independent parts combine as sqrt(s_1^2 + s_2^2)
  a linear map W takes s to sqrt(W^2 s^2); ReLU is 1-Lipschitz
  the pair loss: the output difference carries the outputs' s, its norm r is
      1-Lipschitz in it, the coefficient (2/P)(r - d)/((d + c)^2 r) takes r's
      to first order
  ReLU masks: where a pre-activation lies within lambda s of 0 the float32
      mask may differ; that unit's whole unmasked gradient is then added to a
      deterministic part f, which the later stages carry with |W| (worst case)

The bound is lambda s + f.  u = 2^-23 covers round-to-nearest float32
arithmetic (2^-24) with a factor 2 to spare, and also tensor-core
accumulation, which need not round to nearest, and float32 activations
represented as a sum of bfloat16 pieces.
"""
from __future__ import annotations

import numpy as np

from oracle import mlp as omlp

U = 2.0 ** -23
LAMBDA = 8.0


def _lin(s, W):
    """s [rows, K] through x -> x W^T (W [out, K]), errors independent."""
    return np.sqrt((s ** 2) @ (W ** 2).T)


def _hyp(*a):
    return np.sqrt(sum(x ** 2 for x in a))


def _w(flat):
    p = omlp.unpack(np.asarray(flat, np.float32))
    return {n: np.asarray(omlp.bf16_round(v) if n.startswith("W") else v, np.float64)
            for n, v in p.items()}


def forward_bounds(flat, x, u: float = U):
    """Oracle activations, the proxies s of (z1, z2, y) and the bound of y."""
    w = _w(flat)
    x = np.asarray(x, np.float64)
    z1 = x @ w["W1"].T + w["b1"]
    h1 = np.maximum(z1, 0.0)
    s1 = np.sqrt(omlp.D_IN + 1) * u * (np.abs(x) @ np.abs(w["W1"]).T + np.abs(w["b1"]))
    z2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(z2, 0.0)
    s2 = _hyp(_lin(s1, w["W2"]),
              np.sqrt(omlp.D_H + 1) * u * (h1 @ np.abs(w["W2"]).T + np.abs(w["b2"])))
    y = h2 @ w["W3"].T + w["b3"]
    s3 = _hyp(_lin(s2, w["W3"]),
              np.sqrt(omlp.D_H + 1) * u * (h2 @ np.abs(w["W3"]).T + np.abs(w["b3"])))
    return dict(w=w, x=x, z1=z1, h1=h1, s1=s1, z2=z2, h2=h2, s2=s2, y=y, s3=s3,
                bound_y=LAMBDA * s3)


def pair_grad_bounds(flat, x, pi, pj, d, u: float = U) -> np.ndarray:
    """Flat bound (the oracle's parameter order) on |gradient_float32 -
    gradient_float64| of the pair loss, element by element."""
    x = np.asarray(x, np.float64)
    xs = np.concatenate([x[pi], x[pj]])
    P = len(pi)
    R = 2 * P
    rR = np.sqrt(R)
    f = forward_bounds(flat, xs, u)
    w = f["w"]
    y, s3 = f["y"], f["s3"]
    diff = y[:P] - y[P:]
    sdiff = _hyp(s3[:P], s3[P:])
    r = np.sqrt((diff ** 2).sum(axis=1) + omlp.LOSS_EPS)
    sr = _hyp(np.sqrt((sdiff ** 2).sum(axis=1)), np.sqrt(omlp.D_OUT + 3) * u * r)
    d = np.asarray(d, np.float64)
    wgt = 1.0 / (d + omlp.LOSS_C) ** 2
    e = r - d
    coef = (2.0 / P) * wgt * e / r
    scoef = _hyp((2.0 / P) * wgt * (1.0 / r + np.abs(e) / r ** 2) * sr, 3 * u * np.abs(coef))
    gd = coef[:, None] * diff
    sgd = _hyp(np.abs(coef)[:, None] * sdiff, scoef[:, None] * np.abs(diff))
    gy, sgy = np.concatenate([gd, -gd]), np.concatenate([sgd, sgd])
    h2, s2, h1, s1 = f["h2"], f["s2"], f["h1"], f["s1"]
    b = {}

    def wgrad(g, sg, fg, h, sh):
        # sum over rows of g h^T: upstream proxies in quadrature, the sum's
        # own roundings, and the deterministic part through |h|
        s = _hyp(np.sqrt((sg ** 2).T @ (h ** 2) + (g ** 2).T @ (sh ** 2)),
                 rR * u * (np.abs(g).T @ np.abs(h)))
        return LAMBDA * s + fg.T @ (np.abs(h) + LAMBDA * sh)

    def bgrad(g, sg, fg):
        return LAMBDA * _hyp(np.sqrt((sg ** 2).sum(0)), rR * u * np.abs(g).sum(0)) + fg.sum(0)

    fy = np.zeros_like(gy)
    b["W3"] = wgrad(gy, sgy, fy, h2, s2)
    b["b3"] = bgrad(gy, sgy, fy)
    W3a, W2a = np.abs(w["W3"]), np.abs(w["W2"])
    gh2u = gy @ w["W3"]
    sgh2u = _hyp(_lin(sgy, w["W3"].T), np.sqrt(omlp.D_OUT) * u * (np.abs(gy) @ W3a))
    m2, flip2 = f["z2"] > 0, np.abs(f["z2"]) <= LAMBDA * s2
    gh2 = gh2u * m2
    sgh2 = sgh2u * (m2 | flip2)
    fgh2 = np.abs(gh2u) * flip2
    b["W2"] = wgrad(gh2, sgh2, fgh2, h1, s1)
    b["b2"] = bgrad(gh2, sgh2, fgh2)
    gh1u = gh2 @ w["W2"]
    sgh1u = _hyp(_lin(sgh2, w["W2"].T), np.sqrt(omlp.D_H) * u * (np.abs(gh2) @ W2a))
    fgh1u = fgh2 @ W2a
    m1, flip1 = f["z1"] > 0, np.abs(f["z1"]) <= LAMBDA * s1
    gh1 = gh1u * m1
    sgh1 = sgh1u * (m1 | flip1)
    fgh1 = fgh1u * (m1 | flip1) + (np.abs(gh1u) + LAMBDA * sgh1u) * flip1
    b["W1"] = wgrad(gh1, sgh1, fgh1, xs, np.zeros_like(xs))
    b["b1"] = bgrad(gh1, sgh1, fgh1)
    return omlp.pack(b)
