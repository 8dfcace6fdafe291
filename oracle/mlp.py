"""FP64 numpy oracle of the candidate-pruning network and of k-NN selection.

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's CPU
baseline leg are the only callers.  It shares no code with the CUDA library.

The network is not part of the paper (Sec. 3 computes elastic distances; the
pruning of k-NN candidates by a learned embedding is this library's
addition).  What it computes, written out plainly:

  weights      W1 [256, 64], W2 [256, 256], W3 [64, 256] used in bfloat16
               (round to nearest even of the float32 master values), biases
               b1, b2, b3 in float32; all arithmetic here in float64.
  forward      h1 = relu(x W1^T + b1), h2 = relu(h1 W2^T + b2), y = h2 W3^T + b3
  pair loss    L = (1/P) sum_p (r_p - d_p)^2 / (d_p + c)^2,
               r_p = sqrt(|y_i - y_j|^2 + eps), eps = 1e-12, c = 0.05
               (relative error of the embedding distance against the elastic
               distance d_p, so that near neighbours weigh as much as far ones)
  backward     the chain rule through the three layers (ReLU derivative 0 at
               0); gradients of the bfloat16 weights are taken as gradients of
               the float32 masters (straight-through rounding)
  Adam         m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
               p -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps_a)
               with b1 = 0.9, b2 = 0.999, eps_a = 1e-8
"""
from __future__ import annotations

import numpy as np

D_IN, D_H, D_OUT = 64, 256, 64
SHAPES = (("W1", (D_H, D_IN)), ("b1", (D_H,)), ("W2", (D_H, D_H)), ("b2", (D_H,)),
          ("W3", (D_OUT, D_H)), ("b3", (D_OUT,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)
LOSS_EPS = 1e-12
LOSS_C = 0.05
ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def bf16_round(a) -> np.ndarray:
    """float32 -> bfloat16 (round to nearest, ties to even) -> float32."""
    a = np.ascontiguousarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    nan = np.isnan(a)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).copy()
    out[nan] = np.nan
    return out


def unpack(flat) -> dict:
    """The flat float32 parameter vector (order W1, b1, W2, b2, W3, b3, each
    row-major) as named arrays."""
    flat = np.asarray(flat)
    assert flat.size == N_PARAMS
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = flat[o:o + n].reshape(shp)
        o += n
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in SHAPES])


def _weights(flat, round_bf16: bool):
    p = unpack(np.asarray(flat, np.float32))
    w = {}
    for name, _ in SHAPES:
        v = p[name]
        if name.startswith("W") and round_bf16:
            v = bf16_round(v)
        w[name] = np.asarray(v, np.float64)
    return w


def forward(flat, x, round_bf16: bool = True):
    """y for inputs x [B, 64]; also returns the hidden activations."""
    w = _weights(flat, round_bf16)
    x = np.asarray(x, np.float64)
    h1 = np.maximum(x @ w["W1"].T + w["b1"], 0.0)
    h2 = np.maximum(h1 @ w["W2"].T + w["b2"], 0.0)
    y = h2 @ w["W3"].T + w["b3"]
    return y, h1, h2


def pair_loss_grad(flat, x, pi, pj, d, round_bf16: bool = True):
    """Loss and gradient (flat, float64) of the pair loss over pairs
    (x[pi[p]], x[pj[p]]) with targets d[p]."""
    w = _weights(flat, round_bf16)
    x = np.asarray(x, np.float64)
    xs = np.concatenate([x[pi], x[pj]])
    P = len(pi)
    y, h1, h2 = forward(flat, xs, round_bf16)
    diff = y[:P] - y[P:]
    r = np.sqrt((diff ** 2).sum(axis=1) + LOSS_EPS)
    d = np.asarray(d, np.float64)
    wgt = 1.0 / (d + LOSS_C) ** 2
    e = r - d
    loss = float(np.mean(wgt * e * e))
    gdiff = (2.0 / P) * (wgt * e / r)[:, None] * diff
    gy = np.concatenate([gdiff, -gdiff])
    g = {}
    g["W3"] = gy.T @ h2
    g["b3"] = gy.sum(axis=0)
    gh2 = (gy @ w["W3"]) * (h2 > 0)
    g["W2"] = gh2.T @ h1
    g["b2"] = gh2.sum(axis=0)
    gh1 = (gh2 @ w["W2"]) * (h1 > 0)
    g["W1"] = gh1.T @ xs
    g["b1"] = gh1.sum(axis=0)
    return loss, pack(g)


def adam_step(flat, grad, m, v, t: int, lr: float):
    """One Adam step (t counts from 1); returns new (params, m, v)."""
    flat = np.asarray(flat, np.float64)
    grad = np.asarray(grad, np.float64)
    m = ADAM_B1 * np.asarray(m, np.float64) + (1 - ADAM_B1) * grad
    v = ADAM_B2 * np.asarray(v, np.float64) + (1 - ADAM_B2) * grad * grad
    mh = m / (1 - ADAM_B1 ** t)
    vh = v / (1 - ADAM_B2 ** t)
    return flat - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v


def select_k(keys, k: int) -> np.ndarray:
    """Per row, the positions of the k smallest keys, ordered by (key, position)."""
    keys = np.asarray(keys)
    pos = np.broadcast_to(np.arange(keys.shape[1]), keys.shape)
    order = np.lexsort((pos, keys), axis=1)
    return order[:, :k]


def fourier_descriptors(z, F: int = 32) -> np.ndarray:
    """log |Z[f]| for f = 1..F and f = -1..-F, Z = DFT(z)/N, of uniformly
    resampled curves z [M, N] (the rotation- and cyclic-shift-invariant
    magnitudes; Z[0] is the centroid and is left out)."""
    z = np.asarray(z, np.complex128)
    N = z.shape[1]
    Z = np.fft.fft(z, axis=1) / N
    f = np.arange(1, F + 1)
    mag = np.concatenate([np.abs(Z[:, f]), np.abs(Z[:, (N - f) % N])], axis=1)
    return np.log(mag + 1e-30)
