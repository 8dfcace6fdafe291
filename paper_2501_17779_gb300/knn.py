"""k-NN shape retrieval under the elastic distance (Sec. 3), with learned
candidate pruning.

Host orchestration only: every step runs in the library's kernels through the
C ABI (resampling, Fourier-magnitude descriptors, standardisation, the
pruning network's training and inference, embedding distances, k-selection
and the elastic distance itself).  The pruning network is this library's
addition, not the paper's: it ranks the gallery by the distance of learned
embeddings of rotation- and shift-invariant descriptors, and only the best
``n_cand`` candidates of each query are measured with the elastic distance.
The exact search (every gallery curve measured) is the fallback and the
reference that the pruned search's recall is measured against.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import api

N_FREQ = 32  # descriptor frequencies: |Z[+-1..+-32]|, 64 inputs


@dataclass
class Descriptors:
    x: torch.Tensor        # float32 [M, 64], standardised
    mean: torch.Tensor     # float32 [64]
    inv_std: torch.Tensor  # float32 [64]


def descriptors(curves: torch.Tensor, stats: Descriptors | None = None) -> Descriptors:
    """Standardised log-magnitude descriptors of curves [M, N] (complex128
    CUDA): arc-length resampling to N nodes, |Z[+-f]|, f = 1..32; the column
    statistics are taken from these curves unless ``stats`` is given."""
    M, N = curves.shape
    offs = torch.arange(0, M * N + 1, N, dtype=torch.int64, device=curves.device)
    z, _ = api.resample_arclength(curves.reshape(-1), offs, N)
    x = api.fourier_descriptors(z, N_FREQ)
    if stats is None:
        mean, inv = api.column_stats(x)
    else:
        mean, inv = stats.mean, stats.inv_std
    api.standardize_(x, mean, inv)
    return Descriptors(x, mean, inv)


def elastic_pairs(c1: torch.Tensor, c2: torch.Tensor, i1: torch.Tensor, i2: torch.Tensor,
                  band: int, chunk: int = 1 << 18) -> torch.Tensor:
    """Elastic energies E of pairs (c1[i1[p]], c2[i2[p]]), in chunks."""
    out = torch.empty(i1.numel(), dtype=torch.float64, device=c1.device)
    for a in range(0, i1.numel(), chunk):
        b = min(a + chunk, i1.numel())
        _, _, e, _, _ = api.elastic_distance(c1, c2, idx1=i1[a:b], idx2=i2[a:b], band=band)
        out[a:b] = e
    return out


def training_pairs(desc: Descriptors, n_near: int = 16, n_rand: int = 8, seed: int = 0):
    """Pairs to learn from, chosen without labels: each gallery curve with its
    ``n_near`` nearest curves in descriptor space and ``n_rand`` random ones."""
    G = desc.x.shape[0]
    dev = desc.x.device
    near = []
    step = max(1, (1 << 27) // max(G, 1))  # rows of the G x G distance matrix per block
    for a in range(0, G, step):
        b = min(a + step, G)
        d = api.embed_sqdist(desc.x[a:b], desc.x)
        near.append(api.select_k(d, n_near + 1)[:, 1:])
    near = torch.cat(near)
    gen = torch.Generator(device=dev).manual_seed(seed)
    ar = torch.arange(G, device=dev)
    pi = torch.cat([ar.repeat_interleave(n_near), ar.repeat_interleave(n_rand)])
    pj = torch.cat([near.reshape(-1), torch.randint(0, G, (G * n_rand,), device=dev, generator=gen)])
    return pi, pj


def train_pruner(gallery: torch.Tensor, desc: Descriptors, *, band: int, steps: int = 1500,
                 batch: int = 4096, lr: float = 1e-3, seed: int = 0, n_near: int = 16,
                 n_rand: int = 8):
    """Train the pruning network on elastic distances of gallery pairs (the
    method's own distances are the targets).  Returns (net, final loss,
    number of elastic distances computed)."""
    pi, pj = training_pairs(desc, n_near, n_rand, seed)
    d = torch.sqrt(torch.clamp(elastic_pairs(gallery, gallery, pi, pj, band), min=0.0)).float()
    net = api.Mlp(seed=seed + 1)
    gen = torch.Generator(device=gallery.device).manual_seed(seed + 2)
    loss = None
    for s in range(steps):
        sel = torch.randint(0, pi.numel(), (batch,), device=gallery.device, generator=gen)
        rate = lr * 0.5 * (1.0 + np.cos(np.pi * s / steps)) + 1e-5
        loss = net.pair_grad(desc.x, pi[sel], pj[sel], d[sel])
        net.adam_step(rate)
    return net, (loss.item() if loss is not None else float("nan")), int(pi.numel())


def search(queries: torch.Tensor, gallery: torch.Tensor, *, k: int = 10, band: int,
           n_cand: int | None = None, qdesc: torch.Tensor | None = None,
           gdesc: torch.Tensor | None = None, net: api.Mlp | None = None):
    """The k nearest gallery curves of each query under the elastic distance.

    With ``n_cand`` (and the queries' and gallery's descriptors ``qdesc``,
    ``gdesc``) only the ``n_cand`` candidates nearest in embedding space (the
    network's, or the raw descriptors' when ``net`` is None) are measured;
    without it every gallery curve is (exact search).  Returns (indices
    int64 [Q, k], energies float64 [Q, k]) ascending."""
    Q, G = queries.shape[0], gallery.shape[0]
    dev = queries.device
    if n_cand is None:
        cand = torch.arange(G, device=dev).repeat(Q, 1)
    else:
        eq = net.forward(qdesc) if net is not None else qdesc
        eg = net.forward(gdesc) if net is not None else gdesc
        cand = api.select_k(api.embed_sqdist(eq, eg), n_cand)
    C = cand.shape[1]
    qi = torch.arange(Q, device=dev).repeat_interleave(C)
    e = elastic_pairs(queries, gallery, qi, cand.reshape(-1), band).view(Q, C)
    pos, ek = api.select_k(e, k, with_keys=True)
    return torch.gather(cand, 1, pos), ek


def recall_at_k(found: torch.Tensor, exact: torch.Tensor) -> float:
    f, x = found.cpu().numpy(), exact.cpu().numpy()
    k = x.shape[1]
    return float(np.mean([len(set(f[q]) & set(x[q])) / k for q in range(x.shape[0])]))


def save_pruner(path, net: api.Mlp, stats: Descriptors) -> None:
    """Save the pruning network's float32 parameters and the descriptor
    statistics it was trained with (numpy .npz)."""
    np.savez(path, params=net.get_params(), mean=stats.mean.cpu().numpy(),
             inv_std=stats.inv_std.cpu().numpy(), n_freq=N_FREQ)


def load_pruner(path, device: int | None = None):
    """Load a network saved by ``save_pruner``: returns (net, stats) with
    ``stats`` usable as the ``stats`` argument of ``descriptors``."""
    d = np.load(path)
    if int(d["n_freq"]) != N_FREQ:
        raise ValueError("descriptor size differs from this library's")
    net = api.Mlp(seed=0, device=device)
    net.set_params(d["params"])
    dev = net.device
    stats = Descriptors(torch.empty((0, 2 * N_FREQ), dtype=torch.float32, device=dev),
                        torch.from_numpy(d["mean"]).to(dev), torch.from_numpy(d["inv_std"]).to(dev))
    return net, stats
