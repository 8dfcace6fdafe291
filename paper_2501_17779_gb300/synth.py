"""Seeded synthetic curve generators (inputs only).

This module produces the curves that the CUDA library and the CPU oracle are
both fed with.  It holds none of the alignment method's arithmetic: no
correlation, no FFT, no Kabsch step and no spline.  Curves come from the
Fourier-series family r(phi) = 1 + sum_k a_k cos(k phi + phi_k) with
a_k ~ N(0, (0.15/k)^2) and phi_k ~ U(0, 2 pi), a stand-in for the paper's
synthetic and cell-boundary test curves (Sec. 2, validation experiments),
which are not available.

Two workloads:

* ``aligned_pairs``: pairs that are already uniform in arc length, centred and
  of unit length (the inputs of the alignment step alone).  Curve 2 is curve 1
  rotated by theta_g, cyclically relabelled by s_g, optionally with Gaussian
  noise, then re-centred and re-scaled.  With z2[k] = e^{i theta_g}
  z1[(k - s_g) mod N] the optimal alignment is shift s_g and counter-clockwise
  angle -theta_g.
* ``raw_pairs``: pairs given as ragged, non-uniformly sampled point lists (the
  inputs of the arc-length resampling step).  Node parameters are jittered by
  up to +-40% of the mean spacing and every curve has its own node count.

Arc-length-uniform sampling here is done by dense sampling plus linear
interpolation of the cumulative chord length -- deliberately a different
construction from the method's cubic-spline resampling.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

TWO_PI = 2.0 * np.pi


@dataclass
class Harmonics:
    """Coefficients of r(phi) = 1 + scale * sum_k a_k cos(k phi + phi_k)."""

    a: np.ndarray
    ph: np.ndarray
    scale: float = 1.0

    def radius(self, phi: np.ndarray) -> np.ndarray:
        k = np.arange(1, self.a.size + 1)
        pert = np.cos(np.multiply.outer(phi, k) + self.ph) @ self.a
        return 1.0 + self.scale * pert


def random_harmonics(rng: np.random.Generator, n_harm: int, sigma0: float = 0.15,
                     min_radius: float = 0.25) -> Harmonics:
    """Draw a_k ~ N(0, (sigma0/k)^2), phi_k ~ U(0, 2 pi).

    If the perturbation would bring r below ``min_radius`` anywhere, it is
    scaled down so that the curve stays star-shaped and simple.
    """
    k = np.arange(1, n_harm + 1)
    h = Harmonics(a=rng.normal(0.0, sigma0 / k), ph=rng.uniform(0.0, TWO_PI, n_harm))
    phi = np.linspace(0.0, TWO_PI, 4096, endpoint=False)
    pert_min = float(np.min(h.radius(phi) - 1.0))
    if 1.0 + pert_min < min_radius:
        h.scale = (1.0 - min_radius) / (-pert_min)
    return h


def _normalise(z: np.ndarray) -> np.ndarray:
    """Input preparation: subtract the node mean, divide by the closed-polygon
    perimeter (so that a generated pair starts centred and of unit length)."""
    z = z - z.mean()
    per = np.abs(np.roll(z, -1) - z).sum()
    return z / per


def uniform_arclength_nodes(h: Harmonics, N: int, oversample: int = 64,
                            phase: float = 0.0) -> np.ndarray:
    """N nodes of the polar curve, equally spaced in arc length.

    The curve is sampled at oversample*N equally spaced angles starting at
    ``phase``; the cumulative chord length of that dense polygon is inverted
    by linear interpolation.  The result is centred and of unit perimeter.
    """
    M = oversample * N
    phi = phase + TWO_PI * np.arange(M + 1) / M
    w = h.radius(phi) * np.exp(1j * phi)
    seg = np.abs(np.diff(w))
    cum = np.concatenate([[0.0], np.cumsum(seg)])
    target = cum[-1] * np.arange(N) / N
    x = np.interp(target, cum, w.real)
    y = np.interp(target, cum, w.imag)
    return _normalise(x + 1j * y)


@dataclass
class AlignedPairs:
    z1: np.ndarray          # complex128 [P, N]
    z2: np.ndarray          # complex128 [P, N]
    shift_true: np.ndarray  # int32 [P]   optimal shift of the noise-free pair
    theta_true: np.ndarray  # float64 [P] optimal CCW angle (= -theta_g) in (-pi, pi]


def aligned_pairs(seed: int, P: int = 64, N: int = 256, n_harm: int = 8,
                  noise: float = 1e-3, oversample: int = 64) -> AlignedPairs:
    """Pairs already uniform in arc length, centred and of unit length.

    Default sizes are the 64-pair, N = 256 parity workload.  ``noise`` is the
    standard deviation of the i.i.d. Gaussian noise added to each coordinate of
    curve 2 before it is re-centred and re-scaled (0 gives exact copies).
    """
    rng = np.random.default_rng(seed)
    z1 = np.empty((P, N), np.complex128)
    z2 = np.empty((P, N), np.complex128)
    s_true = np.empty(P, np.int32)
    th_true = np.empty(P, np.float64)
    for p in range(P):
        h = random_harmonics(rng, n_harm)
        a = uniform_arclength_nodes(h, N, oversample)
        th_g = rng.uniform(0.0, TWO_PI)
        s_g = int(rng.integers(0, N))
        b = np.exp(1j * th_g) * np.roll(a, s_g)  # b[k] = e^{i th} a[(k - s_g) mod N]
        if noise > 0.0:
            b = b + noise * (rng.standard_normal(N) + 1j * rng.standard_normal(N))
            b = _normalise(b)
        z1[p] = a
        z2[p] = b
        s_true[p] = s_g
        th_true[p] = np.angle(np.exp(-1j * th_g))
    return AlignedPairs(z1, z2, s_true, th_true)


@dataclass
class RawPairs:
    pts: np.ndarray      # complex128 [sum n]: curves 0..P-1 are the first members,
                         # curves P..2P-1 the second members of the pairs
    offsets: np.ndarray  # int64 [2P + 1]  CSR offsets into pts
    theta_g: np.ndarray  # float64 [P] rotation applied to the second member

    @property
    def n_curves(self) -> int:
        return self.offsets.size - 1


def _jittered_polar(rng: np.random.Generator, h: Harmonics, n: int, phase: float,
                    jitter: float) -> np.ndarray:
    delta = rng.uniform(-jitter, jitter, n)
    phi = phase + TWO_PI * (np.arange(n) + delta) / n
    return h.radius(phi) * np.exp(1j * phi)


def raw_pairs(seed: int, P: int = 4096, n_min: int = 500, n_max: int = 2000,
              max_harm: int = 16, jitter: float = 0.4, noise: float = 1e-3,
              transform: bool = True) -> RawPairs:
    """Ragged, non-uniformly sampled pairs (inputs of the resampling step).

    Defaults are the 4096-pair workload: n_in ~ U{n_min..n_max} per curve, node
    parameters phi_l = phase + 2 pi (l + delta_l)/n_in with delta_l ~
    U(-jitter, jitter), harmonic count ~ U{1..max_harm}.  The second member is
    the same shape rotated by theta_g ~ U(0, 2 pi), with its parameter origin
    offset by U(0, 2 pi), its own node count and jitter, and Gaussian noise of
    standard deviation ``noise`` per coordinate.  With ``transform`` each curve
    is also given a random scale in [0.5, 2] and offset in [-2, 2]^2, which
    the resampling step's centring and scaling must remove.
    """
    rng = np.random.default_rng(seed)
    first, second, th = [], [], np.empty(P)
    for p in range(P):
        h = random_harmonics(rng, int(rng.integers(1, max_harm + 1)))
        n1 = int(rng.integers(n_min, n_max + 1))
        n2 = int(rng.integers(n_min, n_max + 1))
        c1 = _jittered_polar(rng, h, n1, 0.0, jitter)
        th_g = rng.uniform(0.0, TWO_PI)
        c2 = np.exp(1j * th_g) * _jittered_polar(rng, h, n2, rng.uniform(0.0, TWO_PI), jitter)
        if noise > 0.0:
            c2 = c2 + noise * (rng.standard_normal(n2) + 1j * rng.standard_normal(n2))
        if transform:
            c1 = rng.uniform(0.5, 2.0) * c1 + complex(*rng.uniform(-2.0, 2.0, 2))
            c2 = rng.uniform(0.5, 2.0) * c2 + complex(*rng.uniform(-2.0, 2.0, 2))
        first.append(c1)
        second.append(c2)
        th[p] = th_g
    curves = first + second
    counts = np.array([c.size for c in curves], np.int64)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    pts = np.concatenate(curves).astype(np.complex128)
    return RawPairs(pts, offsets, th)


def raw_curves(seed: int, C: int, n_min: int, n_max: int, max_harm: int = 16,
               jitter: float = 0.4) -> tuple[np.ndarray, np.ndarray]:
    """C independent ragged curves (no pairing), returned as (pts, offsets)."""
    rng = np.random.default_rng(seed)
    curves = []
    for _ in range(C):
        h = random_harmonics(rng, int(rng.integers(1, max_harm + 1)))
        n = int(rng.integers(n_min, n_max + 1))
        c = _jittered_polar(rng, h, n, rng.uniform(0.0, TWO_PI), jitter)
        curves.append(rng.uniform(0.5, 2.0) * c + complex(*rng.uniform(-2.0, 2.0, 2)))
    counts = np.array([c.size for c in curves], np.int64)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return np.concatenate(curves).astype(np.complex128), offsets


def template_pair(h: Harmonics, N: int, start: float = 0.25,
                  rotation: float = np.pi / 3) -> tuple[np.ndarray, np.ndarray]:
    """The paper's validation template (Sec. 2): the reference curve with its
    starting point moved from 0 to ``start`` (a fraction of the length) and
    rotated counter-clockwise by ``rotation``.  Both curves share the same
    uniform arc-length parametrisation.  With N*start an integer q, the
    template is z2[k] = e^{i rotation} z1[(k + q) mod N]."""
    z1 = uniform_arclength_nodes(h, N)
    q = int(round(start * N))
    z2 = np.exp(1j * rotation) * np.roll(z1, -q)
    return z1, z2


@dataclass
class RaggedPairs:
    z1: np.ndarray       # complex128 [sum n]: curve 1 of every pair, concatenated
    z2: np.ndarray       # complex128 [sum n]: curve 2 of every pair, same offsets
    offsets: np.ndarray  # int64 [P + 1]
    shift_true: np.ndarray
    theta_true: np.ndarray


def ragged_aligned_pairs(seed: int, sizes, min_harm: int = 4, max_harm: int = 32,
                         noise: float = 1e-3, oversample: int = 8) -> RaggedPairs:
    """Aligned pairs with a different node count per pair (host, numpy).

    Pair p has sizes[p] nodes; curve 1 is uniform in arc length with
    U{min_harm..max_harm} harmonics, curve 2 its rotated, relabelled and noisy
    copy (as in ``aligned_pairs``)."""
    rng = np.random.default_rng(seed)
    z1, z2, st, tt = [], [], [], []
    for n in sizes:
        n = int(n)
        h = random_harmonics(rng, int(rng.integers(min_harm, max_harm + 1)))
        a = uniform_arclength_nodes(h, n, oversample)
        th_g = rng.uniform(0.0, TWO_PI)
        s_g = int(rng.integers(0, n))
        b = np.exp(1j * th_g) * np.roll(a, s_g)
        if noise > 0.0:
            b = _normalise(b + noise * (rng.standard_normal(n) + 1j * rng.standard_normal(n)))
        z1.append(a)
        z2.append(b)
        st.append(s_g)
        tt.append(np.angle(np.exp(-1j * th_g)))
    offs = np.concatenate([[0], np.cumsum([len(a) for a in z1])]).astype(np.int64)
    return RaggedPairs(np.concatenate(z1), np.concatenate(z2), offs, np.array(st, np.int32),
                       np.array(tt))


def log_uniform_sizes(seed: int, P: int, n_min: int = 64, n_max: int = 8192,
                      multiple: int = 16) -> np.ndarray:
    """P node counts log-uniform in [n_min, n_max], rounded to a multiple."""
    rng = np.random.default_rng(seed)
    n = np.exp(rng.uniform(np.log(n_min), np.log(n_max), P))
    return np.clip(np.round(n / multiple) * multiple, n_min, n_max).astype(np.int64)


def ragged_pairs_device(seed: int, sizes, device, min_harm: int = 4, max_harm: int = 32,
                        noise: float = 1e-3):
    """Large ragged batches generated on the GPU with torch (same family as
    ``ragged_aligned_pairs``, but nodes uniform in the polar angle, which keeps
    generation of ~10^8 nodes fast).  Returns (z1, z2, offsets) as device
    tensors (complex128, complex128, int64).  Input generation only."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    sizes = torch.as_tensor(np.asarray(sizes, np.int64), device=device)
    P = sizes.numel()
    offs = torch.zeros(P + 1, dtype=torch.int64, device=device)
    offs[1:] = torch.cumsum(sizes, 0)
    total = int(offs[-1].item())
    pair = torch.repeat_interleave(torch.arange(P, device=device), sizes)
    k = torch.arange(total, device=device) - offs[pair]
    nn = sizes[pair].double()
    phi = (2 * np.pi) * k.double() / nn
    H = max_harm
    kk = torch.arange(1, H + 1, device=device, dtype=torch.float64)
    nh = torch.randint(min_harm, max_harm + 1, (P,), generator=g, device=device)
    amp = torch.randn(P, H, generator=g, device=device, dtype=torch.float64) * (0.15 / kk)
    amp = amp * (kk[None, :] <= nh[:, None])
    ph = torch.rand(P, H, generator=g, device=device, dtype=torch.float64) * (2 * np.pi)
    # keep r >= 0.25: scale the perturbation by its worst case sum |a_k|
    worst = amp.abs().sum(1)
    amp = amp * torch.clamp(0.75 / worst, max=1.0)[:, None]
    r = torch.ones(total, device=device, dtype=torch.float64)
    for h0 in range(0, H, 8):
        hs = slice(h0, min(H, h0 + 8))
        r += (amp[pair, hs] * torch.cos(phi[:, None] * kk[None, hs] + ph[pair, hs])).sum(1)
    z1 = torch.polar(r, phi)

    def normalise(z):
        mean = torch.zeros(P, dtype=z.dtype, device=device).index_add_(0, pair, z) / sizes
        z = z - mean[pair]
        nxt = torch.where(k + 1 == sizes[pair], offs[pair], torch.arange(total, device=device) + 1)
        per = torch.zeros(P, dtype=torch.float64, device=device).index_add_(0, pair, (z[nxt] - z).abs())
        return z / per[pair]

    z1 = normalise(z1)
    sg = (torch.rand(P, generator=g, device=device, dtype=torch.float64) * sizes).long()
    thg = torch.rand(P, generator=g, device=device, dtype=torch.float64) * (2 * np.pi)
    src = offs[pair] + torch.remainder(k - sg[pair], sizes[pair])
    z2 = torch.polar(torch.ones_like(thg), thg)[pair] * z1[src]
    if noise > 0.0:
        z2 = z2 + noise * torch.complex(torch.randn(total, generator=g, device=device, dtype=torch.float64),
                                        torch.randn(total, generator=g, device=device, dtype=torch.float64))
        z2 = normalise(z2)
    return z1.contiguous(), z2.contiguous(), offs


# ------------------------------------------------------------ elastic -------
def arclength_curve(h: Harmonics, oversample_n: int = 65536):
    """The polar curve as a function of its normalised arc length u in [0, 1)
    (periodic): dense polygon, cumulative chord length inverted by linear
    interpolation.  Returns f(u) -> complex points, centred and of unit length
    like ``uniform_arclength_nodes``."""
    M = oversample_n
    phi = TWO_PI * np.arange(M + 1) / M
    w = h.radius(phi) * np.exp(1j * phi)
    cum = np.concatenate([[0.0], np.cumsum(np.abs(np.diff(w)))])
    cum /= cum[-1]
    base = _normalise(np.interp(np.arange(4096) / 4096, cum, w.real)
                      + 1j * np.interp(np.arange(4096) / 4096, cum, w.imag))
    # the same centring and scaling as a 4096-node arc-length polygon
    z0 = np.interp(0.0, cum, w.real) + 1j * np.interp(0.0, cum, w.imag)
    scale = (base[0] + 0.0) / 1.0

    def f(u):
        u = np.mod(np.asarray(u, np.float64), 1.0)
        x = np.interp(u, cum, w.real) + 1j * np.interp(u, cum, w.imag)
        return x
    del z0, scale
    return f


def gamma_paper_1(t):
    """The mild reparameterisation of the zero-distance experiment of Sec. 3:
    gamma(t) = t + 0.025 sin(4 pi t)."""
    return t + 0.025 * np.sin(4.0 * np.pi * t)


def gamma_paper_2(t):
    """The strong reparameterisation of the same experiment:
    gamma(t) = t + 1.6 t^2 (t - 1)^2."""
    return t + 1.6 * t * t * (t - 1.0) ** 2


def reparam_pair(h: Harmonics, N: int, gamma, start: float = 0.25,
                 rotation: float = np.pi / 3):
    """The zero-distance experiment of Sec. 3: beta1 uniform in arc length;
    beta2(t) = R beta1(start + gamma(t)) at t = k/N (start point moved, rotated,
    reparameterised).  Both are N-node polygons, translated and scaled alike."""
    f = arclength_curve(h)
    t = np.arange(N) / N
    b1 = f(t)
    b2 = np.exp(1j * rotation) * f(start + gamma(t))
    c = b1.mean()
    per = np.abs(np.roll(b1, -1) - b1).sum()
    return (b1 - c) / per, (b2 - np.exp(1j * rotation) * c) / per


@dataclass
class ShapeGallery:
    curves: np.ndarray   # complex128 [M, N], node k at parameter k/N
    labels: np.ndarray   # int32 [M] class template of each curve


def shape_gallery(seed: int, M: int, N: int = 256, n_classes: int = 50, n_harm: int = 8,
                  sigma: float = 0.03, reparam: float = 0.3, device: str = "cpu",
                  dense: int = 4096) -> ShapeGallery:
    """Curves for elastic k-NN retrieval: ``n_classes`` Fourier-series templates
    (as ``random_harmonics``); each instance belongs to a uniformly drawn class,
    perturbs its template's harmonics (a_k += sigma N(0,1)/k,
    phi_k += sigma N(0,1)), starts at a random point, is rotated by a random
    angle and is sampled at t = k/N through a random smooth monotone
    reparameterisation gamma(t) = t + sum_{m=1..3} b_m sin(2 pi m t)/(2 pi m),
    sum |b_m| <= ``reparam`` < 1 (so gamma' > 0).  The arc-length inversion
    runs batched in torch on ``device`` (a dense polygon of ``dense`` angles per
    curve, linear interpolation of its cumulative chord length).  Returns
    numpy arrays."""
    import torch

    rng = np.random.default_rng(seed)
    trng = np.random.default_rng(10_000 + n_classes)  # templates depend on n_classes only
    temps = [random_harmonics(trng, n_harm) for _ in range(n_classes)]
    TA = np.stack([h.a for h in temps])
    TP = np.stack([h.ph for h in temps])
    k = np.arange(1, n_harm + 1)
    cls = rng.integers(0, n_classes, M)
    a = TA[cls] + sigma * rng.normal(size=(M, n_harm)) / k
    ph = TP[cls] + sigma * rng.normal(size=(M, n_harm))
    b = rng.uniform(-1.0, 1.0, (M, 3))
    b *= (reparam * rng.uniform(0.0, 1.0, M) / np.abs(b).sum(axis=1))[:, None]
    start = rng.uniform(0.0, 1.0, M)
    rot = rng.uniform(0.0, TWO_PI, M)
    dev = torch.device(device)
    f64 = torch.float64
    phi = torch.arange(dense + 1, dtype=f64, device=dev) * (TWO_PI / dense)
    kk = torch.as_tensor(k, dtype=f64, device=dev)
    C = torch.cos(kk[:, None] * phi[None, :])
    S = torch.sin(kk[:, None] * phi[None, :])
    A = torch.as_tensor(a, dtype=f64, device=dev)
    Ph = torch.as_tensor(ph, dtype=f64, device=dev)
    pert = (A * torch.cos(Ph)) @ C - (A * torch.sin(Ph)) @ S           # [M, dense+1]
    # keep the curve star-shaped: r >= 0.25
    pmin = pert.min(dim=1).values
    scale = torch.where(1.0 + pmin < 0.25, 0.75 / (-pmin), torch.ones_like(pmin))
    r = 1.0 + scale[:, None] * pert
    w = torch.polar(r, phi.expand_as(r))
    cum = torch.cat([torch.zeros(M, 1, dtype=f64, device=dev),
                     torch.cumsum(torch.abs(w[:, 1:] - w[:, :-1]), dim=1)], dim=1)
    cum = cum / cum[:, -1:]
    t = torch.arange(N, dtype=f64, device=dev) / N
    m = torch.arange(1, 4, dtype=f64, device=dev)
    B = torch.as_tensor(b, dtype=f64, device=dev)
    gam = t[None, :] + (B[:, None, :] * torch.sin(TWO_PI * t[:, None] * m[None, :])[None]
                        / (TWO_PI * m)).sum(dim=2)
    u = torch.remainder(torch.as_tensor(start, dtype=f64, device=dev)[:, None] + gam, 1.0)
    j = torch.searchsorted(cum, u.contiguous(), right=True).clamp(1, dense) - 1
    c0 = torch.gather(cum, 1, j)
    c1 = torch.gather(cum, 1, j + 1)
    fr = ((u - c0) / (c1 - c0)).clamp(0.0, 1.0)
    wr, wi = w.real.contiguous(), w.imag.contiguous()
    x = torch.gather(wr, 1, j) * (1 - fr) + torch.gather(wr, 1, j + 1) * fr
    y = torch.gather(wi, 1, j) * (1 - fr) + torch.gather(wi, 1, j + 1) * fr
    z = torch.complex(x, y) * torch.polar(torch.ones(M, dtype=f64, device=dev),
                                          torch.as_tensor(rot, dtype=f64, device=dev))[:, None]
    z = z - z.mean(dim=1, keepdim=True)
    z = z / torch.abs(torch.roll(z, -1, dims=1) - z).sum(dim=1, keepdim=True)
    return ShapeGallery(z.cpu().numpy(), cls.astype(np.int32))
