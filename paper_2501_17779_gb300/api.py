"""Python binding of libfftalign.so: argument marshalling only.

Every step of the method runs in the library's CUDA kernels; PyTorch supplies
device memory and the current CUDA stream.  Functions mirror the C ABI of
include/fftalign.h:

* ``resample_arclength``  -> fa_resample_arclength
* ``align_pairs``         -> fa_align_pairs
* ``align_all_pairs``     -> fa_align_all_pairs
* ``align_pairs_ragged``  -> fa_align_pairs_ragged (+ _autotune)
* ``align_curves_host``   -> fa_align_curves_host (host buffers in and out)
"""
from __future__ import annotations

import ctypes
import threading

import torch

from . import _lib

_handles: dict[int, int] = {}
_hlock = threading.Lock()


def handle(device: int | None = None) -> int:
    """The process-wide library handle for a CUDA device (created on first use)."""
    if not torch.cuda.is_available():
        raise RuntimeError("libfftalign needs a CUDA device; none is available")
    dev = torch.cuda.current_device() if device is None else int(device)
    with _hlock:
        h = _handles.get(dev)
        if h is None:
            L = _lib.load()
            hp = ctypes.c_void_p()
            _lib.check(L.fa_create(ctypes.byref(hp), dev))
            h = _handles[dev] = hp.value
    return h


def _stream_ptr(device: torch.device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def _need_cuda(name: str, t: torch.Tensor, dtype=None) -> None:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def resample_workspace_size(C: int, n_pts: int, N_out: int, fp32: bool = False) -> int:
    L = _lib.load()
    flags = _lib.CENTER | _lib.UNIT_LENGTH | (_lib.STORE_FP32 if fp32 else 0)
    return int(L.fa_resample_workspace_size(C, n_pts, N_out, flags))


def resample_arclength(pts: torch.Tensor, offsets: torch.Tensor, N_out: int, *,
                       center: bool = True, unit_length: bool = True, fp32: bool = False,
                       out: torch.Tensor | None = None, status: torch.Tensor | None = None,
                       workspace: torch.Tensor | None = None):
    """Arc-length resampling of C ragged curves (Sec. 2 of the paper).

    pts: complex128 CUDA tensor [n_pts] (all curves' distinct nodes);
    offsets: int64 CUDA tensor [C+1].  Returns (z [C, N_out] complex128 or
    complex64, status int8 [C]).  A workspace (uint8 CUDA tensor of at least
    resample_workspace_size() bytes) is allocated through torch when not given.
    """
    _need_cuda("pts", pts, torch.complex128)
    _need_cuda("offsets", offsets, torch.int64)
    C = offsets.numel() - 1
    if C < 0:
        raise ValueError("offsets must have at least one entry")
    dev = pts.device
    flags = (_lib.CENTER if center else 0) | (_lib.UNIT_LENGTH if unit_length else 0) | \
            (_lib.STORE_FP32 if fp32 else 0)
    zdt = torch.complex64 if fp32 else torch.complex128
    if out is None:
        out = torch.empty((C, N_out), dtype=zdt, device=dev)
    else:
        _need_cuda("out", out, zdt)
    if status is None:
        status = torch.empty(C, dtype=torch.int8, device=dev)
    L = _lib.load()
    n_pts = pts.numel()
    need = int(L.fa_resample_workspace_size(C, n_pts, N_out, flags))
    if workspace is None:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    h = handle(dev.index)
    rc = L.fa_resample_arclength(h, _ptr(pts), _ptr(offsets), C, n_pts, N_out, flags,
                                 _ptr(out), _ptr(status), _ptr(workspace), workspace.numel(),
                                 _stream_ptr(dev))
    _lib.check(rc)
    return out, status


_METHODS = {"fft": _lib.FFT, "direct": _lib.DIRECT}
_PRECS = {"fp64": _lib.PREC_FP64, "mixed": _lib.PREC_MIXED, "tc_bf16x3": _lib.PREC_TC_BF16X3,
          "tc_fp16x3": _lib.PREC_TC_FP16X3, "tc_tf32": _lib.PREC_TC_TF32,
          "tc_tf32x3": _lib.PREC_TC_TF32X3}


def align_pairs(z1: torch.Tensor, z2: torch.Tensor, *, method: str = "fft", prec: str = "fp64",
                out: tuple | None = None):
    """Optimal start point and rotation for P pairs of curves (Algorithm 2).

    z1, z2: [P, N] complex128 or complex64 CUDA tensors (centred, unit length).
    Returns (shift int32 [P], theta float64 [P], energy float64 [P],
    status int8 [P]); theta is the counter-clockwise angle applied to curve 2.
    """
    if z1.dtype not in (torch.complex128, torch.complex64):
        raise ValueError("z1 must be complex128 or complex64")
    _need_cuda("z1", z1, z1.dtype)
    _need_cuda("z2", z2, z1.dtype)
    if z1.dim() != 2 or z1.shape != z2.shape:
        raise ValueError("z1 and z2 must both be [P, N]")
    P, N = z1.shape
    dev = z1.device
    if out is None:
        shift = torch.empty(P, dtype=torch.int32, device=dev)
        theta = torch.empty(P, dtype=torch.float64, device=dev)
        energy = torch.empty(P, dtype=torch.float64, device=dev)
        status = torch.empty(P, dtype=torch.int8, device=dev)
    else:
        shift, theta, energy, status = out
    ztype = _lib.Z_F64 if z1.dtype == torch.complex128 else _lib.Z_F32
    L = _lib.load()
    h = handle(dev.index)
    rc = L.fa_align_pairs(h, _ptr(z1), _ptr(z2), P, N, ztype, _METHODS[method], _PRECS[prec],
                          _ptr(shift), _ptr(theta), _ptr(energy), _ptr(status), _stream_ptr(dev))
    _lib.check(rc)
    return shift, theta, energy, status


def align_all_pairs(z: torch.Tensor, *, prec: str = "fp64", workspace: torch.Tensor | None = None):
    """Alignment matrix of M curves (fa_align_all_pairs).

    z: [M, N] complex128 or complex64 CUDA tensor.  prec: "fp64", "mixed", or
    a tensor-core search "tc_bf16x3", "tc_fp16x3", "tc_tf32", "tc_tf32x3"
    (N = 256 or 512).  Returns (shift int32 [M, M], theta float64 [M, M],
    energy float64 [M, M], status int8 [M]); entry (i, j) aligns curve j onto
    curve i.
    """
    if z.dtype not in (torch.complex128, torch.complex64):
        raise ValueError("z must be complex128 or complex64")
    _need_cuda("z", z, z.dtype)
    if z.dim() != 2:
        raise ValueError("z must be [M, N]")
    M, N = z.shape
    dev = z.device
    shift = torch.empty((M, M), dtype=torch.int32, device=dev)
    theta = torch.empty((M, M), dtype=torch.float64, device=dev)
    energy = torch.empty((M, M), dtype=torch.float64, device=dev)
    status = torch.empty(M, dtype=torch.int8, device=dev)
    L = _lib.load()
    need = int(L.fa_align_all_pairs_workspace_size_prec(M, N, _PRECS[prec]))
    if workspace is None:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    ztype = _lib.Z_F64 if z.dtype == torch.complex128 else _lib.Z_F32
    rc = L.fa_align_all_pairs(handle(dev.index), _ptr(z), M, N, ztype, _PRECS[prec], _ptr(shift),
                              _ptr(theta), _ptr(energy), _ptr(status), _ptr(workspace),
                              workspace.numel(), _stream_ptr(dev))
    _lib.check(rc)
    return shift, theta, energy, status


def align_pairs_ragged(z1: torch.Tensor, z2: torch.Tensor, offsets: torch.Tensor, *,
                       max_n: int | None = None, workspace: torch.Tensor | None = None,
                       autotune: bool = False, out: tuple | None = None):
    """Alignment of pairs with different node counts (fa_align_pairs_ragged).

    z1, z2: flat complex128/complex64 CUDA tensors of offsets[-1] points; pair p
    is [offsets[p], offsets[p+1]) in both.  offsets: int64 CUDA tensor [P+1].
    max_n bounds every pair's node count (default: computed from offsets, which
    reads them back to the host).  With ``autotune`` each bucket's plan (CTA
    size, pairs per CTA) is chosen by timed runs first
    (fa_align_pairs_ragged_autotune; see ragged_plan).  Returns (shift, theta,
    energy, status) [P] each.
    """
    if z1.dtype not in (torch.complex128, torch.complex64):
        raise ValueError("z1 must be complex128 or complex64")
    _need_cuda("z1", z1, z1.dtype)
    _need_cuda("z2", z2, z1.dtype)
    _need_cuda("offsets", offsets, torch.int64)
    P = offsets.numel() - 1
    dev = z1.device
    if max_n is None:
        max_n = int((offsets[1:] - offsets[:-1]).max().item()) if P > 0 else 4
        max_n = min(max(max_n, 4), 8192)
    if out is None:
        shift = torch.empty(P, dtype=torch.int32, device=dev)
        theta = torch.empty(P, dtype=torch.float64, device=dev)
        energy = torch.empty(P, dtype=torch.float64, device=dev)
        status = torch.empty(P, dtype=torch.int8, device=dev)
    else:
        shift, theta, energy, status = out
    L = _lib.load()
    h = handle(dev.index)
    need = int(L.fa_align_pairs_ragged_workspace_size(h, P, max_n))
    if workspace is None:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    ztype = _lib.Z_F64 if z1.dtype == torch.complex128 else _lib.Z_F32
    args = (h, _ptr(z1), _ptr(z2), _ptr(offsets), P, max_n, ztype, _ptr(shift), _ptr(theta),
            _ptr(energy), _ptr(status), _ptr(workspace), workspace.numel(), _stream_ptr(dev))
    if autotune:
        chosen = ctypes.c_int32(0)
        _lib.check(L.fa_align_pairs_ragged_autotune(*args, ctypes.byref(chosen)))
    else:
        _lib.check(L.fa_align_pairs_ragged(*args))
    return shift, theta, energy, status


def ragged_plan(device: int | None = None) -> dict:
    """The handle's per-bucket plan for align_pairs_ragged (fa_align_pairs_ragged_plan):
    {log2 L: (CTA size, pairs per CTA, ms of the last autotuning)} for the
    supported transform lengths; pairs per CTA is -R for a plan in which a
    thread-block cluster of R CTAs shares one pair (L = 8192, 16384)."""
    L = _lib.load()
    t = (ctypes.c_int32 * 16)()
    g = (ctypes.c_int32 * 16)()
    ms = (ctypes.c_float * 16)()
    _lib.check(L.fa_align_pairs_ragged_plan(handle(device), t, g, ms))
    return {b: (int(t[b]), int(g[b]), float(ms[b])) for b in range(16) if t[b] > 0}


def set_ragged_plan(bucket: int, threads: int, pairs_per_cta: int,
                    device: int | None = None) -> None:
    """Pins the plan of one transform-length bucket (fa_align_pairs_ragged_set_plan)."""
    L = _lib.load()
    _lib.check(L.fa_align_pairs_ragged_set_plan(handle(device), bucket, threads, pairs_per_cta))


def ragged_workspace_size(P: int, max_n: int, device: int | None = None) -> int:
    L = _lib.load()
    return int(L.fa_align_pairs_ragged_workspace_size(handle(device), P, max_n))


def elastic_workspace_size(M1: int, M2: int, P: int, N: int, band: int = -1,
                           device: int | None = None) -> int:
    L = _lib.load()
    return int(L.fa_elastic_workspace_size(handle(device), M1, M2, P, N, band))


def elastic_distance(curves1: torch.Tensor, curves2: torch.Tensor, *,
                     idx1: torch.Tensor | None = None, idx2: torch.Tensor | None = None,
                     band: int = -1, max_iter: int = 20, gamma: bool = False,
                     workspace: torch.Tensor | None = None, out: tuple | None = None,
                     lm_steps: torch.Tensor | None = None):
    """Elastic shape distance (fa_elastic_distance).

    curves1 [M1, N], curves2 [M2, N]: complex128 CUDA tensors, node k of a curve
    at parameter k/N.  Pair p is (idx1[p], idx2[p]) (int64 CUDA tensors) or,
    without them, (p, p).  Returns (shift int32, theta, energy, iters int32,
    status int8) [P] each, plus gamma [P, N+1] when ``gamma``; the distance is
    sqrt(energy).  ``lm_steps`` (int32 CUDA tensor [P]) receives the
    refinement steps each pair took.
    """
    _need_cuda("curves1", curves1, torch.complex128)
    _need_cuda("curves2", curves2, torch.complex128)
    if curves1.dim() != 2 or curves2.dim() != 2 or curves1.shape[1] != curves2.shape[1]:
        raise ValueError("curves1, curves2 must be [M1, N], [M2, N]")
    M1, N = curves1.shape
    M2 = curves2.shape[0]
    if (idx1 is None) != (idx2 is None):
        raise ValueError("give both index arrays or neither")
    if idx1 is not None:
        _need_cuda("idx1", idx1, torch.int64)
        _need_cuda("idx2", idx2, torch.int64)
        P = idx1.numel()
        if idx2.numel() != P:
            raise ValueError("idx1 and idx2 differ in length")
    else:
        P = min(M1, M2)
    dev = curves1.device
    if out is None:
        shift = torch.empty(P, dtype=torch.int32, device=dev)
        theta = torch.empty(P, dtype=torch.float64, device=dev)
        energy = torch.empty(P, dtype=torch.float64, device=dev)
        iters = torch.empty(P, dtype=torch.int32, device=dev)
        status = torch.empty(P, dtype=torch.int8, device=dev)
    else:
        shift, theta, energy, iters, status = out
    g = torch.empty((P, N + 1), dtype=torch.float64, device=dev) if gamma else None
    L = _lib.load()
    h = handle(dev.index)
    need = int(L.fa_elastic_workspace_size(h, M1, M2, P, N, band))
    if workspace is None:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    rc = L.fa_elastic_distance(h, _ptr(curves1), M1, _ptr(curves2), M2, N, _ptr(idx1),
                               _ptr(idx2), P, band, max_iter, _ptr(shift), _ptr(theta),
                               _ptr(energy), _ptr(g), _ptr(iters), _ptr(lm_steps), _ptr(status),
                               _ptr(workspace), workspace.numel(), _stream_ptr(dev))
    _lib.check(rc)
    res = (shift, theta, energy, iters, status)
    return res + (g,) if gamma else res


def align_curves_host(pts: torch.Tensor, offsets: torch.Tensor, N: int, *, method: str = "fft",
                      prec: str = "fp64", fp32_storage: bool = False, out: tuple | None = None,
                      device: int | None = None):
    """Resample 2P raw curves to N nodes and align curve p with curve P+p,
    from host buffers to host buffers (fa_align_curves_host).

    pts: complex128 CPU tensor (pinned memory for asynchronous copies);
    offsets: int64 CPU tensor [2P+1].  Returns CPU tensors (shift, theta,
    energy, status) of P entries; blocks until they are filled.
    """
    if pts.is_cuda or offsets.is_cuda:
        raise ValueError("align_curves_host takes host (CPU) tensors")
    if pts.dtype != torch.complex128 or offsets.dtype != torch.int64:
        raise ValueError("pts must be complex128 and offsets int64")
    C = offsets.numel() - 1
    if C % 2:
        raise ValueError("offsets must describe an even number of curves (2P)")
    P = C // 2
    if out is None:
        pin = torch.cuda.is_available()
        shift = torch.empty(P, dtype=torch.int32, pin_memory=pin)
        theta = torch.empty(P, dtype=torch.float64, pin_memory=pin)
        energy = torch.empty(P, dtype=torch.float64, pin_memory=pin)
        status = torch.empty(P, dtype=torch.int8, pin_memory=pin)
    else:
        shift, theta, energy, status = out
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    L = _lib.load()
    h = handle(dev.index)
    flags = _lib.STORE_FP32 if fp32_storage else 0
    rc = L.fa_align_curves_host(h, _ptr(pts), _ptr(offsets), P, N, flags, _METHODS[method],
                                _PRECS[prec], _ptr(shift), _ptr(theta), _ptr(energy),
                                _ptr(status), _stream_ptr(dev))
    _lib.check(rc)
    return shift, theta, energy, status


# ------------------------------------------------ k-NN retrieval helpers ----
def fourier_descriptors(z: torch.Tensor, F: int = 32) -> torch.Tensor:
    """log |Z[+-f]|, f = 1..F, of uniformly resampled curves z [M, N]
    (complex128 CUDA) -> float32 [M, 2F] (fa_fourier_descriptors)."""
    _need_cuda("z", z, torch.complex128)
    M, N = z.shape
    out = torch.empty((M, 2 * F), dtype=torch.float32, device=z.device)
    _lib.check(_lib.load().fa_fourier_descriptors(handle(z.device.index), _ptr(z), M, N, F,
                                                  _ptr(out), _stream_ptr(z.device)))
    return out


def column_stats(X: torch.Tensor):
    _need_cuda("X", X, torch.float32)
    M, D = X.shape
    mean = torch.empty(D, dtype=torch.float32, device=X.device)
    inv = torch.empty(D, dtype=torch.float32, device=X.device)
    _lib.check(_lib.load().fa_column_stats(handle(X.device.index), _ptr(X), M, D, _ptr(mean),
                                           _ptr(inv), _stream_ptr(X.device)))
    return mean, inv


def standardize_(X: torch.Tensor, mean: torch.Tensor, inv_std: torch.Tensor) -> torch.Tensor:
    _need_cuda("X", X, torch.float32)
    M, D = X.shape
    _lib.check(_lib.load().fa_standardize(handle(X.device.index), _ptr(X), M, D, _ptr(mean),
                                          _ptr(inv_std), _stream_ptr(X.device)))
    return X


def embed_sqdist(A: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
    _need_cuda("A", A, torch.float32)
    _need_cuda("B", B, torch.float32)
    Q, D = A.shape
    G = B.shape[0]
    out = torch.empty((Q, G), dtype=torch.float32, device=A.device)
    _lib.check(_lib.load().fa_embed_sqdist(handle(A.device.index), _ptr(A), Q, _ptr(B), G, D,
                                           _ptr(out), _stream_ptr(A.device)))
    return out


def select_k(keys: torch.Tensor, k: int, with_keys: bool = False):
    """Positions of the k smallest keys per row, ascending by (key, position)."""
    if keys.dtype not in (torch.float32, torch.float64):
        raise ValueError("keys must be float32 or float64")
    _need_cuda("keys", keys, keys.dtype)
    rows, C = keys.shape
    pos = torch.empty((rows, k), dtype=torch.int64, device=keys.device)
    kv = torch.empty((rows, k), dtype=keys.dtype, device=keys.device) if with_keys else None
    kt = _lib.KEY_F32 if keys.dtype == torch.float32 else _lib.KEY_F64
    _lib.check(_lib.load().fa_select_k(handle(keys.device.index), _ptr(keys), kt, rows, C, k,
                                       _ptr(pos), _ptr(kv), _stream_ptr(keys.device)))
    return (pos, kv) if with_keys else pos


class Mlp:
    """The pruning network (fa_mlp_*): 64 -> 256 -> 256 -> 64, bfloat16 weights."""

    def __init__(self, seed: int = 0, device: int | None = None):
        self._L = _lib.load()
        self._h = handle(device)
        self.device = torch.device("cuda", device if device is not None else torch.cuda.current_device())
        p = ctypes.c_void_p()
        _lib.check(self._L.fa_mlp_create(self._h, seed, ctypes.byref(p)))
        self._m = p.value
        self.n_params = int(self._L.fa_mlp_num_params())

    def close(self):
        if self._m:
            self._L.fa_mlp_destroy(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        import numpy as np
        out = np.empty(self.n_params, np.float32)
        _lib.check(self._L.fa_mlp_get_params(self._m, out.ctypes.data))
        return out

    def set_params(self, params):
        import numpy as np
        p = np.ascontiguousarray(params, np.float32)
        assert p.size == self.n_params
        _lib.check(self._L.fa_mlp_set_params(self._m, p.ctypes.data))

    def forward(self, X: torch.Tensor) -> torch.Tensor:
        _need_cuda("X", X, torch.float32)
        B = X.shape[0]
        Y = torch.empty((B, 64), dtype=torch.float32, device=X.device)
        _lib.check(self._L.fa_mlp_forward(self._m, _ptr(X), B, _ptr(Y), _stream_ptr(X.device)))
        return Y

    def pair_grad(self, X, pi, pj, d, grad: bool = False):
        _need_cuda("X", X, torch.float32)
        _need_cuda("pi", pi, torch.int64)
        _need_cuda("pj", pj, torch.int64)
        _need_cuda("d", d, torch.float32)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        g = torch.empty(self.n_params, dtype=torch.float32, device=X.device) if grad else None
        _lib.check(self._L.fa_mlp_pair_grad(self._m, _ptr(X), X.shape[0], _ptr(pi), _ptr(pj),
                                            _ptr(d), pi.numel(), _ptr(loss), _ptr(g),
                                            _stream_ptr(X.device)))
        return (loss, g) if grad else loss

    def adam_step(self, lr: float):
        _lib.check(self._L.fa_mlp_adam_step(self._m, float(lr), _stream_ptr(self.device)))
