"""ctypes binding of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's CPU
baseline leg are the only callers.  The oracle shares no code with the CUDA
library (paper_2501_17779_gb300/) and neither side imports the other.

The oracle is the plain definition of the method's result: the O(N^2) search
over all cyclic start points with a Kabsch solve per shift (Algorithm 1 inside
the loop of Algorithm 2, with A(s) from Eq. A-mtx instead of FFTs), the
periodic-cubic-spline arc-length resampling of Sec. 2, and the elastic shape
distance of Sec. 3 (SRV functions, Eq. dist2-energy, the alternation of
"Approach 2" with a lattice-path dynamic programme as its gamma-step).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "oracle.c"
_LIB = _HERE / "_build" / "liboracle.so"

CENTER = 1
UNIT_LENGTH = 2

ST_OK, ST_DEGENERATE, ST_NONFINITE = 0, 1, 2

_lib = None


def build(force: bool = False) -> Path:
    """Compile oracle.c into oracle/_build/liboracle.so with gcc (OpenMP).

    Floating-point contraction is disabled so that the oracle rounds the same
    way on every host (no fused multiply-add substitutions)."""
    if _LIB.exists() and not force and _LIB.stat().st_mtime >= _SRC.stat().st_mtime:
        return _LIB
    _LIB.parent.mkdir(exist_ok=True)
    tmp = _LIB.with_suffix(f".so.{os.getpid()}")
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", str(tmp), str(_SRC), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(_LIB))
        dp = ctypes.POINTER(ctypes.c_double)
        L.oracle_svd2x2.argtypes = [dp, dp, dp, dp]
        L.oracle_kabsch.argtypes = [dp, dp]
        L.oracle_kabsch.restype = ctypes.c_double
        L.oracle_shift_scores.argtypes = [dp, dp, ctypes.c_int, dp]
        L.oracle_align_pairs.argtypes = [dp, dp, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p, dp, dp, dp, ctypes.c_void_p]
        L.oracle_resample.argtypes = [dp, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, dp, ctypes.c_void_p]
        L.oracle_max_threads.restype = ctypes.c_int
        vp = ctypes.c_void_p
        L.oracle_elastic_pairs.argtypes = [dp, dp, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, vp, dp, dp, vp, vp, vp, vp]
        L.oracle_elastic_from_start.argtypes = [dp, dp, ctypes.c_int64, ctypes.c_int, vp, dp, dp,
                                                ctypes.c_int, ctypes.c_int, vp, dp, dp, vp, vp, vp]
        for nm, extra in (("oracle_elastic_dp", [ctypes.c_int, dp]),
                          ("oracle_elastic_refine", [ctypes.c_int, dp, dp, ctypes.c_int]),
                          ("oracle_elastic_energy", [dp])):
            f = getattr(L, nm)
            f.argtypes = [dp, dp, ctypes.c_int] + extra
            f.restype = ctypes.c_double
        L.oracle_srv.argtypes = [dp, ctypes.c_int, dp, dp]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def svd2x2(A) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """2x2 SVD A = U diag(S) V^T (S descending)."""
    A = np.ascontiguousarray(A, np.float64).reshape(4)
    U, S, V = np.empty(4), np.empty(2), np.empty(4)
    _load().oracle_svd2x2(_dp(A), _dp(U), _dp(S), _dp(V))
    return U.reshape(2, 2), S, V.reshape(2, 2)


def kabsch(A) -> tuple[np.ndarray, float]:
    """Algorithm 1: the proper rotation R maximising tr(R A^T), and that trace."""
    A = np.ascontiguousarray(A, np.float64).reshape(4)
    R = np.empty(4)
    tr = _load().oracle_kabsch(_dp(A), _dp(R))
    return R.reshape(2, 2), float(tr)


def shift_scores(z1, z2) -> np.ndarray:
    """tr(R(s) A(s)^T) for every shift s of one pair (complex inputs)."""
    z1 = np.ascontiguousarray(z1, np.complex128)
    z2 = np.ascontiguousarray(z2, np.complex128)
    N = z1.size
    out = np.empty(N)
    rc = _load().oracle_shift_scores(_dp(z1.view(np.float64)), _dp(z2.view(np.float64)), N,
                                     _dp(out))
    if rc != 0:
        raise ValueError("oracle_shift_scores: bad arguments")
    return out


def align_pairs(z1, z2, nthreads: int | None = None) -> dict:
    """O1 on P pairs of complex [P, N] arrays.

    Returns shift (int32), theta (CCW angle applied to curve 2), energy (direct
    Eq. disc-energy at the winner), gap (energy of the runner-up shift minus
    the winner's) and status (0 ok, 2 non-finite input)."""
    z1 = np.ascontiguousarray(z1, np.complex128)
    z2 = np.ascontiguousarray(z2, np.complex128)
    if z1.ndim == 1:
        z1, z2 = z1[None], z2[None]
    P, N = z1.shape
    assert z2.shape == (P, N)
    out = dict(shift=np.empty(P, np.int32), theta=np.empty(P), energy=np.empty(P),
               gap=np.empty(P), status=np.empty(P, np.int8))
    nt = nthreads if nthreads is not None else (os.cpu_count() or 1)
    rc = _load().oracle_align_pairs(_dp(z1.view(np.float64)), _dp(z2.view(np.float64)), P, N,
                                    nt, out["shift"].ctypes.data, _dp(out["theta"]),
                                    _dp(out["energy"]), _dp(out["gap"]),
                                    out["status"].ctypes.data)
    if rc != 0:
        raise ValueError("oracle_align_pairs: bad arguments")
    return out


def resample(pts, offsets, N: int, flags: int = CENTER | UNIT_LENGTH,
             nthreads: int | None = None) -> tuple[np.ndarray, np.ndarray]:
    """O2 on C ragged curves given as CSR (complex pts, int64 offsets[C+1]).

    Returns (z complex128 [C, N], status int8 [C])."""
    pts = np.ascontiguousarray(pts, np.complex128)
    offsets = np.ascontiguousarray(offsets, np.int64)
    C = offsets.size - 1
    z = np.empty((C, N), np.complex128)
    st = np.empty(C, np.int8)
    nt = nthreads if nthreads is not None else (os.cpu_count() or 1)
    rc = _load().oracle_resample(_dp(pts.view(np.float64)), offsets.ctypes.data, C, N, flags, nt,
                                 _dp(z.view(np.float64)), st.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_resample: bad arguments")
    return z, st


def _c128(a):
    return np.ascontiguousarray(a, np.complex128)


def elastic_pairs(b1, b2, band: int = -1, max_iter: int = 20, nthreads: int | None = None,
                  gamma: bool = False, trace: bool = False) -> dict:
    """O3 on P pairs of N-node closed curves (complex [P, N] each, node k at
    parameter k/N).  band < 0 searches the full lattice.

    Returns shift s (t0 = s/N, applied to curve 1), theta (CCW rotation of
    curve 1), energy (Eq. dist2-energy of the final triple), dist = sqrt(energy),
    iters (iterations run), status, and optionally gamma ([P, N+1], the node
    values g_k = N gamma(k/N)) and trace ([P, max_iter], the energy after each
    iteration)."""
    b1, b2 = _c128(b1), _c128(b2)
    if b1.ndim == 1:
        b1, b2 = b1[None], b2[None]
    P, N = b1.shape
    assert b2.shape == (P, N)
    out = dict(shift=np.empty(P, np.int32), theta=np.empty(P), energy=np.empty(P),
               iters=np.empty(P, np.int32), status=np.empty(P, np.int8))
    g = np.empty((P, N + 1)) if gamma else None
    t = np.empty((P, max_iter)) if trace else None
    nt = nthreads if nthreads is not None else (os.cpu_count() or 1)
    rc = _load().oracle_elastic_pairs(
        _dp(b1.view(np.float64)), _dp(b2.view(np.float64)), P, N, band, max_iter, nt,
        out["shift"].ctypes.data, _dp(out["theta"]), _dp(out["energy"]),
        out["iters"].ctypes.data, out["status"].ctypes.data,
        g.ctypes.data if gamma else None, t.ctypes.data if trace else None)
    if rc != 0:
        raise ValueError("oracle_elastic_pairs: bad arguments")
    out["dist"] = np.sqrt(np.maximum(out["energy"], 0.0))
    if gamma:
        out["gamma"] = g
    if trace:
        out["trace"] = t
    return out


def elastic_from_start(b1, b2, shift0, theta0, g0, max_iter: int = 20,
                       nthreads: int | None = None) -> dict:
    """The alternation of O3 alone, started from a given triple per pair
    (shift0 [P], theta0 [P], g0 [P, N+1]) instead of the pre-alignment and the
    lattice programme: refinement and (t0,R)-steps until an iteration lowers
    the energy by at most 1e-12, or max_iter.  Returns the same keys as
    elastic_pairs (gamma included)."""
    b1, b2 = _c128(b1), _c128(b2)
    if b1.ndim == 1:
        b1, b2 = b1[None], b2[None]
    P, N = b1.shape
    s0 = np.ascontiguousarray(shift0, np.int32)
    t0 = np.ascontiguousarray(theta0, np.float64)
    g0 = np.ascontiguousarray(g0, np.float64)
    assert s0.shape == (P,) and t0.shape == (P,) and g0.shape == (P, N + 1)
    out = dict(shift=np.empty(P, np.int32), theta=np.empty(P), energy=np.empty(P),
               iters=np.empty(P, np.int32), status=np.empty(P, np.int8))
    g = np.empty((P, N + 1))
    nt = nthreads if nthreads is not None else (os.cpu_count() or 1)
    rc = _load().oracle_elastic_from_start(
        _dp(b1.view(np.float64)), _dp(b2.view(np.float64)), P, N, s0.ctypes.data, _dp(t0),
        _dp(g0), max_iter, nt, out["shift"].ctypes.data, _dp(out["theta"]),
        _dp(out["energy"]), out["iters"].ctypes.data, out["status"].ctypes.data, g.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_elastic_from_start: bad arguments")
    out["dist"] = np.sqrt(np.maximum(out["energy"], 0.0))
    out["gamma"] = g
    return out


def elastic_dp(q1s, q2, band: int = -1) -> tuple[np.ndarray, float]:
    """The lattice dynamic programme alone: node values g [N+1] of the
    minimising path for fixed SRV samples q1s, q2 (complex [N]), and its energy."""
    q1s, q2 = _c128(q1s), _c128(q2)
    N = q1s.size
    g = np.empty(N + 1)
    e = _load().oracle_elastic_dp(_dp(q1s.view(np.float64)), _dp(q2.view(np.float64)), N, band,
                                  _dp(g))
    return g, float(e)


def elastic_refine(q1, q2, s: int, theta: float, g, iters: int = 16):
    """The continuous refinement alone (node values g and the angle theta, for
    the fixed shift s of q1); returns (g, theta, energy)."""
    q1, q2 = _c128(q1), _c128(q2)
    g = np.array(g, np.float64)
    th = np.array([theta], np.float64)
    e = _load().oracle_elastic_refine(_dp(q1.view(np.float64)), _dp(q2.view(np.float64)),
                                      q1.size, s, _dp(th), _dp(g), iters)
    return g, float(th[0]), float(e)


def elastic_energy(q1s, q2, g) -> float:
    """Eq. dist2-energy (midpoint rule) of node values g for fixed q1s, q2."""
    q1s, q2 = _c128(q1s), _c128(q2)
    g = np.ascontiguousarray(g, np.float64)
    return float(_load().oracle_elastic_energy(_dp(q1s.view(np.float64)),
                                               _dp(q2.view(np.float64)), q1s.size, _dp(g)))


def srv(beta) -> tuple[np.ndarray, np.ndarray, int]:
    """SRV samples q (complex [N]) of the unit-length polygon through beta's
    nodes (at the cell midpoints), the cumulative chord-length fractions
    sigma [N+1] and the status."""
    beta = _c128(beta)
    N = beta.size
    q = np.empty(N, np.complex128)
    sg = np.empty(N + 1)
    st = _load().oracle_srv(_dp(beta.view(np.float64)), N, _dp(q.view(np.float64)), _dp(sg))
    if st < 0:
        raise ValueError("oracle_srv: bad arguments")
    return q, sg, int(st)
