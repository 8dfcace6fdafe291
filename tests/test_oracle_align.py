"""Pins for oracle O1 (rigid alignment by exhaustive search, Algorithms 1-2).

Every check here compares the oracle with something other than itself: a
library SVD, brute-force minimisation over the rotation angle, closed forms
for the circle and the ellipse, values fixed by construction (the paper's
start-point/rotation template), and invariances of the energy.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2501_17779_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _unit(z):
    z = z - z.mean()
    return z / np.abs(np.roll(z, -1) - z).sum()


# ---------------------------------------------------------------- 2x2 SVD ---
@pytest.mark.parametrize("seed", range(20))
def test_svd2x2_matches_numpy(seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(2, 2))
    if seed % 5 == 1:
        A[:, 1] = 3.0 * A[:, 0]          # rank one
    if seed % 5 == 2:
        A = np.diag([2.0, -0.5])         # negative determinant
    if seed % 5 == 3:
        A = np.zeros((2, 2))
    U, S, V = oracle.svd2x2(A)
    np.testing.assert_allclose(S, np.linalg.svd(A, compute_uv=False), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(U @ np.diag(S) @ V.T, A, atol=1e-14)
    np.testing.assert_allclose(U.T @ U, np.eye(2), atol=1e-14)
    np.testing.assert_allclose(V.T @ V, np.eye(2), atol=1e-14)
    assert S[0] >= S[1] >= 0.0


@pytest.mark.parametrize("seed", range(20))
def test_kabsch_is_the_best_proper_rotation(seed):
    """Algorithm 1's R is a proper rotation and attains the maximum of
    tr(R(phi) A^T) over a dense grid of angles (brute force, no SVD)."""
    rng = np.random.default_rng(100 + seed)
    A = rng.normal(size=(2, 2))
    if seed % 4 == 0:
        A[1] = -A[1]
    R, tr = oracle.kabsch(A)
    assert abs(np.linalg.det(R) - 1.0) < 1e-14
    np.testing.assert_allclose(R.T @ R, np.eye(2), atol=1e-14)
    phi = np.linspace(-np.pi, np.pi, 200001)
    c, s = np.cos(phi), np.sin(phi)
    # R(phi) = [[c, -s], [s, c]]; tr(R A^T) = sum_ij R_ij A_ij
    vals = c * A[0, 0] - s * A[0, 1] + s * A[1, 0] + c * A[1, 1]
    assert tr >= vals.max() - 1e-12
    assert tr <= vals.max() + 1e-9
    # the complex form: the maximum over SO(2) is |(A11 + A22) + i(A21 - A12)|
    assert abs(tr - abs(complex(A[0, 0] + A[1, 1], A[1, 0] - A[0, 1]))) < 1e-14


# ----------------------------------------------------- golden fixtures -----
def test_golden_delta_n4():
    g = json.load(open(os.path.join(GOLDEN, "delta_n4.json")))
    z1 = np.array([complex(*p) for p in g["z1"]])
    z2 = np.array([complex(*p) for p in g["z2"]])
    np.testing.assert_allclose(oracle.shift_scores(z1, z2), g["expected_scores"], atol=1e-15)
    o = oracle.align_pairs(z1, z2)
    assert o["shift"][0] == g["expected_shift"]
    assert abs(o["theta"][0] - g["expected_theta"]) < 1e-15
    assert abs(o["energy"][0] - g["expected_energy"]) < 1e-15
    assert abs(o["gap"][0] - g["expected_gap"]) < 1e-15


def test_golden_template_protocol():
    """Sec. 2's template: start point 0 -> 0.25 and rotation pi/3, zero energy."""
    g = json.load(open(os.path.join(GOLDEN, "template_protocol.json")))
    rng = np.random.default_rng(7)
    for N in g["N"]:
        h = synth.random_harmonics(rng, 8)
        z1, z2 = synth.template_pair(h, N, g["start"], g["rotation"])
        o = oracle.align_pairs(z1, z2)
        assert o["shift"][0] == round(g["expected_shift_fraction"] * N)
        assert abs(o["theta"][0] - g["expected_theta"]) < g["theta_atol"]
        assert abs(o["energy"][0] - g["expected_energy"]) < g["energy_atol"]


# ------------------------------------------------------- self alignment ----
def test_self_alignment_exact_recovery():
    ap = synth.aligned_pairs(1001, P=32, N=256, noise=0.0)
    o = oracle.align_pairs(ap.z1, ap.z2)
    np.testing.assert_array_equal(o["shift"], ap.shift_true)
    d = np.angle(np.exp(1j * (o["theta"] - ap.theta_true)))
    assert np.abs(d).max() < 1e-13
    assert o["energy"].max() < 1e-15
    assert (o["status"] == 0).all()


# ----------------------------------------------------------- closed forms ---
@pytest.mark.parametrize("N", [16, 64, 256])
def test_circle_closed_form(N):
    """z1 = r e^{2 pi i k/N}, z2 = e^{i a} z1: |c(s)| = N r^2 for all s, so
    every shift is optimal with zero energy (rounding picks one of them) and
    the angle at shift s is arg c(s) = -a - 2 pi s / N."""
    a = 0.7
    z1 = _unit(np.exp(2j * np.pi * np.arange(N) / N))
    r = abs(z1[0])
    z2 = np.exp(1j * a) * z1
    np.testing.assert_allclose(oracle.shift_scores(z1, z2), N * r * r, rtol=1e-13)
    o = oracle.align_pairs(z1, z2)
    s = int(o["shift"][0])
    assert 0 <= s < N
    assert abs(np.angle(np.exp(1j * (o["theta"][0] + a + 2 * np.pi * s / N)))) < 1e-13
    assert o["energy"][0] < 1e-16
    assert o["gap"][0] < 1e-15


@pytest.mark.parametrize("N", [16, 64, 256])
def test_ellipse_closed_form_whole_vector(N):
    """z[k] = a cos(phi_k) + i b sin(phi_k) = A e^{i phi_k} + B e^{-i phi_k}
    with A = (a+b)/2, B = (a-b)/2, phi_k = 2 pi k / N.  Against itself,
    c(s) = N (A^2 e^{-i phi_s} + B^2 e^{i phi_s}) for N > 2, so
    |c(s)|^2 = N^2 (A^4 + B^4 + 2 A^2 B^2 cos 2 phi_s).  Exact tie between
    s = 0 (angle 0) and s = N/2 (angle pi); rounding picks one of them."""
    a, b = 1.3, 0.6
    phi = 2 * np.pi * np.arange(N) / N
    z = a * np.cos(phi) + 1j * b * np.sin(phi)
    A, B = (a + b) / 2, (a - b) / 2
    expect = N * np.sqrt(A**4 + B**4 + 2 * A * A * B * B * np.cos(2 * phi))
    np.testing.assert_allclose(oracle.shift_scores(z, z), expect, rtol=1e-13)
    o = oracle.align_pairs(z, z)
    s = int(o["shift"][0])
    assert s in (0, N // 2)
    assert o["gap"][0] < 1e-13           # the s = 0 / s = N/2 tie
    want = 0.0 if s == 0 else np.pi
    assert abs(np.angle(np.exp(1j * (o["theta"][0] - want)))) < 1e-13
    assert o["energy"][0] < 1e-15


# -------------------------------------------------------------- brute force -
def _brute_energy(z1, z2, s):
    """min over theta of h sum |z1[k] - e^{i theta} z2[k+s]|^2 by a dense grid
    plus golden-section refinement (no Kabsch, no SVD)."""
    N = z1.size
    w = np.roll(z2, -s)
    f = lambda th: np.sum(np.abs(z1 - np.exp(1j * th) * w) ** 2) / N
    grid = np.linspace(-np.pi, np.pi, 100001)
    vals = np.concatenate([np.sum(np.abs(z1[None] - np.exp(1j * t)[:, None] * w[None]) ** 2, axis=1)
                           for t in np.array_split(grid, 50)]) / N
    i = int(np.argmin(vals))
    lo, hi = grid[max(i - 1, 0)], grid[min(i + 1, grid.size - 1)]
    gr = (np.sqrt(5) - 1) / 2
    for _ in range(80):
        m1, m2 = hi - gr * (hi - lo), lo + gr * (hi - lo)
        if f(m1) < f(m2):
            hi = m2
        else:
            lo = m1
    th = 0.5 * (lo + hi)
    return f(th), th


@pytest.mark.parametrize("N,seed", [(5, 0), (8, 1), (12, 2), (16, 3)])
def test_bruteforce_small_n(N, seed):
    rng = np.random.default_rng(seed)
    z1 = _unit(rng.normal(size=N) + 1j * rng.normal(size=N))
    z2 = _unit(rng.normal(size=N) + 1j * rng.normal(size=N))
    scores = oracle.shift_scores(z1, z2)
    h = 1.0 / N
    E_or = h * (np.sum(np.abs(z1) ** 2) + np.sum(np.abs(z2) ** 2) - 2 * scores)
    brute = [_brute_energy(z1, z2, s) for s in range(N)]
    E_bf = np.array([b[0] for b in brute])
    np.testing.assert_allclose(E_or, E_bf, atol=1e-13)
    o = oracle.align_pairs(z1, z2)
    s = int(np.argmin(E_bf))
    assert o["shift"][0] == s
    assert abs(o["energy"][0] - E_bf[s]) < 1e-13
    assert abs(np.angle(np.exp(1j * (o["theta"][0] - brute[s][1])))) < 1e-7


# ------------------------------------------------------------- invariances --
def test_invariances():
    ap = synth.aligned_pairs(77, P=4, N=128, noise=2e-3)
    base = oracle.align_pairs(ap.z1, ap.z2)
    # rotating curve 1 by b changes theta by +b, nothing else
    b = 0.9
    rot = oracle.align_pairs(np.exp(1j * b) * ap.z1, ap.z2)
    np.testing.assert_array_equal(rot["shift"], base["shift"])
    np.testing.assert_allclose(np.angle(np.exp(1j * (rot["theta"] - base["theta"] - b))), 0,
                               atol=1e-12)
    np.testing.assert_allclose(rot["energy"], base["energy"], rtol=1e-10)
    # relabelling curve 2 cyclically by q moves the shift by +q
    q = 17
    rel = oracle.align_pairs(ap.z1, np.roll(ap.z2, q, axis=1))
    np.testing.assert_array_equal(rel["shift"], (base["shift"] + q) % 128)
    np.testing.assert_allclose(rel["energy"], base["energy"], rtol=1e-10)
    # swapping the curves: s -> -s mod N, theta -> -theta, same energy
    sw = oracle.align_pairs(ap.z2, ap.z1)
    np.testing.assert_array_equal(sw["shift"], (-base["shift"]) % 128)
    np.testing.assert_allclose(np.angle(np.exp(1j * (sw["theta"] + base["theta"]))), 0, atol=1e-12)
    np.testing.assert_allclose(sw["energy"], base["energy"], rtol=1e-10)


def test_nonfinite_input_status():
    ap = synth.aligned_pairs(5, P=3, N=32)
    z2 = ap.z2.copy()
    z2[1, 3] = np.nan
    o = oracle.align_pairs(ap.z1, z2)
    assert list(o["status"]) == [0, 2, 0]
    assert o["shift"][1] == -1 and np.isnan(o["energy"][1])
