"""Pins of the elastic-distance oracle (Sec. 3) to facts outside itself:
the unit-norm property of SRV functions, the continuous energy of
Eq. dist2-energy (second-order convergence of its discretisation), brute
force over all lattice paths, stationarity of the refinement, exact zero
distance under rigid motions and the zero-distance experiment of Table 2."""
import itertools
import json
from math import gcd
from pathlib import Path

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2501_17779_gb300 import synth

GOLD = Path(__file__).parent / "golden"
STEPS = [(a, b) for a in range(1, 4) for b in range(1, 4) if gcd(a, b) == 1]


def _curve(seed, N, n_harm=6):
    h = synth.random_harmonics(np.random.default_rng(seed), n_harm)
    return synth.uniform_arclength_nodes(h, N)


def test_srv_unit_norm_and_circle():
    """Sec. 3: a unit-length curve has ||q|| = 1; for a regular polygon
    (a sampled circle) |q| is constant and q turns by 2 pi / N per node."""
    for seed in range(4):
        b = _curve(seed, 200) * 3.7 + (0.3 - 2j)
        q, sg, st = oracle.srv(b)
        assert st == 0
        assert abs(np.mean(np.abs(q) ** 2) - 1.0) < 1e-14
        assert sg[0] == 0.0 and abs(sg[-1] - 1.0) < 1e-15 and (np.diff(sg) > 0).all()
    N = 64
    c = np.exp(2j * np.pi * np.arange(N) / N)
    q, _, _ = oracle.srv(c)
    np.testing.assert_allclose(np.abs(q), 1.0, atol=1e-14)
    np.testing.assert_allclose(q[1:] / q[:-1], np.exp(2j * np.pi / N), atol=1e-14)


def test_srv_status():
    b = _curve(1, 32)
    b[5] = np.nan
    assert oracle.srv(b)[2] == 2
    assert oracle.srv(np.zeros(16, complex))[2] == 1


def _Q1(t):
    return np.exp(2j * np.pi * t) * (1.0 + 0.3 * np.cos(4 * np.pi * t)) + 0.2 * np.exp(-6j * np.pi * t)


def _Q2(u):
    return (0.9 + 0.25 * np.sin(2 * np.pi * u)) * np.exp(2j * np.pi * u + 0.4j)


def _gam(t):
    return t + 0.06 * np.sin(2 * np.pi * t)


def _dgam(t):
    return 1.0 + 0.12 * np.pi * np.cos(2 * np.pi * t)


def test_energy_converges_to_the_integral():
    """The midpoint-rule energy of sampled smooth q1, q2 and gamma tends to the
    integral of Eq. dist2-energy (computed by adaptive quadrature from the
    functions themselves) at second order."""
    def f(t):
        d = _Q1(t) - np.sqrt(_dgam(t)) * _Q2(_gam(t))
        return abs(d) ** 2
    exact = integrate.quad(f, 0.0, 1.0, limit=200, epsabs=1e-14, epsrel=1e-13)[0]
    errs = []
    for N in (64, 128, 256, 512):
        mid = (np.arange(N) + 0.5) / N
        g = N * _gam(np.arange(N + 1) / N)
        E = oracle.elastic_energy(_Q1(mid), _Q2(mid), g)
        errs.append(abs(E - exact))
    errs = np.array(errs)
    assert exact > 0.1
    assert (errs[:-1] / errs[1:] > 3.5).all(), errs
    assert errs[-1] < 2e-4 * exact


def _paths(N, band):
    """All lattice paths (0,0) -> (N,N) with the steps above, vertices in the band."""
    out = []

    def rec(i, j, acc):
        if i == N and j == N:
            out.append(list(acc))
            return
        for a, b in STEPS:
            i2, j2 = i + a, j + b
            if i2 <= N and j2 <= N and (band < 0 or abs(i2 - j2) <= band):
                acc.append((a, b))
                rec(i2, j2, acc)
                acc.pop()
    rec(0, 0, [])
    return out


def _g_of(path, N):
    g = np.empty(N + 1)
    i = j = 0
    for a, b in path:
        for p in range(a):
            g[i + p] = j + p * b / a
        i, j = i + a, j + b
    g[N] = N
    return g


@pytest.mark.parametrize("N,band", [(5, -1), (6, -1), (7, 1), (7, -1), (8, 2)])
def test_dp_equals_brute_force(N, band):
    rng = np.random.default_rng(N * 10 + band)
    q1s = rng.normal(size=N) + 1j * rng.normal(size=N)
    q2 = rng.normal(size=N) + 1j * rng.normal(size=N)
    best = min((oracle.elastic_energy(q1s, q2, _g_of(p, N)), i)
               for i, p in enumerate(_paths(N, band)))
    g, E = oracle.elastic_dp(q1s, q2, band)
    assert abs(E - best[0]) <= 1e-13 * max(1.0, best[0])
    assert abs(oracle.elastic_energy(q1s, q2, g) - E) <= 1e-13 * max(1.0, E)


def test_refinement_reaches_a_stationary_point():
    """From the dynamic programme's path the refinement lowers the energy and
    ends where the finite-difference gradient in (g_0..g_{N-1}, theta) has
    collapsed (g_N = g_0 + N moves with g_0)."""
    N = 64
    q1, _, _ = oracle.srv(_curve(21, N))
    q2, _, _ = oracle.srv(_curve(22, N))
    g0, E0 = oracle.elastic_dp(q1, q2)
    g, th, E = oracle.elastic_refine(q1, q2, 0, 0.0, g0, iters=200)
    assert E < E0 and np.all(np.diff(g) > 0) and abs(g[N] - g[0] - N) < 1e-12

    def energy(gv, t):
        return oracle.elastic_energy(np.exp(1j * t) * q1, q2, gv)

    def grad(gv, t, h=1e-7):
        out = []
        for k in range(N):
            e = np.zeros(N + 1)
            e[k] = h
            if k == 0:
                e[N] = h
            out.append((energy(gv + e, t) - energy(gv - e, t)) / (2 * h))
        out.append((energy(gv, t + h) - energy(gv, t - h)) / (2 * h))
        return np.array(out)
    assert abs(energy(g, th) - E) < 1e-15
    g_start = np.linalg.norm(grad(g0, 0.0))
    g_end = np.linalg.norm(grad(g, th))
    assert g_end < 1e-5 * g_start, (g_start, g_end)


def test_zero_distance_under_rigid_motion():
    """beta2[k] = e^{i phi} beta1[k + m]: distance 0, s = m, theta = phi
    (the motion acts on curve 1); translation and scale do not matter."""
    N = 128
    b1 = _curve(5, N)
    for m, phi in [(0, 0.0), (17, 2.5), (100, -1.0)]:
        b2 = np.exp(1j * phi) * np.roll(b1, -m) * 2.5 + (1 - 3j)
        r = oracle.elastic_pairs(b1, b2, trace=True)
        assert r["status"][0] == 0 and r["shift"][0] == m
        assert abs(np.angle(np.exp(1j * (r["theta"][0] - phi)))) < 1e-12
        assert r["energy"][0] < 1e-26 and r["iters"][0] <= 2


@pytest.mark.parametrize("which", ["gamma1", "gamma2"])
def test_table2_zero_distance_experiment(which):
    """Table 2 (Approach 2): the distance to a start-shifted, rotated and
    reparameterised copy vanishes with N."""
    gold = json.loads((GOLD / "elastic_table2.json").read_text())
    gam = synth.gamma_paper_1 if which == "gamma1" else synth.gamma_paper_2
    h = synth.random_harmonics(np.random.default_rng(3), 6)
    d = []
    for N in gold["N"]:
        b1, b2 = synth.reparam_pair(h, N, gam, gold["start"], gold["rotation"])
        r = oracle.elastic_pairs(b1, b2, trace=True)
        assert r["status"][0] == 0 and r["shift"][0] == round(gold["start"] * N)
        tr = r["trace"][0][: r["iters"][0]]
        assert (np.diff(tr) <= 1e-15).all()
        d.append(r["dist"][0])
    d = np.array(d)
    assert d[0] < gold["max_distance_at_64"] and d[-1] < gold["max_distance_at_1024"]
    ratio = d[:-1] / d[1:]
    assert (ratio > gold["min_ratio_per_doubling"]).all(), d
    assert (ratio[2:] > gold["min_ratio_per_doubling_from_256"]).all(), d
    assert abs(r["theta"][0] - gold["rotation"]) < gold["theta_atol_at_1024"]
    # far below what a slope-limited dynamic programme alone reaches
    assert d[-1] < 0.01 * gold["paper_approach1_distance_gamma1"][3]


def test_elastic_distance_properties():
    """On distinct curves: the distance is below the energy of the
    pre-aligned, unreparameterised pair (the first iterate starts there), the
    energy trace never increases, a band that holds the optimal path changes
    nothing, and statuses flag bad inputs."""
    P, N = 6, 96
    b1 = np.stack([_curve(40 + p, N, 8) for p in range(P)])
    b2 = np.stack([_curve(60 + p, N, 8) for p in range(P)])
    r = oracle.elastic_pairs(b1, b2, trace=True, gamma=True)
    assert (r["status"] == 0).all()
    for p in range(P):
        tr = r["trace"][p][: r["iters"][p]]
        assert (np.diff(tr) <= 1e-15).all() and abs(tr[-1] - r["energy"][p]) < 1e-15
        g = r["gamma"][p]
        assert (np.diff(g) > 0).all() and abs(g[-1] - g[0] - N) < 1e-9
        q1, _, _ = oracle.srv(b1[p])
        q2, _, _ = oracle.srv(b2[p])
        rigid = min(oracle.elastic_energy(np.exp(1j * t) * np.roll(q1, -s), q2,
                                          np.arange(N + 1.0))
                    for s in range(N) for t in np.linspace(-np.pi, np.pi, 73))
        assert r["energy"][p] < rigid
    rb = oracle.elastic_pairs(b1, b2, band=N // 2)
    np.testing.assert_allclose(rb["energy"], r["energy"], rtol=1e-12, atol=1e-15)
    bad = b2.copy()
    bad[2, 3] = np.inf
    bad[4] = 0.0
    rs = oracle.elastic_pairs(b1, bad)
    assert list(rs["status"]) == [0, 0, 2, 0, 1, 0] and np.isnan(rs["energy"][[2, 4]]).all()


def test_alternation_from_a_given_start_continues_the_full_run():
    """oracle.elastic_from_start runs the alternation alone.  Started from the
    triple that the full pipeline holds after its first iteration, it ends
    where the full pipeline ends (same shift, energy to rounding), and a bad
    starting shift is flagged per pair."""
    N, P = 64, 6
    rng = np.random.default_rng(11)
    b1 = np.stack([synth.uniform_arclength_nodes(synth.random_harmonics(rng, 6), N)
                   for _ in range(P)])
    b2 = np.stack([synth.uniform_arclength_nodes(synth.random_harmonics(rng, 6), N)
                   for _ in range(P)])
    one = oracle.elastic_pairs(b1, b2, max_iter=1, gamma=True)
    full = oracle.elastic_pairs(b1, b2, max_iter=20, gamma=True)
    cont = oracle.elastic_from_start(b1, b2, one["shift"], one["theta"], one["gamma"],
                                     max_iter=19)
    assert (cont["status"] == 0).all()
    np.testing.assert_array_equal(cont["shift"], full["shift"])
    assert np.abs(cont["energy"] - full["energy"]).max() <= 1e-14
    assert np.abs(cont["gamma"] - full["gamma"]).max() <= 1e-9
    s0 = one["shift"].copy()
    s0[2] = N
    bad = oracle.elastic_from_start(b1, b2, s0, one["theta"], one["gamma"], max_iter=3)
    assert bad["status"][2] == 3 and bad["shift"][2] == -1
    assert (np.delete(bad["status"], 2) == 0).all()
