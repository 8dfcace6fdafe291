"""Pins for oracle O2 (arc-length resampling, Sec. 2: Eq. arc-length-param
and the cubic-spline interpolation at uniform parameters).

The spline is checked against scipy's independent periodic CubicSpline, the
knot construction against polygons whose chord lengths are known exactly, and
the whole step against interpolation and convergence properties.
"""
import numpy as np
import pytest
from scipy.interpolate import CubicSpline

import oracle
from paper_2501_17779_gb300 import synth


def _csr(curves):
    offs = np.concatenate([[0], np.cumsum([c.size for c in curves])]).astype(np.int64)
    return np.concatenate(curves).astype(np.complex128), offs


def _scipy_resample(p, N, knots):
    """Periodic cubic spline through (knots, p) with p_n = p_0, at k/N."""
    u = np.concatenate([knots, [1.0]])
    pc = np.concatenate([p, p[:1]])
    t = np.arange(N) / N
    x = CubicSpline(u, pc.real, bc_type="periodic")(t)
    y = CubicSpline(u, pc.imag, bc_type="periodic")(t)
    return x + 1j * y


def test_rectangle_knots_exact():
    """A 3 x 1 rectangle: chord lengths 3, 1, 3, 1, so the arc-length knots
    are 0, 3/8, 1/2, 7/8 exactly (Eq. arc-length-param)."""
    p = np.array([0, 3, 3 + 1j, 1j])
    knots = np.array([0.0, 3 / 8, 1 / 2, 7 / 8])
    pts, offs = _csr([p])
    z, st = oracle.resample(pts, offs, 64, flags=0)
    assert st[0] == 0
    np.testing.assert_allclose(z[0], _scipy_resample(p, 64, knots), atol=1e-13)
    # t = 0, 3/8, 1/2, 7/8 fall on the knots: the spline interpolates the corners
    for k, node in zip([0, 24, 32, 56], p):
        assert abs(z[0, k] - node) < 1e-13


@pytest.mark.parametrize("seed", range(6))
def test_matches_scipy_periodic_spline(seed):
    pts, offs = synth.raw_curves(500 + seed, C=3, n_min=40, n_max=300)
    z, st = oracle.resample(pts, offs, 256, flags=0)
    assert (st == 0).all()
    for i in range(3):
        p = pts[offs[i]:offs[i + 1]]
        d = np.abs(np.roll(p, -1) - p)
        knots = np.concatenate([[0.0], np.cumsum(d)[:-1]]) / d.sum()
        ref = _scipy_resample(p, 256, knots)
        assert np.abs(z[i] - ref).max() < 1e-12 * np.abs(p).max()


@pytest.mark.parametrize("n", [8, 37, 256])
def test_regular_polygon_reproduces_nodes(n):
    """Equal chords give knots l/n; resampling at N = n and N = 2n returns the
    input nodes at the knots (interpolation property)."""
    p = 2.0 * np.exp(2j * np.pi * np.arange(n) / n) + (0.3 - 0.1j)
    pts, offs = _csr([p])
    z, st = oracle.resample(pts, offs, n, flags=0)
    np.testing.assert_allclose(z[0], p, atol=1e-12)
    z2, _ = oracle.resample(pts, offs, 2 * n, flags=0)
    np.testing.assert_allclose(z2[0, ::2], p, atol=1e-12)


def test_circle_convergence_fourth_order():
    """Jittered dense samples of a circle resample onto the circle with an error
    that drops like h^4 (cubic spline)."""
    errs = []
    for n in (64, 128, 256):
        rng = np.random.default_rng(n)
        phi = 2 * np.pi * (np.arange(n) + rng.uniform(-0.3, 0.3, n)) / n
        pts, offs = _csr([np.exp(1j * phi)])
        z, _ = oracle.resample(pts, offs, 512, flags=0)
        errs.append(np.abs(np.abs(z[0]) - 1.0).max())
    assert errs[0] / errs[1] > 10 and errs[1] / errs[2] > 10
    assert errs[2] < 1e-7


def test_centring_and_unit_length():
    pts, offs = synth.raw_curves(9, C=8, n_min=500, n_max=2000)
    z, st = oracle.resample(pts, offs, 1024)
    assert (st == 0).all()
    assert np.abs(z.mean(axis=1)).max() < 2e-15
    per = np.abs(np.roll(z, -1, axis=1) - z).sum(axis=1)
    np.testing.assert_allclose(per, 1.0, atol=1e-14)


def test_similarity_invariance_and_closing_duplicate():
    """Translating, scaling and rotating the input moves the normalised output
    only by the rotation; an explicit closing duplicate is ignored."""
    pts, offs = synth.raw_curves(11, C=1, n_min=300, n_max=300)
    z0, _ = oracle.resample(pts, offs, 256)
    rot = np.exp(0.4j)
    z1, _ = oracle.resample(3.5 * rot * pts + (1 - 2j), offs, 256)
    np.testing.assert_allclose(z1[0], rot * z0[0], atol=1e-13)
    closed = np.concatenate([pts, pts[:1]])
    z2, st = oracle.resample(closed, np.array([0, closed.size]), 256)
    assert st[0] == 0
    np.testing.assert_allclose(z2[0], z0[0], atol=0)


def test_degenerate_statuses():
    good = np.exp(2j * np.pi * np.arange(10) / 10)
    three = good[:3]
    rep = good.copy()
    rep[4] = rep[3]
    nan = good.copy()
    nan[2] = np.nan
    pts, offs = _csr([good, three, rep, nan, good[:0]])
    z, st = oracle.resample(pts, offs, 32)
    assert list(st) == [0, 1, 1, 2, 1]
    assert np.isfinite(z[0]).all() and np.isnan(z[1:]).all()
