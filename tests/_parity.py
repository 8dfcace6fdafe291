"""Shared parity rules for comparing the CUDA path with the FP64 oracle.

Tolerances (FP64 path):
* shift: exact, unless the oracle's energy gap between its best and
  second-best shift is below 1e-9; then the GPU's shift must have an oracle
  energy within 1e-9 of the optimum (several shifts are then correct).
* theta: within 1e-10 rad (mod 2 pi) where the shifts agree.
* energy: relative 1e-12 when E > 1e-10 (||b1||^2 + ||b2||^2), else absolute
  1e-14 (||b1||^2 + ||b2||^2), with ||b||^2 = h sum |z|^2.
"""
from __future__ import annotations

import numpy as np

import oracle

GAP = 1e-9


def wrap(a):
    return np.angle(np.exp(1j * np.asarray(a)))


def check_align(z1, z2, shift, theta, energy, status, orc=None, *, theta_tol=1e-10,
                e_rel=1e-12, e_abs=1e-14, shift_frac=1.0):
    """Compare GPU outputs (numpy) with the oracle on the same inputs.

    Returns the oracle's result dict.  ``shift_frac`` < 1 allows that fraction
    of shifts to disagree outside ties (reduced-precision storage variants).
    """
    z1 = np.asarray(z1)
    z2 = np.asarray(z2)
    if orc is None:
        orc = oracle.align_pairs(z1, z2)
    P, N = z1.shape
    h = 1.0 / N
    norm = h * (np.sum(np.abs(z1) ** 2, axis=1) + np.sum(np.abs(z2) ** 2, axis=1))
    theta_tol = np.broadcast_to(np.asarray(theta_tol, np.float64), (P,))
    e_rel = np.broadcast_to(np.asarray(e_rel, np.float64), (P,))
    assert (status == orc["status"]).all(), "status mismatch"
    ok = orc["status"] == 0
    bad_shift = 0
    for p in np.nonzero(ok)[0]:
        if shift[p] != orc["shift"][p]:
            sc = oracle.shift_scores(z1[p], z2[p])
            E = h * (np.sum(np.abs(z1[p]) ** 2) + np.sum(np.abs(z2[p]) ** 2) - 2 * sc)
            if not (0 <= shift[p] < N and E[shift[p]] - E.min() <= GAP):
                bad_shift += 1
                continue
            # a tie: the energy at the GPU's shift must match the oracle's energy
            # there (the oracle's per-shift energies come from the expanded form,
            # so the absolute floor allows for its cancellation error)
            lim = max(e_rel[p] * E[shift[p]], max(e_abs, 1e-13) * norm[p])
            assert abs(energy[p] - E[shift[p]]) <= lim, (p, energy[p], E[shift[p]])
            continue
        dth = abs(wrap(theta[p] - orc["theta"][p]))
        assert dth <= theta_tol[p], (p, theta[p], orc["theta"][p], dth)
        Eo = orc["energy"][p]
        if Eo > 1e-10 * norm[p]:
            assert abs(energy[p] - Eo) <= e_rel[p] * Eo, (p, energy[p], Eo)
        else:
            assert abs(energy[p] - Eo) <= e_abs * norm[p], (p, energy[p], Eo)
    assert bad_shift <= np.floor((1.0 - shift_frac) * ok.sum() + 1e-9), f"{bad_shift} shifts differ"
    nok = ~ok
    assert (shift[nok] == -1).all() and np.isnan(theta[nok]).all() and np.isnan(energy[nok]).all()
    return orc


def e2e_tolerances(z1, z2, energy, node_tol=1e-12, e_rel=1e-12, theta_tol=1e-10):
    """Per-pair tolerances (relative energy, angle) when each side resampled
    the raw curves itself: the resampled nodes agree to node_tol (the
    resampling bound), and the aligners agree to (e_rel, theta_tol) on equal
    inputs.  With n_i = h sum |z_i|^2, E the energy and h|c| = (n_1 + n_2 -
    E)/2 the correlation at the winning shift: node perturbations of at most
    node_tol move E = h sum |z1 - R z2|^2, minimised over R and the shift, by
    at most 2 sqrt(E) (2 node_tol) + (2 node_tol)^2, and h c by at most
    node_tol (sqrt(n_1) + sqrt(n_2)) (Cauchy-Schwarz), hence theta = arg c by
    that divided by h|c|."""
    z1, z2 = np.asarray(z1), np.asarray(z2)
    h = 1.0 / z1.shape[1]
    n1 = h * np.sum(np.abs(z1) ** 2, axis=1)
    n2 = h * np.sum(np.abs(z2) ** 2, axis=1)
    E = np.maximum(np.asarray(energy, np.float64), 0.0)
    dz = 2.0 * node_tol
    e_abs = 2.0 * np.sqrt(E) * dz + dz * dz
    er = e_rel + e_abs / np.maximum(E, 1e-300)
    hc = np.maximum((n1 + n2 - E) / 2.0, 1e-300)
    th = theta_tol + node_tol * (np.sqrt(n1) + np.sqrt(n2)) / hc
    return er, th
