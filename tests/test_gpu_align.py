"""GPU parity of fa_align_pairs (FA_FFT and FA_DIRECT) against the FP64 oracle.

All calls go through the C ABI (paper_2501_17779_gb300.api -> libfftalign.so).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2501_17779_gb300 import api, synth

from _parity import check_align, wrap

pytestmark = pytest.mark.gpu

DEV = "cuda"


# (method, prec) combinations of the alignment path; FA_PREC_MIXED must meet the
# same FP64 bounds as FA_PREC_FP64
PATHS = [("fft", "fp64"), ("fft", "mixed"), ("direct", "fp64")]
FFT_PATHS = [("fft", "fp64"), ("fft", "mixed")]


def _run(z1, z2, method="fft", dtype=torch.complex128, prec="fp64"):
    if isinstance(method, tuple):
        method, prec = method
    t1 = torch.from_numpy(np.ascontiguousarray(z1)).to(DEV, dtype)
    t2 = torch.from_numpy(np.ascontiguousarray(z2)).to(DEV, dtype)
    s, th, e, st = api.align_pairs(t1, t2, method=method, prec=prec)
    torch.cuda.synchronize()
    return s.cpu().numpy(), th.cpu().numpy(), e.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("method", PATHS)
def test_parity_64_pairs_n256(method):
    """The 64-pair, N = 256 workload: noisy rotated and shifted copies."""
    ap = synth.aligned_pairs(1001, P=64, N=256)
    out = _run(ap.z1, ap.z2, method)
    check_align(ap.z1, ap.z2, *out)


@pytest.mark.parametrize("method", PATHS)
def test_exact_recovery_noise_free(method):
    ap = synth.aligned_pairs(2001, P=64, N=256, noise=0.0)
    s, th, e, st = _run(ap.z1, ap.z2, method)
    np.testing.assert_array_equal(s, ap.shift_true)
    assert np.abs(wrap(th - ap.theta_true)).max() < 1e-12
    assert e.max() < 1e-15
    assert (st == 0).all()


@pytest.mark.parametrize("path", FFT_PATHS)
@pytest.mark.parametrize("logn", range(2, 13))
def test_fft_all_sizes(logn, path):
    """Every supported FFT size (radix-2 first stage for odd log2 N, several
    pairs per CTA for small N, one pair per CTA for large N); an odd pair count
    leaves a ragged tail block."""
    N = 1 << logn
    P = 37 if N <= 1024 else 9
    ap = synth.aligned_pairs(300 + logn, P=P, N=N, n_harm=min(8, N // 4), noise=2e-3)
    out = _run(ap.z1, ap.z2, path)
    check_align(ap.z1, ap.z2, *out)


@pytest.mark.parametrize("N", [1, 2, 3, 7, 100, 257, 1000, 4096])
def test_direct_any_size(N):
    rng = np.random.default_rng(N)
    z1 = rng.normal(size=(5, N)) + 1j * rng.normal(size=(5, N))
    z2 = rng.normal(size=(5, N)) + 1j * rng.normal(size=(5, N))
    out = _run(z1, z2, "direct")
    check_align(z1, z2, *out)


def test_fft_and_direct_agree_n1024():
    ap = synth.aligned_pairs(77, P=48, N=1024, n_harm=16)
    orc = None
    for path in PATHS:
        orc = check_align(ap.z1, ap.z2, *_run(ap.z1, ap.z2, path), orc=orc)


def test_complex64_storage_matches_oracle_on_rounded_input():
    """FA_Z_F32 widens each stored float to FP64 on load, so the oracle run on
    the float-rounded curves is the exact reference (FP64 tolerances)."""
    ap = synth.aligned_pairs(5, P=64, N=512)
    z1 = ap.z1.astype(np.complex64).astype(np.complex128)
    z2 = ap.z2.astype(np.complex64).astype(np.complex128)
    for path in PATHS:
        out = _run(ap.z1, ap.z2, path, dtype=torch.complex64)
        check_align(z1, z2, *out)


@pytest.mark.parametrize("path", FFT_PATHS)
def test_closed_forms_circle_and_ellipse(path):
    """(For FA_PREC_MIXED every shift of the circle is a candidate.)"""
    N = 256
    phi = 2 * np.pi * np.arange(N) / N
    circ = np.exp(1j * phi)
    ell = 1.3 * np.cos(phi) + 0.6j * np.sin(phi)
    z1 = np.stack([circ, ell])
    z2 = np.stack([np.exp(0.7j) * circ, ell])
    s, th, e, st = _run(z1, z2, path)
    # circle: every shift optimal, angle -0.7 - 2 pi s / N at the chosen shift
    assert abs(wrap(th[0] + 0.7 + 2 * np.pi * s[0] / N)) < 1e-12
    assert e[0] < 1e-14
    # ellipse against itself: s = 0 (angle 0) or s = N/2 (angle pi), energy 0
    assert s[1] in (0, N // 2)
    assert abs(wrap(th[1] - (0.0 if s[1] == 0 else np.pi))) < 1e-12
    assert e[1] < 1e-14


@pytest.mark.parametrize("path", FFT_PATHS)
def test_template_protocol(path):
    """Sec. 2 template: start point moved by 1/4, rotated by pi/3."""
    rng = np.random.default_rng(3)
    for N in (64, 256, 1024, 4096):
        z1, z2 = synth.template_pair(synth.random_harmonics(rng, 8), N)
        s, th, e, st = _run(z1[None], z2[None], path)
        assert s[0] == 3 * N // 4
        assert abs(th[0] + np.pi / 3) < 1e-12
        assert e[0] < 1e-15


def test_nonfinite_and_zero_inputs():
    ap = synth.aligned_pairs(9, P=6, N=128)
    z1, z2 = ap.z1.copy(), ap.z2.copy()
    z1[1, 5] = np.nan
    z2[3, 0] = np.inf
    z1[4] = 0.0  # c(s) = 0 for all s: theta 0, energy ||b2||^2
    for method in PATHS:
        s, th, e, st = _run(z1, z2, method)
        assert list(st) == [0, 2, 0, 2, 0, 0]
        assert s[1] == -1 and np.isnan(th[1]) and np.isnan(e[1])
        assert th[4] == 0.0 and s[4] == 0
        assert abs(e[4] - np.sum(np.abs(z2[4]) ** 2) / 128) < 1e-15


def test_empty_batch_and_bad_arguments():
    z = torch.zeros((0, 256), dtype=torch.complex128, device=DEV)
    s, th, e, st = api.align_pairs(z, z)
    assert s.numel() == 0
    z = torch.zeros((2, 100), dtype=torch.complex128, device=DEV)
    with pytest.raises(api._lib.FAError) as ei:
        api.align_pairs(z, z, method="fft")
    assert ei.value.code == api._lib.ERR_UNSUPPORTED
    with pytest.raises(api._lib.FAError) as ei:
        api.align_pairs(z, z, method="direct", prec="mixed")
    assert ei.value.code == api._lib.ERR_INVALID_ARG


def test_full_size_sampled_against_oracle():
    """4096 pairs at N = 1024 in the benchmark's launch configuration; the
    oracle checks a sample of 48 pairs, every pair is checked for validity,
    and the mixed-precision search agrees with the FP64 search on all pairs
    (identical shifts unless the FP64 energies are within the tie tolerance)."""
    ap = synth.aligned_pairs(1234, P=4096, N=1024, n_harm=16, oversample=8)
    s, th, e, st = _run(ap.z1, ap.z2, "fft")
    assert (st == 0).all()
    assert ((s >= 0) & (s < 1024)).all() and np.isfinite(th).all() and (e >= 0).all()
    idx = np.random.default_rng(0).choice(4096, 48, replace=False)
    check_align(ap.z1[idx], ap.z2[idx], s[idx], th[idx], e[idx], st[idx])
    sm, thm, em, stm = _run(ap.z1, ap.z2, ("fft", "mixed"))
    assert (stm == 0).all()
    same = sm == s
    assert np.abs(em[~same] - e[~same]).max(initial=0.0) <= 1e-9
    assert np.abs(wrap(thm[same] - th[same])).max() <= 1e-10
    assert (np.abs(em[same] - e[same]) <= 1e-12 * e[same]).all()
    check_align(ap.z1[idx], ap.z2[idx], sm[idx], thm[idx], em[idx], stm[idx])


@pytest.mark.parametrize("path", FFT_PATHS)
def test_repeatable_bitwise(path):
    ap = synth.aligned_pairs(42, P=128, N=1024)
    a = _run(ap.z1, ap.z2, path)
    b = _run(ap.z1, ap.z2, path)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_mixed_near_ties():
    """Pairs built to have two nearly equal shifts (a curve with a two-fold
    symmetry plus a tiny perturbation): the double-float search must still
    return the oracle's winner or a shift inside the tie tolerance."""
    N = 512
    rng = np.random.default_rng(11)
    phi = 2 * np.pi * np.arange(N) / N
    z1 = []
    z2 = []
    for p in range(32):
        base = (1 + 0.3 * np.cos(2 * phi + rng.uniform(0, 6))) * np.exp(1j * phi)
        pert = base * (1 + 1e-6 * (p + 1) * np.cos(phi + rng.uniform(0, 6)))
        a = pert - pert.mean()
        a /= np.abs(np.roll(a, -1) - a).sum()
        b = np.exp(1j * rng.uniform(0, 6)) * np.roll(a, int(rng.integers(0, N)))
        z1.append(a)
        z2.append(b)
    z1, z2 = np.array(z1), np.array(z2)
    check_align(z1, z2, *_run(z1, z2, ("fft", "mixed")))
