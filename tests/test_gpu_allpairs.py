"""GPU parity of fa_align_all_pairs against the FP64 oracle (C ABI)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2501_17779_gb300 import api, synth

from _parity import check_align, wrap

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _curves(seed, M, N, n_harm=8):
    ap = synth.aligned_pairs(seed, P=(M + 1) // 2, N=N, n_harm=n_harm, oversample=16)
    return np.concatenate([ap.z1, ap.z2])[:M]


def _gpu_all(z, dtype=torch.complex128, prec="fp64"):
    s, th, e, st = api.align_all_pairs(torch.from_numpy(z).to(DEV, dtype), prec=prec)
    torch.cuda.synchronize()
    return s.cpu().numpy(), th.cpu().numpy(), e.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("M,N", [(24, 256), (17, 64), (9, 1024), (2, 16)])
def test_all_pairs_match_oracle(M, N, prec):
    z = _curves(M * 7 + N, M, N)
    s, th, e, st = _gpu_all(z, prec=prec)
    assert (st == 0).all()
    iu, ju = np.triu_indices(M, 1)
    ok = np.zeros(len(iu), np.int8)
    # upper triangle: curve j aligned onto curve i
    check_align(z[iu], z[ju], s[iu, ju], th[iu, ju], e[iu, ju], ok)
    # lower triangle: by symmetry, still a correct alignment of (j, i)
    check_align(z[ju], z[iu], s[ju, iu], th[ju, iu], e[ju, iu], ok)
    np.testing.assert_array_equal(s[ju, iu], (N - s[iu, ju]) % N)
    np.testing.assert_array_equal(e[ju, iu], e[iu, ju])
    assert (np.diag(s) == 0).all() and (np.diag(th) == 0).all() and (np.diag(e) == 0).all()


def test_all_pairs_complex64_and_bad_curve():
    M, N = 12, 128
    z = _curves(5, M, N)
    z[4, 7] = np.nan
    s, th, e, st = _gpu_all(z, torch.complex64)
    assert list(np.nonzero(st)[0]) == [4] and st[4] == 2
    assert (s[4, np.arange(M) != 4] == -1).all() and np.isnan(e[:, 4][np.arange(M) != 4]).all()
    good = [m for m in range(M) if m != 4]
    zr = z.astype(np.complex64).astype(np.complex128)
    iu, ju = np.triu_indices(M, 1)
    keep = (iu != 4) & (ju != 4)
    iu, ju = iu[keep], ju[keep]
    check_align(zr[iu], zr[ju], s[iu, ju], th[iu, ju], e[iu, ju], np.zeros(len(iu), np.int8))
    assert len(good) == M - 1


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_all_pairs_full_size_sample(prec):
    """M = 2048 curves at N = 512 (2,096,128 ordered pairs); the oracle checks a
    sample of 64 pairs, every entry is checked for validity and symmetry."""
    M, N = 2048, 512
    z = _curves(777, M, N, n_harm=12)
    s, th, e, st = _gpu_all(z, prec=prec)
    assert (st == 0).all()
    off = ~np.eye(M, dtype=bool)
    assert ((s >= 0) & (s < N)).all() and np.isfinite(th).all() and (e[off] >= 0).all()
    np.testing.assert_array_equal(e, e.T)
    rng = np.random.default_rng(3)
    i = rng.integers(0, M, 64)
    j = (i + rng.integers(1, M, 64)) % M
    check_align(z[i], z[j], s[i, j], th[i, j], e[i, j], np.zeros(64, np.int8))


# ---- the tensor-core search (FA_PREC_TC_*) ----------------------------------
TC_PRECS = ["tc_bf16x3", "tc_fp16x3", "tc_tf32x3", "tc_tf32"]
# tie-aware shift agreement with the FP64 oracle required of each variant: the
# float16 and TF32 split (x3) forms carry 21-22 significant bits into the GEMM,
# enough to keep the best shift among the 8 re-scored candidates on >= 99.9 %
# of pairs; bfloat16 pieces carry ~16 bits, and on the flat correlation peaks
# of smooth curves (neighbouring shifts within 1e-5 of the best) the best
# shift can fall outside the 8 kept (measured: 1 pair in 780 at N = 512 here,
# 99.98 % of the 2.1 M pairs of the full-size matrix); plain TF32 (11 bits)
# cannot separate those shifts at all (measured 52 % at N = 512, 75 % at 256)
# and is held to a floor only.  Every reported result is still the exact
# optimum at its own shift (checked below).
TC_AGREE = {"tc_bf16x3": 0.99, "tc_fp16x3": 0.999, "tc_tf32x3": 0.999, "tc_tf32": 0.4}


def _exact_at_reported_shift(z1, z2, s, th, e):
    """Whatever shift a pair reports, its angle and energy must be the FP64
    optimum at that shift: the oracle's Kabsch score there gives
    E(s) = h (|z1|^2 + |z2|^2 - 2 score(s)) (expanded form, so the floor allows
    its cancellation) and the angle is checked through the energy."""
    P, N = z1.shape
    h = 1.0 / N
    for p in range(P):
        sc = oracle.shift_scores(z1[p], z2[p])
        n = h * (np.sum(np.abs(z1[p]) ** 2) + np.sum(np.abs(z2[p]) ** 2))
        E = n - 2 * h * sc[s[p]]
        assert abs(e[p] - E) <= max(1e-12 * E, 1e-13 * n), (p, e[p], E)
        # the reported angle reproduces the reported energy by its definition
        w = np.exp(1j * th[p]) * np.roll(z2[p], -int(s[p]))
        Ed = h * np.sum(np.abs(z1[p] - w) ** 2)
        assert abs(Ed - e[p]) <= max(1e-12 * Ed, 1e-14 * n), (p, Ed, e[p])


@pytest.mark.parametrize("prec", TC_PRECS)
@pytest.mark.parametrize("M,N", [(40, 512), (33, 256)])
def test_all_pairs_tensor_core_search(M, N, prec):
    """Tensor-core DFT-GEMM search, top-8 candidates re-scored in double-float:
    the tie-aware shift agreement with the FP64 oracle reaches the variant's
    floor, every reported (shift, angle, energy) is the exact optimum at its
    shift, and the lower triangle mirrors the upper one."""
    z = _curves(M * 11 + N, M, N)
    s, th, e, st = _gpu_all(z, prec=prec)
    assert (st == 0).all()
    iu, ju = np.triu_indices(M, 1)
    orc = oracle.align_pairs(z[iu], z[ju])
    same = s[iu, ju] == orc["shift"]
    tie = ~same & (np.abs(e[iu, ju] - orc["energy"]) <= 1e-9)
    agree = float((same | tie).mean())
    print(f"{prec} M={M} N={N}: shift agreement {same.mean():.4f}, with ties {agree:.4f}")
    assert agree >= TC_AGREE[prec]
    _exact_at_reported_shift(z[iu], z[ju], s[iu, ju], th[iu, ju], e[iu, ju])
    # where the shift agrees, the FP64 bounds of the plain search
    if prec != "tc_tf32":
        check_align(z[iu], z[ju], s[iu, ju], th[iu, ju], e[iu, ju], np.zeros(len(iu), np.int8),
                    orc, shift_frac=TC_AGREE[prec])
    np.testing.assert_array_equal(s[ju, iu], (N - s[iu, ju]) % N)
    np.testing.assert_array_equal(e[ju, iu], e[iu, ju])
    assert (np.diag(s) == 0).all() and (np.diag(e) == 0).all()


def test_all_pairs_tensor_core_complex64_bad_curve_and_edges():
    """complex64 input, a non-finite curve (its row and column NaN, status 2),
    and the smallest matrices (M = 0, 1, 2)."""
    M, N = 20, 256
    z = _curves(6, M, N)
    z[3, 5] = np.nan
    s, th, e, st = _gpu_all(z, torch.complex64, prec="tc_bf16x3")
    assert list(np.nonzero(st)[0]) == [3] and st[3] == 2
    others = np.arange(M) != 3
    assert (s[3, others] == -1).all() and np.isnan(e[others, 3]).all()
    zr = z.astype(np.complex64).astype(np.complex128)
    iu, ju = np.triu_indices(M, 1)
    keep = (iu != 3) & (ju != 3)
    _exact_at_reported_shift(zr[iu[keep]], zr[ju[keep]], s[iu[keep], ju[keep]],
                             th[iu[keep], ju[keep]], e[iu[keep], ju[keep]])
    for m in (1, 2):
        s, th, e, st = _gpu_all(_curves(9, m, N), prec="tc_fp16x3")
        assert (st == 0).all() and s.shape == (m, m) and (np.diag(e) == 0).all()
    s, th, e, st = _gpu_all(np.zeros((0, N), np.complex128), prec="tc_fp16x3")
    assert s.shape == (0, 0)
    with pytest.raises(RuntimeError):
        _gpu_all(_curves(9, 4, 128), prec="tc_bf16x3")  # N outside {256, 512}


@pytest.mark.parametrize("prec", ["tc_bf16x3", "tc_fp16x3"])
def test_all_pairs_tensor_core_full_size_sample(prec):
    """M = 2048 curves at N = 512, the benchmark's all-pairs launch: every entry
    valid and symmetric, agreement with the FP64 search on the whole matrix,
    and the oracle on a sample of 64 pairs."""
    M, N = 2048, 512
    z = _curves(777, M, N, n_harm=12)
    s, th, e, st = _gpu_all(z, prec=prec)
    sr, thr, er, _ = _gpu_all(z, prec="mixed")
    assert (st == 0).all()
    off = ~np.eye(M, dtype=bool)
    assert ((s >= 0) & (s < N)).all() and np.isfinite(th).all() and (e[off] >= 0).all()
    np.testing.assert_array_equal(e, e.T)
    same = s == sr
    tie = ~same & (np.abs(e - er) <= 1e-9)
    agree = float((same | tie)[off].mean())
    print(f"{prec}: agreement with the double-float search {same[off].mean():.5f}, "
          f"with ties {agree:.5f}")
    assert agree >= TC_AGREE[prec]
    rng = np.random.default_rng(3)
    i = rng.integers(0, M, 64)
    j = (i + rng.integers(1, M, 64)) % M
    _exact_at_reported_shift(z[i], z[j], s[i, j], th[i, j], e[i, j])
