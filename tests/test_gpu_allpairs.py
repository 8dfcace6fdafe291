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
