"""GPU parity of fa_align_pairs_ragged (uneven node counts, one persistent
launch) against the FP64 oracle (C ABI)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2501_17779_gb300 import _lib, api, synth

from _parity import check_align, wrap

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _split(rp):
    P = rp.offsets.size - 1
    n = np.diff(rp.offsets)
    return P, n


def _check_ragged(rp, out):
    """Oracle per pair (any length), FP64 bounds."""
    s, th, e, st = [x.cpu().numpy() for x in out]
    P, n = _split(rp)
    for N in np.unique(n):
        idx = np.nonzero(n == N)[0]
        z1 = np.stack([rp.z1[rp.offsets[p]:rp.offsets[p + 1]] for p in idx])
        z2 = np.stack([rp.z2[rp.offsets[p]:rp.offsets[p + 1]] for p in idx])
        check_align(z1, z2, s[idx], th[idx], e[idx], st[idx])


def _dev(rp, dtype=torch.complex128):
    return (torch.from_numpy(rp.z1).to(DEV, dtype), torch.from_numpy(rp.z2).to(DEV, dtype),
            torch.from_numpy(rp.offsets).to(DEV))


def test_ragged_mixed_sizes_all_decompositions():
    """Powers of two (L = n, one to two sub-transforms), non-powers with
    L = 2..4 x 4096 (one, two and four sub-transforms), the smallest sizes."""
    sizes = [4, 5, 7, 16, 17, 64, 100, 256, 333, 1000, 1024, 2047, 2048, 2049, 3000, 4096,
             4097, 5000, 6144, 8191, 8192]
    rp = synth.ragged_aligned_pairs(21, sizes, min_harm=2, max_harm=12)
    out = api.align_pairs_ragged(*_dev(rp))
    torch.cuda.synchronize()
    _check_ragged(rp, out)


def test_ragged_noise_free_exact_recovery():
    sizes = synth.log_uniform_sizes(5, 40, 64, 8192)
    rp = synth.ragged_aligned_pairs(22, sizes, noise=0.0)
    s, th, e, st = [x.cpu().numpy() for x in api.align_pairs_ragged(*_dev(rp))]
    np.testing.assert_array_equal(s, rp.shift_true)
    assert np.abs(wrap(th - rp.theta_true)).max() < 1e-12
    assert e.max() < 1e-15 and (st == 0).all()


def test_ragged_bad_sizes_and_nonfinite():
    good = synth.ragged_aligned_pairs(23, [64, 100, 8192, 128])
    z1 = np.concatenate([good.z1[:64], np.zeros(3), good.z1[64:164], np.zeros(9000),
                         good.z1[164:]])
    z2 = np.concatenate([good.z2[:64], np.zeros(3), good.z2[64:164], np.zeros(9000),
                         good.z2[164:]])
    sizes = [64, 3, 100, 9000, 0, 8192, 128]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    z1[offs[6] + 5] = np.nan  # pair 6 non-finite
    rp = synth.RaggedPairs(z1, z2, offs, None, None)
    s, th, e, st = [x.cpu().numpy() for x in api.align_pairs_ragged(*_dev(rp), max_n=8192)]
    assert list(st) == [0, 3, 0, 3, 3, 0, 2]
    assert (s[[1, 3, 4, 6]] == -1).all() and np.isnan(e[[1, 3, 4, 6]]).all()
    ok = [0, 2, 5]
    for p in ok:
        a = z1[offs[p]:offs[p + 1]][None]
        b = z2[offs[p]:offs[p + 1]][None]
        check_align(a, b, s[[p]], th[[p]], e[[p]], st[[p]])


def test_ragged_max_n_bound_and_complex64():
    rp = synth.ragged_aligned_pairs(24, [100, 200, 300])
    s, th, e, st = [x.cpu().numpy() for x in api.align_pairs_ragged(*_dev(rp, torch.complex64),
                                                                    max_n=250)]
    assert list(st) == [0, 0, 3]
    r = synth.RaggedPairs(rp.z1.astype(np.complex64).astype(np.complex128),
                          rp.z2.astype(np.complex64).astype(np.complex128), rp.offsets, None, None)
    for p in (0, 1):
        a = r.z1[r.offsets[p]:r.offsets[p + 1]][None]
        b = r.z2[r.offsets[p]:r.offsets[p + 1]][None]
        check_align(a, b, s[[p]], th[[p]], e[[p]], st[[p]])


def test_ragged_graph_capture_and_autotune():
    """The whole call (a memset, the bucketing launches and one launch per
    transform-length bucket) captured in a CUDA graph and replayed gives the
    same result as a direct call; the autotuner picks a plan per bucket and
    leaves a valid result."""
    sizes = synth.log_uniform_sizes(9, 300, 64, 4096)
    rp = synth.ragged_aligned_pairs(25, sizes, min_harm=4, max_harm=16)
    z1, z2, offs = _dev(rp)
    P = offs.numel() - 1
    ws = torch.empty(api.ragged_workspace_size(P, 4096), dtype=torch.uint8, device=DEV)
    ref = api.align_pairs_ragged(z1, z2, offs, max_n=4096, workspace=ws, autotune=True)
    torch.cuda.synchronize()
    plan = api.ragged_plan()
    tuned = {b: v for b, v in plan.items() if v[2] > 0}
    print("autotuned plans (log2 L: threads, pairs per CTA, ms):", tuned)
    assert tuned  # at least one bucket was timed
    ref = [x.clone() for x in ref]
    out = tuple(torch.empty_like(x) for x in ref)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        api.align_pairs_ragged(z1, z2, offs, max_n=4096, workspace=ws, out=out)  # warm-up
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        api.align_pairs_ragged(z1, z2, offs, max_n=4096, workspace=ws, out=out)
    for x in out:
        x.zero_()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(ref, out):
        torch.testing.assert_close(a, b, rtol=0, atol=0)
    _check_ragged(rp, ref)


def test_ragged_large_batch_sampled():
    """4000 pairs, n log-uniform in [64, 8192] (multiples of 16), 4..32
    harmonics, generated on the device; the oracle checks a sample of 24 pairs
    across the size range, every pair is checked for validity."""
    sizes = synth.log_uniform_sizes(31, 4000)
    z1, z2, offs = synth.ragged_pairs_device(31, sizes, DEV)
    s, th, e, st = api.align_pairs_ragged(z1, z2, offs, max_n=8192)
    torch.cuda.synchronize()
    s, th, e, st = [x.cpu().numpy() for x in (s, th, e, st)]
    n = np.asarray(sizes)
    assert (st == 0).all() and (s >= 0).all() and (s < n).all() and np.isfinite(e).all()
    order = np.argsort(n)
    idx = order[np.linspace(0, len(n) - 1, 24).astype(int)]
    o = offs.cpu().numpy()
    a1, a2 = z1.cpu().numpy(), z2.cpu().numpy()
    for p in idx:
        check_align(a1[o[p]:o[p + 1]][None], a2[o[p]:o[p + 1]][None], s[[p]], th[[p]], e[[p]],
                    st[[p]])


# (CTA size, pairs per CTA); -R: one pair per cluster of R CTAs (L = R 4096)
PLANS = [(256, 1), (512, 1), (1024, 1), (128, 2), (256, 2), (512, 2), (128, 4), (256, 4),
         (512, 4), (256, 8), (256, 16), (256, -2), (512, -2), (256, -4), (512, -4)]


def test_ragged_every_plan_on_every_bucket_it_fits():
    """Each compiled plan (CTA size, pairs per CTA, or a cluster of CTAs per
    pair), pinned on every transform length it can run, against the FP64 oracle: buckets log2 L = 2..14 with
    several pairs each (partly filled multi-pair CTAs included), powers of two
    and padded lengths, one radix-R split length per R."""
    sizes = [4, 5, 7, 9, 16, 17, 20, 33, 60, 64, 65, 100, 128, 129, 200, 256, 257, 300, 400,
             512, 513, 700, 1000, 1024, 1025, 1500, 2048, 2049, 3000, 4096, 4097, 6000, 8192]
    rp = synth.ragged_aligned_pairs(26, sizes, min_harm=2, max_harm=12)
    z1, z2, offs = _dev(rp)
    P, n = _split(rp)
    orc = {}
    for N in np.unique(n):
        idx = np.nonzero(n == N)[0]
        a = np.stack([rp.z1[rp.offsets[p]:rp.offsets[p + 1]] for p in idx])
        b = np.stack([rp.z2[rp.offsets[p]:rp.offsets[p + 1]] for p in idx])
        orc[N] = (idx, a, b, oracle.align_pairs(a, b))
    L = np.array([m if m & (m - 1) == 0 else 1 << int(2 * m - 1).bit_length() for m in n])
    buckets = sorted(set(int(np.log2(x)) for x in L))
    try:
        for T, G in PLANS:
            used = []
            for b in buckets:
                try:
                    api.set_ragged_plan(b, T, G)
                    used.append(b)
                except RuntimeError:
                    api.set_ragged_plan(b, 256, 1)
            s, th, e, st = [x.cpu().numpy() for x in api.align_pairs_ragged(z1, z2, offs,
                                                                            max_n=8192)]
            for N, (idx, a, b, o) in orc.items():
                check_align(a, b, s[idx], th[idx], e[idx], st[idx], o)
            print(f"plan ({T}, {G}) ran on buckets {used}")
            assert used  # every plan fits some length of this batch
    finally:
        for b in range(2, 15):
            api.set_ragged_plan(b, 256, 1)


def test_ragged_plan_rejects_what_does_not_fit():
    with pytest.raises(RuntimeError):
        api.set_ragged_plan(12, 256, 4)   # 4 pairs of 4096 points exceed shared memory
    with pytest.raises(RuntimeError):
        api.set_ragged_plan(5, 256, 2)    # 128 threads per 32-point pair
    with pytest.raises(RuntimeError):
        api.set_ragged_plan(8, 640, 1)    # not compiled
    with pytest.raises(RuntimeError):
        api.set_ragged_plan(13, 512, -4)  # a cluster of 4 needs L = 16384
    with pytest.raises(RuntimeError):
        api.set_ragged_plan(12, 256, -2)  # 4096 points fit one CTA
    plan = api.ragged_plan()
    assert set(plan) == set(range(2, 15))
    assert all(t > 0 and (g >= 1 or g in (-2, -4)) for t, g, _ in plan.values())
