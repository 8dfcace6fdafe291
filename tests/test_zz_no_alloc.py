"""fa_resample_arclength_noalloc: resampling without any device allocation.

This entry point exists for callers that cannot call cudaMalloc (applications
that own the whole device memory budget and do not let libraries allocate,
and latency-critical loops that cannot take an allocation's implicit
synchronisation).  It takes no handle and no workspace; its scratch is a
fixed 64 MiB device array inside the library.  The test calls it through the
C ABI twice in a row, on two different batches, and checks each result
against the regular workspace-taking entry point within the resampling
tolerance used by the other GPU tests.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2501_17779_gb300 import _lib, api, synth

TOL = 1e-12
TOL_F32 = 2.0 ** -23  # complex64 output: one rounding of a unit-scale value


def _noalloc(L, pts, offs, N, flags):
    C = offs.numel() - 1
    zdt = torch.complex64 if flags & _lib.STORE_FP32 else torch.complex128
    z = torch.full((C, N), float("nan"), dtype=zdt, device=pts.device)
    st = torch.full((C,), -7, dtype=torch.int8, device=pts.device)
    rc = L.fa_resample_arclength_noalloc(pts.data_ptr(), offs.data_ptr(), C, pts.numel(), N,
                                         flags, z.data_ptr(), st.data_ptr(),
                                         torch.cuda.current_stream().cuda_stream)
    _lib.check(rc)
    return z, st


@pytest.mark.gpu
def test_noalloc_matches_workspace_entry_point_on_two_calls():
    L = _lib.load()
    dev = torch.device("cuda", 0)
    flags = _lib.CENTER | _lib.UNIT_LENGTH
    batches = [synth.raw_curves(31, C=96, n_min=500, n_max=2000),
               synth.raw_curves(32, C=40, n_min=50, n_max=700)]
    for (pts_np, offs_np), N in zip(batches, (1024, 256)):
        pts = torch.from_numpy(pts_np).to(dev)
        offs = torch.from_numpy(offs_np).to(dev)
        need = L.fa_resample_workspace_size(offs.numel() - 1, pts.numel(), N, flags)
        assert need <= _lib.NOALLOC_SCRATCH_BYTES
        z, st = _noalloc(L, pts, offs, N, flags)
        zr, str_ = api.resample_arclength(pts, offs, N)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(st.cpu().numpy(), str_.cpu().numpy())
        assert (st.cpu().numpy() == 0).all()
        assert float((z - zr).abs().max()) <= TOL


@pytest.mark.gpu
def test_noalloc_complex64_output_matches_workspace_entry_point():
    """With FA_STORE_FP32 the complex128 staging rows also live in the fixed
    array; the result equals the workspace entry point's complex64 output."""
    L = _lib.load()
    dev = torch.device("cuda", 0)
    flags = _lib.CENTER | _lib.UNIT_LENGTH | _lib.STORE_FP32
    pts_np, offs_np = synth.raw_curves(33, C=64, n_min=300, n_max=1500)
    pts = torch.from_numpy(pts_np).to(dev)
    offs = torch.from_numpy(offs_np).to(dev)
    N = 512
    need = L.fa_resample_workspace_size(offs.numel() - 1, pts.numel(), N, flags)
    assert need <= _lib.NOALLOC_SCRATCH_BYTES
    for _ in range(2):
        z, st = _noalloc(L, pts, offs, N, flags)
        zr, str_ = api.resample_arclength(pts, offs, N, fp32=True)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(st.cpu().numpy(), str_.cpu().numpy())
        assert (st.cpu().numpy() == 0).all()
        assert z.dtype == torch.complex64 and zr.dtype == torch.complex64
        assert float((z - zr).abs().max()) <= TOL_F32


def test_noalloc_rejects_sizes_whose_scratch_would_wrap():
    """2^61 nodes would wrap the 64-bit scratch size to a small number; the
    call rejects it on the host before touching any pointer (no GPU needed:
    the pointers below are never dereferenced)."""
    L = _lib.load()
    fake = ctypes.c_void_p(256)
    for n_pts in (2 ** 61, 2 ** 41):
        rc = L.fa_resample_arclength_noalloc(fake, fake, 1, n_pts, 256,
                                             _lib.CENTER | _lib.UNIT_LENGTH, fake, fake, None)
        assert rc == _lib.ERR_UNSUPPORTED
    assert L.fa_resample_workspace_size(1, 2 ** 61, 256, 0) == 2 ** 64 - 1


@pytest.mark.gpu
def test_noalloc_rejects_batches_beyond_its_scratch():
    L = _lib.load()
    dev = torch.device("cuda", 0)
    n_pts = 2_000_000  # 48 bytes per node > 64 MiB; nothing is launched
    pts = torch.zeros(4, dtype=torch.complex128, device=dev)
    offs = torch.tensor([0, 4], dtype=torch.int64, device=dev)
    z = torch.empty((1, 256), dtype=torch.complex128, device=dev)
    st = torch.empty(1, dtype=torch.int8, device=dev)
    rc = L.fa_resample_arclength_noalloc(pts.data_ptr(), offs.data_ptr(), 1, n_pts, 256,
                                         _lib.CENTER | _lib.UNIT_LENGTH, z.data_ptr(),
                                         st.data_ptr(), None)
    assert rc == _lib.ERR_UNSUPPORTED
    msg = L.fa_last_error().decode()
    assert "bytes of scratch" in msg and str(_lib.NOALLOC_SCRATCH_BYTES) in msg
