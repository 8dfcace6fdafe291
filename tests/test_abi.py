"""CPU-only checks of the C ABI: the library builds for sm_103a, loads, and
exports every function that include/fftalign.h declares (no GPU calls)."""
import ctypes
import re
from pathlib import Path

import pytest

from paper_2501_17779_gb300 import _lib, build

ROOT = Path(__file__).resolve().parent.parent


def _declared():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        txt = h.read_text()
        names |= set(re.findall(r"^\s*(?:int|int64_t|size_t|const char\*)\s+(fa_\w+)\s*\(", txt, re.M))
    return names


def test_header_declares_the_abi():
    assert {"fa_create", "fa_destroy", "fa_resample_arclength", "fa_align_pairs",
            "fa_align_curves_host", "fa_last_error", "fa_version",
            "fa_resample_workspace_size"} <= _declared()


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    L = ctypes.CDLL(str(path))
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing
    assert set(_lib.EXPORTS) == _declared()


def test_calls_without_gpu_return_codes():
    """Functions that need no device return their documented values on a host
    without a GPU: version, workspace size, and argument errors."""
    L = _lib.load()
    assert L.fa_version() == 10000
    ws = L.fa_resample_workspace_size(8, 1000, 256, 0)
    assert ws >= 1000 * (2 * 8 + 2 * 16)  # 48 bytes of workspace per input node
    assert L.fa_resample_workspace_size(-1, 10, 256, 0) == 0
    assert L.fa_align_pairs(None, None, None, 1, 256, 0, 0, 0, None, None, None, None, None) == \
        _lib.ERR_INVALID_ARG
    assert b"null handle" in L.fa_last_error()
