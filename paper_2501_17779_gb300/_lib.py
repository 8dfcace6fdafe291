"""ctypes declarations of libfftalign.so (the C ABI of include/fftalign.h).

Loading fails loudly when the library has not been built: there is no CPU
fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

from . import build as _build

# return codes
OK = 0
ERR_INVALID_ARG = -1
ERR_UNSUPPORTED = -2
ERR_CUDA = -3
ERR_WORKSPACE = -4
# per-item status
STATUS_OK = 0
STATUS_DEGENERATE = 1
STATUS_NONFINITE = 2
# flags
CENTER = 1
UNIT_LENGTH = 2
STORE_FP32 = 4
# storage types, methods, precisions
Z_F64 = 0
Z_F32 = 1
FFT = 0
DIRECT = 1
PREC_FP64 = 0
PREC_MIXED = 1
PREC_TC_BF16X3 = 2
PREC_TC_FP16X3 = 3
PREC_TC_TF32 = 4
PREC_TC_TF32X3 = 5

EXPORTS = (
    "fa_create", "fa_destroy", "fa_last_error", "fa_version",
    "fa_resample_workspace_size", "fa_resample_arclength", "fa_align_pairs",
    "fa_align_curves_host", "fa_resample_arclength_noalloc",
    "fa_align_all_pairs_workspace_size", "fa_align_all_pairs_workspace_size_prec",
    "fa_align_all_pairs",
    "fa_align_pairs_ragged_workspace_size", "fa_align_pairs_ragged",
    "fa_align_pairs_ragged_autotune", "fa_align_pairs_ragged_plan",
    "fa_align_pairs_ragged_set_plan",
    "fa_elastic_workspace_size", "fa_elastic_distance",
    "fa_fourier_descriptors", "fa_column_stats", "fa_standardize", "fa_embed_sqdist",
    "fa_select_k", "fa_mlp_num_params", "fa_mlp_create", "fa_mlp_destroy", "fa_mlp_set_params",
    "fa_mlp_get_params", "fa_mlp_forward", "fa_mlp_pair_grad", "fa_mlp_adam_step",
)
KEY_F32 = 0
KEY_F64 = 1
STATUS_BAD_SIZE = 3
NOALLOC_SCRATCH_BYTES = 64 << 20

_lib = None


class FAError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libfftalign error {code}: {msg}")
        self.code = code


def lib_path() -> Path:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libfftalign.so and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not path.exists():
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(
                f"libfftalign.so not found at {path}; build it first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(str(path))
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    L.fa_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
    L.fa_create.restype = ctypes.c_int
    L.fa_destroy.argtypes = [vp]
    L.fa_destroy.restype = ctypes.c_int
    L.fa_last_error.argtypes = []
    L.fa_last_error.restype = ctypes.c_char_p
    L.fa_version.argtypes = []
    L.fa_version.restype = ctypes.c_int
    L.fa_resample_workspace_size.argtypes = [i64, i64, i32, i32]
    L.fa_resample_workspace_size.restype = sz
    L.fa_resample_arclength.argtypes = [vp, vp, vp, i64, i64, i32, i32, vp, vp, vp, sz, vp]
    L.fa_resample_arclength.restype = ctypes.c_int
    L.fa_align_pairs.argtypes = [vp, vp, vp, i64, i32, i32, i32, i32, vp, vp, vp, vp, vp]
    L.fa_align_pairs.restype = ctypes.c_int
    L.fa_align_curves_host.argtypes = [vp, vp, vp, i64, i32, i32, i32, i32, vp, vp, vp, vp, vp]
    L.fa_align_curves_host.restype = ctypes.c_int
    L.fa_align_all_pairs_workspace_size.argtypes = [i64, i32]
    L.fa_align_all_pairs_workspace_size.restype = sz
    L.fa_align_all_pairs_workspace_size_prec.argtypes = [i64, i32, i32]
    L.fa_align_all_pairs_workspace_size_prec.restype = sz
    L.fa_align_all_pairs.argtypes = [vp, vp, i64, i32, i32, i32, vp, vp, vp, vp, vp, sz, vp]
    L.fa_align_all_pairs.restype = ctypes.c_int
    L.fa_align_pairs_ragged_workspace_size.argtypes = [vp, i64, i32]
    L.fa_align_pairs_ragged_workspace_size.restype = sz
    L.fa_align_pairs_ragged.argtypes = [vp, vp, vp, vp, i64, i32, i32, vp, vp, vp, vp, vp, sz, vp]
    L.fa_align_pairs_ragged.restype = ctypes.c_int
    L.fa_align_pairs_ragged_autotune.argtypes = [vp, vp, vp, vp, i64, i32, i32, vp, vp, vp, vp,
                                                 vp, sz, vp, vp]
    L.fa_align_pairs_ragged_autotune.restype = ctypes.c_int
    L.fa_align_pairs_ragged_plan.argtypes = [vp, vp, vp, vp]
    L.fa_align_pairs_ragged_plan.restype = ctypes.c_int
    L.fa_align_pairs_ragged_set_plan.argtypes = [vp, i32, i32, i32]
    L.fa_align_pairs_ragged_set_plan.restype = ctypes.c_int
    L.fa_resample_arclength_noalloc.argtypes = [vp, vp, i64, i64, i32, i32, vp, vp, vp]
    L.fa_resample_arclength_noalloc.restype = ctypes.c_int
    L.fa_elastic_workspace_size.argtypes = [vp, i64, i64, i64, i32, i32]
    L.fa_elastic_workspace_size.restype = sz
    L.fa_elastic_distance.argtypes = [vp, vp, i64, vp, i64, i32, vp, vp, i64, i32, i32, vp, vp, vp,
                                      vp, vp, vp, vp, vp, sz, vp]
    L.fa_elastic_distance.restype = ctypes.c_int
    for name, args in (
            ("fa_fourier_descriptors", [vp, vp, i64, i32, i32, vp, vp]),
            ("fa_column_stats", [vp, vp, i64, i32, vp, vp, vp]),
            ("fa_standardize", [vp, vp, i64, i32, vp, vp, vp]),
            ("fa_embed_sqdist", [vp, vp, i64, vp, i64, i32, vp, vp]),
            ("fa_select_k", [vp, vp, i32, i64, i64, i32, vp, vp, vp]),
            ("fa_mlp_create", [vp, ctypes.c_uint64, ctypes.POINTER(vp)]),
            ("fa_mlp_destroy", [vp]),
            ("fa_mlp_set_params", [vp, vp]),
            ("fa_mlp_get_params", [vp, vp]),
            ("fa_mlp_forward", [vp, vp, i64, vp, vp]),
            ("fa_mlp_pair_grad", [vp, vp, i64, vp, vp, vp, i64, vp, vp, vp]),
            ("fa_mlp_adam_step", [vp, ctypes.c_float, vp])):
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.fa_mlp_num_params.argtypes = []
    L.fa_mlp_num_params.restype = i64
    _lib = L
    return L


def check(rc: int) -> None:
    if rc != OK:
        msg = _lib.fa_last_error().decode() if _lib is not None else "?"
        raise FAError(rc, msg)
