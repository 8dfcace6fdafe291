"""GB300-native (sm_103a) FFT-based rigid alignment of closed planar curves.

The method of Dogan, Bernal & Hagwood (arXiv 2501.17779): arc-length
resampling, then for every cyclic start point the optimal rotation in closed
form from the cross-correlation c(s) = sum_k z1[k] conj(z2[k+s]), evaluated
for all s with FFTs.  The kernels live in libfftalign.so (csrc/, C ABI in
include/fftalign.h); ``api`` is its Python binding.  Importing this package
does not load the library; the first call into ``api`` does.
"""
__version__ = "1.0.0"


def __getattr__(name):
    if name in ("align_pairs", "resample_arclength", "align_curves_host", "handle",
                "resample_workspace_size", "align_all_pairs"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
