"""GB300 (sm_103a) streaming two-sided TT sketching: PSTT2 / PSTT2-onepass.

Shi, Ruth & Townsend, "Parallel algorithms for computing the tensor-train
decomposition" (Sec. 3.2, 4.2).  Every step of the path runs in the CUDA
library libttsketch.so behind the C ABI of include/ttsketch.h; this package is
its thin binding.  PyTorch is used only for device memory and streams.
"""
from . import _native
from ._native import (TT_F32, TT_F64, TT_PREC_BF16, TT_PREC_FP16, TT_PREC_FP64, TT_PREC_TF32, TTError,
                      check, lib, make_problem)
from .api import PSTT2Fn, TTReconstructFn, TTSketch, pstt2, tt2tucker, tucker2tt, x_scale_log2

__all__ = [
    "TTSketch", "PSTT2Fn", "TTReconstructFn", "pstt2", "tt2tucker", "tucker2tt", "x_scale_log2", "TTError", "lib",
    "make_problem", "check", "TT_F32", "TT_F64", "TT_PREC_FP64", "TT_PREC_TF32", "TT_PREC_BF16", "TT_PREC_FP16",
    "_native",
]
