"""GB300 (sm_103a) library for the RPA polarization chi0_GG'(q, w) and screened
interaction W of RESPACK (arXiv 2001.02351), with a thin Python binding.

The compute path is the C-ABI shared library librespack_gb300.so (include/respack_gb300.h);
this package only marshals arguments.  Build it with `paper_2001_02351_gb300.build.build()`.
"""
from ._lib import (Context, RPError, context_for, library, probe_peaks, EXPORTS, RP_OK, RP_ERR_ARG, RP_ERR_STATE,
                   RP_ERR_OOM, RP_ERR_CUDA, RP_ERR_NUMERIC, RP_ERR_TIMEOUT, RP_ERR_UNSUPPORTED,
                   RP_FP64_NATIVE, RP_FP64_EMULATED, RP_TF32X3, RP_BF16X3, RP_AXIS_REAL, RP_AXIS_IMAG,
                   RP_TIME_ORDERED, RP_RETARDED, TILE_WIDTHS)

__all__ = ["Context", "RPError", "context_for", "library", "probe_peaks", "EXPORTS", "RP_OK", "RP_ERR_ARG", "RP_ERR_STATE",
           "RP_ERR_OOM", "RP_ERR_CUDA", "RP_ERR_NUMERIC", "RP_ERR_TIMEOUT", "RP_ERR_UNSUPPORTED",
           "RP_FP64_NATIVE", "RP_FP64_EMULATED", "RP_TF32X3", "RP_BF16X3", "RP_AXIS_REAL", "RP_AXIS_IMAG",
           "RP_TIME_ORDERED", "RP_RETARDED", "TILE_WIDTHS"]
