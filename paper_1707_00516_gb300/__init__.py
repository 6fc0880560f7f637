"""GB300 (sm_103a) library for the FastID all-pairs SNP profile comparison of
arXiv:1707.00516: every unknown profile against every known one as an
overloaded matrix multiply, reduced on the device to per-query top-k or a
thresholded hit list.

The compute lives in ``libfastid.so`` (CUDA kernels behind the C ABI of
``include/fastid.h``); ``binding`` marshals torch tensors into it and
``search`` adds the host-buffer convenience path.
"""
from .binding import (EXPORTS, FORM_AUTO, FORM_PLAIN, FORM_TENSOR, MAX_K, MODE_MISMATCH, MODE_UNEXPLAINED,
                      NO_THRESHOLD, REFS_TENSOR, Context, FastIDError, RefDB, load_library)

__all__ = ["EXPORTS", "FORM_AUTO", "FORM_PLAIN", "FORM_TENSOR", "MAX_K", "MODE_MISMATCH", "MODE_UNEXPLAINED",
           "NO_THRESHOLD", "REFS_TENSOR", "Context", "FastIDError", "RefDB", "load_library"]
