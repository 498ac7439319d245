"""GB300-native profiled incoherent dedispersion and boxcar S/N detection.

Implements the hot path of Clarke, Macquart & Trott, "Performance of a novel fast
transients detection system" (arXiv:1301.3968): the profiled dedispersion sum of
eq. p_dedisp with programmable per-channel delays, taps and weights, followed by
boxcar S/N detection (eq. snr), as hand-written sm_103a CUDA kernels behind the C ABI
of include/dd.h.  This package is the thin Python binding.
"""
from ._lib import DDError, LIB_PATH  # noqa: F401
from .api import (Band, Batch, DDFunction, Plan, alu_peak, candidates_to_list, detector_profile,  # noqa: F401
                  predict_rect, select_profiles, select_samples, trial_dms)

__all__ = ["Band", "Plan", "Batch", "DDFunction", "DDError", "alu_peak", "trial_dms", "candidates_to_list",
           "predict_rect", "select_samples", "select_profiles", "detector_profile"]
