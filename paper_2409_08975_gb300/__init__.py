"""GB300-native temporal 3-path sampling for temporal motif counts.

Implements the estimator of Pu et al., "Accurate and Fast Estimation of
Temporal Motifs using Path Sampling" (ICDM 2024) as CUDA kernels for sm_103a
behind the C ABI in include/tc.h; ``tc`` is its Python binding.
"""
from . import tc  # noqa: F401
