"""GB300-native Gaussian Belief Propagation for bundle adjustment.

The compute path is the CUDA library ``libgbp.so`` (C ABI in
``include/gbp.h``); ``gbp`` is its thin Python binding and ``synth`` the
seeded synthetic-problem generator.
"""
from . import synth  # noqa: F401
