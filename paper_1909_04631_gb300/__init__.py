"""GB300-native (sm_103a) semantic Bayesian kernel inference (S-BKI) map update.

The compute path is libsbki.so (hand-written CUDA, C ABI in include/sbki.h);
this package is its ctypes binding.  ``build.build()`` compiles it in-tree.
"""
from .sbki import (EXPORTED, Map, Params, SbkiError, Stats, default_params, library_path,  # noqa: F401
                   load)

__all__ = ["Map", "Params", "Stats", "SbkiError", "default_params", "load", "library_path", "EXPORTED"]
