"""GB300-native (sm_103a) semantic Bayesian kernel inference (S-BKI) map update.

The compute path is libsbki.so (hand-written CUDA, C ABI in include/sbki.h);
this package is its ctypes binding.  ``build.build()`` compiles it in-tree.
"""
from .sbki import (ERR_CAPACITY, ERR_CUDA, ERR_INVALID_ARG, ERR_LABEL_RANGE, ERR_NOT_FOUND, ERR_TIMEOUT,  # noqa: F401
                   EXPORTED, OK, Map, Params, SbkiError, Stats, default_params, forward_alpha, grad, library_path,
                   load, query_points, set_param, training_set_noalloc)

__all__ = ["Map", "Params", "Stats", "SbkiError", "default_params", "load", "library_path", "EXPORTED",
           "training_set_noalloc", "forward_alpha", "grad", "query_points", "set_param"]
