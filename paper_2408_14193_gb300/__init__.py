"""GB300 (sm_103a) implementation of the recursive sparse LU fast direct solver (spaLU).

The compute path lives in the CUDA library built from ``csrc/`` into ``_build/libspalu.so``
(C ABI: ``include/spalu.h``); ``spalu`` is a thin ctypes binding with the same names.
"""
from .spalu import (BatchGraph, Factor, NestedDissection, Options, Predictor, SpaluError, factor_batch,
                    library_path, load_library, solve_batch, status_string)

__all__ = ["BatchGraph", "Factor", "NestedDissection", "Options", "Predictor", "SpaluError", "factor_batch",
           "library_path", "load_library", "solve_batch", "status_string"]
