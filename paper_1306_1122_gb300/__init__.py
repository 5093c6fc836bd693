"""GB300-native DBIE (direct boundary integral equation) NLFFF quadrature library.

The compute path is libdbie.so (hand-written CUDA for sm_103a behind the C ABI in
include/dbie.h); this package holds its ctypes binding and a PyTorch front end.  Importing the
package never falls back to a CPU path: if the library is missing, import fails.
"""
from . import _native  # noqa: F401  (raises ImportError when libdbie.so is missing)
from ._native import DBIEError  # noqa: F401
from .field import (QUAD_PIXEL_EXACT, DBIEField, Options, dbie_apply, dbie_solve_apply,  # noqa: F401
                    solve_batched)

__all__ = ["DBIEField", "Options", "dbie_apply", "dbie_solve_apply", "solve_batched", "DBIEError",
           "QUAD_PIXEL_EXACT"]
