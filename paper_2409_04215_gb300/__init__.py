"""GB300-native hot path of the recompleted MFS elastance and mobility solvers.

The compute runs in libmfs.so (hand-written CUDA for sm_103a, C ABI declared in
include/mfs.h).  This package is a thin ctypes binding with the same entry-point
names; importing it does not load the library -- the first call does, and fails
loudly when the library is missing.
"""

from .api import MFS, MFSError, SolveInfo, Options, load_library, mobility  # noqa: F401

__all__ = ["MFS", "MFSError", "SolveInfo", "Options", "load_library", "mobility"]
