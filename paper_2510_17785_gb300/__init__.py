"""GB300 vertex-patch smoother with a nested matrix-free p-multigrid local solver.

The compute path is libpmg.so (hand-written sm_103a CUDA behind the C ABI in
include/pmg.h); ``pmg`` is its ctypes binding, ``inputs`` the seeded synthetic
workload generator.  Importing the package does not load the library.
"""
__all__ = ["pmg", "inputs", "build"]
