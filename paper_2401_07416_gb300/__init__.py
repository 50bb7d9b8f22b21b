"""GB300-native FDTD leapfrog for the 3-D time-dependent Schrodinger equation.

The compute path is ``libtdse.so`` (CUDA for sm_103a behind a C ABI declared in
``include/tdse.h``); ``tdse`` is its thin ctypes binding with the same function
names, and ``sim`` wraps it for PyTorch users.  Importing this package loads
nothing: the library is opened on first use and fails loudly if it is missing.
"""

__all__ = ["workloads"]
