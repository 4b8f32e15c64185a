"""GB300-native replica-parallel Metropolis sweep with parallel tempering.

The compute path lives in the CUDA shared library built from ``csrc/`` and is
reached through :mod:`paper_1004_0024_gb300.ising` (a ctypes binding of the C
ABI declared in ``include/ising_gb300.h``).  Importing this package does not
load the library; importing ``ising`` does, and fails loudly when it is
missing.
"""
__all__ = ["workloads"]
__version__ = "0.1.0"
