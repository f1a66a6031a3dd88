"""GB300-native single-GPU state-vector simulator (libqsim) and its Python binding.

The compute path is the C-ABI library ``_build/libqsim.so`` (hand-written sm_103a CUDA kernels); the
binding in ``qsim`` only marshals arguments. Importing this package does not load the library; the
first call that needs it does (building it with nvcc when missing).
"""
from . import qsim  # noqa: F401

__all__ = ["qsim"]
