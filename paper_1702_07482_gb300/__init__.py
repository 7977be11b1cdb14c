"""GB300 (sm_103a) implementation of the TRDMD despeckling stage.

The compute path is libtnrd.so (CUDA kernels behind the C ABI of
include/tnrd.h); `binding` is its ctypes binding and `ops` marshals torch
tensors into it.  `build.build()` compiles the library in-tree.
"""
from . import binding  # noqa: F401

__all__ = ["binding", "ops", "build"]
