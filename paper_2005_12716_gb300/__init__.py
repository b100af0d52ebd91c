"""GB300 (sm_103a) incident-wave reconstruction for the two-phase SWENSE method.

The compute path lives in the CUDA library ``libswense.so`` (C ABI in ``include/swense.h``);
``_swense`` is its ctypes binding and ``api`` a small torch-facing convenience layer that only
allocates device buffers and marshals arguments. There is no CPU fallback: every call goes to the
library, and importing ``api`` without the built library raises.
"""
from ._swense import SwenseError, load  # noqa: F401

__all__ = ["SwenseError", "load"]
