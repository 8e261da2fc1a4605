"""GB300-native rule-based blocking (matching dependencies) behind the libhb C-ABI.

The compute path is libhb.so (hand-written sm_103a CUDA kernels); ``hb`` is
its ctypes binding.  Build the library with ``build.build()``.
"""
from . import hb
from .hb import Context, HBError, plan_order

__all__ = ["hb", "Context", "HBError", "plan_order"]
