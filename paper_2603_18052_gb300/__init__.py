"""GB300-native dense small-d Lindblad propagation.

The compute path is liblb.so (CUDA C++ for sm_103a behind the C ABI in
include/lb.h); ``paper_2603_18052_gb300.lb`` is its ctypes binding.
"""

from . import _build  # noqa: F401

__all__ = ["lb", "accounting"]
