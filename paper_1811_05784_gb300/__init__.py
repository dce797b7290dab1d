"""GB300-native batched ray propagation for hybrid ray-tracing / image-source
room acoustics (Aussal & Gueguen 2018, arXiv:1811.05784).

The compute path is the CUDA library libroomrays.so (C ABI in
include/roomrays.h); ``rt`` is its thin Python binding.
"""
from . import rt  # noqa: F401
from .rt import (RtError, rt_api_version, rt_build_tree, rt_last_error, rt_rir,  # noqa: F401
                 rt_set_allocator, rt_trace)

__all__ = ["rt", "RtError", "rt_build_tree", "rt_trace", "rt_rir", "rt_last_error", "rt_api_version",
           "rt_set_allocator"]
