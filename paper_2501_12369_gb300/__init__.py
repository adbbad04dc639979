"""GB300 (sm_103a) differentiable tile rasterizer for DARB splats (arxiv 2501.12369).

The compute path is libdarb.so (CUDA, C ABI in include/darb.h); this package holds its
build script, the ctypes binding (``darb``) and the seeded input generators (``synth``).
"""
from . import synth  # noqa: F401

__all__ = ["synth", "darb", "build"]
