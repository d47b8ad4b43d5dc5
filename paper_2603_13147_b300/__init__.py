"""LLP sweep engine for NVIDIA B300 (sm_103a).

The library itself is libllp.so (C ABI in include/llp.h, CUDA sources in
csrc/); this package is its thin Python binding.
"""
from .binding import *  # noqa: F401,F403
from .binding import lib, version  # noqa: F401


def build(force: bool = False) -> str:
    from ._build import build as _b
    return _b(force=force)
