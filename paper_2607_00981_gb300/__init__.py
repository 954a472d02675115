"""GB300-native RCCSDT residual path (compact triples storage) behind a C ABI.

``load()`` returns the ctypes handle of the in-tree CUDA library
``librccsdt.so``; ``Context`` (from ``binding``) wraps one problem.  There is no
CPU implementation in this package: without the built library or a CUDA
device the calls fail.
"""
from __future__ import annotations

import os

from . import binding
from .binding import Context, RccsdtError  # noqa: F401

_LIB = None


def library_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), binding.LIB_NAME)


def load(build_if_missing: bool = True):
    """Load librccsdt.so (building it in-tree first if it is missing)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"{path} is missing; run paper_2607_00981_gb300.build.build()")
            from .build import build
            build()
        _LIB = binding.load_library(path)
    return _LIB


def context(o: int, v: int, naux: int, stream: int = 0, **options) -> Context:
    """Create a Context on the CUDA library (raises if no CUDA device is usable)."""
    return Context(load(), o, v, naux, stream, **options)
