"""GB300 (sm_103a) implementation of the Gaussian-Splatting periphery fit step.

The CUDA kernels live in csrc/ behind the C ABI of include/gsfit.h and are
built in-tree into _lib/libgsfit.so; gsfit.py is the thin ctypes binding and
fit.py drives one fit iteration (and its CUDA graph) from PyTorch-owned
device buffers. There is no CPU fallback: calls fail if the library is
missing.
"""
from ._build import build as build_library
from . import gsfit
from .gsfit import load


def build(force: bool = False) -> None:
    build_library(force=force)
    load()


__all__ = ["build", "build_library", "gsfit", "load"]
