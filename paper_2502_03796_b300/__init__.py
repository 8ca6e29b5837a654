"""B300-native replay of the MAGUS uncore-frequency control step (arXiv 2502.03796).

The compute path is libmagus.so (hand-written CUDA for sm_103a behind the C ABI in
include/magus.h); ``magus`` is its ctypes binding.
"""
from . import magus  # noqa: F401
from .magus import MagusError, Replay, lib  # noqa: F401

__all__ = ["magus", "Replay", "MagusError", "lib"]
