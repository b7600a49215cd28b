"""GB300-native parallel-in-time continuous-time MAP trajectory estimation.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/map_smoother.h``); this package holds its build driver, the ctypes
binding (``_binding``), a PyTorch-facing wrapper (``MapSmoother``) and the
seeded synthetic workloads (``synth``).
"""
from __future__ import annotations

__all__ = ["MapSmoother"]


def __getattr__(name):
    if name == "MapSmoother":
        from .smoother import MapSmoother
        return MapSmoother
    raise AttributeError(name)
