"""GB300 (sm_103a) implementation of ROSEFusion's PFO/PST depth tracker hot path.

Zhang, Zhu, Zheng, Xu, "ROSEFusion: Random Optimization for Online Dense
Reconstruction under Fast Camera Motion", ACM TOG 40(4), 2021.

The compute path is librosefusion.so (hand-written CUDA behind the C ABI in
include/rosefusion.h); ``paper_2105_05600_gb300._native`` is its ctypes
binding, re-exported here on first use.  ``synth`` builds seeded synthetic
inputs and ``metrics`` computes ATE / TE on the host.
"""
from __future__ import annotations

import importlib

__all__ = ["synth", "metrics", "build", "learned"]


def __getattr__(name):
    if name in ("synth", "metrics", "build", "learned"):
        return importlib.import_module(f"{__name__}.{name}")
    native = importlib.import_module(f"{__name__}._native")
    try:
        return getattr(native, name)
    except AttributeError:
        raise AttributeError(f"module {__name__!r} has no attribute {name!r}") from None
