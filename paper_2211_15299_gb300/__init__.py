"""GB300-native generalized radix-2 transform for homogeneous frequency supports.

The transform of arxiv 2211.15299 (Algorithm 1, the Hi-DFT): given N = 2^M, a
homogeneous support J of k = 2^s frequencies and the k samples of f on the
pivoted sampling pattern I_r, return the k DFT coefficients (F f)_J.

The compute path is the CUDA library libsdft.so (C ABI in include/sdft.h);
`_native` binds it with the same function names and `Plan` wraps a plan.
"""
from __future__ import annotations

from . import _native
from ._native import *  # noqa: F401,F403  (C-ABI names)
from .api import Plan, Batch, Server, Sas, execute_batched  # noqa: F401

__all__ = ["Plan", "Batch", "Server", "Sas", "execute_batched"] + [n for n in _native.SIGNATURES]
