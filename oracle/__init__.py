"""FP64 CPU oracle for the generalized radix-2 transform.

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the bench's
CPU-baseline leg; never by the library. See `oracle/fp64.py`.
"""
from .fp64 import *  # noqa: F401,F403
