"""FP64 CPU oracle for the generalized radix-2 transform and Shift-and-Sample.

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the bench's
CPU legs; never by the library. See `oracle/fp64.py` and `oracle/sas.py`.
"""
from .fp64 import *  # noqa: F401,F403
from .sas import *  # noqa: F401,F403
