"""Seeded synthetic workloads (supports, pivots, coefficients); no transform arithmetic."""
from .generators import *  # noqa: F401,F403
