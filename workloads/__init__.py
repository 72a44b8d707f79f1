"""Seeded synthetic inputs and plain configuration numbers.

This module is shared by the tests, the benchmark, the oracle-driven checks and
users of the library.  It holds no arithmetic of the method itself: only the
workload shapes (mesh sizes, physical parameters, boundary states) and seeded
macroscopic initial fields (density, velocity, temperature) evaluated at node
coordinates passed in by the caller.  Random numbers come from numpy's Philox
counter-based generator so every consumer receives identical arrays.
"""
from .configs import CONFIGS, get_config  # noqa: F401
from .fields import initial_fields  # noqa: F401
