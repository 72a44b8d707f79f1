"""GB300-native semi-Lagrangian lattice Boltzmann (SLLBM) hot path.

The compute path is the CUDA library libsllbm.so (include/sllbm.h); this
package only builds it (``build``), binds it (``capi``) and wraps a context
(``sim.Sim``).  There is no CPU fallback.
"""
from .capi import SllbmError, lib  # noqa: F401
