"""GB300-native parallel replica (ParRep) dynamics for bistable reaction networks.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/parrep.h``); ``api`` is its thin Python binding.  Nothing here
falls back to the CPU.
"""
from .api import ParRep, ParRepBatch, ParRepError, ParRepServer, parrep_philox, parrep_ssa, parrep_uq  # noqa: F401

__all__ = ["ParRep", "ParRepBatch", "ParRepServer", "ParRepError", "parrep_ssa", "parrep_philox", "parrep_uq"]
