"""GB300-native shaken dynamics (arXiv:1908.07341): the synchronous half-step
of the probabilistic cellular automaton as hand-written sm_103a CUDA behind a
C ABI (include/shaken.h), with a thin Python binding.

The library must be built (``__graft_entry__.build()``); there is no CPU
fallback.
"""
from ._lib import (BITPACK, INIT_ALL_DOWN, INIT_ALL_UP, INIT_RANDOM, INT8, NOBS, ShakenError,
                   lib)
from .lattice import (Lattice, alloc_plane, halfstep, init_plane, lattice_bytes, pack_bits,
                      plane_bytes, specialize, specialize_status, thresholds, unpack_bits,
                      wait_specialized)

__all__ = ["BITPACK", "INT8", "INIT_ALL_UP", "INIT_ALL_DOWN", "INIT_RANDOM", "NOBS", "ShakenError",
           "Lattice", "alloc_plane", "halfstep", "init_plane", "lattice_bytes", "pack_bits",
           "plane_bytes", "specialize", "specialize_status", "thresholds", "unpack_bits",
           "wait_specialized", "lib"]
