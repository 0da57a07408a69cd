"""GB300-native checkerboard-Metropolis Ising engine (2D square / 3D cubic,
J = 1, h = 0, periodic), after Tomov et al. (2003), Sec. 2.2.

The simulation runs in hand-written CUDA kernels for sm_103a behind the C ABI
of ``include/ising.h``; ``engine`` is its Python binding.  There is no CPU
fallback: without the compiled library, ``engine.load_library()`` raises.
"""
from .engine import (AUTO, BITPACK, COLD_DOWN, COLD_UP, HOT, INT8, RULE_DEMON,  # noqa: F401
                     RULE_HEATBATH, RULE_METROPOLIS, RULE_MULTIHIT, Batch, IsingError, Lattice,
                     batch_run, batch_run_static, load_library, observables_gather)

__all__ = ["Lattice", "Batch", "IsingError", "load_library", "INT8", "BITPACK", "AUTO", "HOT",
           "COLD_UP", "COLD_DOWN", "RULE_METROPOLIS", "RULE_HEATBATH", "RULE_DEMON", "RULE_MULTIHIT",
           "batch_run", "batch_run_static", "observables_gather"]
