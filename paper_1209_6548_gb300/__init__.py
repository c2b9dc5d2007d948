"""GB300-native lattice ES-BGK solver (arXiv 1209.6548): the fused per-time-step
update of one distribution function on a Gauss-Hermite velocity set, as
hand-written sm_103a CUDA behind the C ABI of include/lesbgk.h.

``lesbgk`` is the ctypes binding (argument marshalling only), ``build``
compiles the library in-tree, ``inputs`` draws the seeded synthetic workloads.
"""
from . import build, inputs, lesbgk  # noqa: F401
from .lesbgk import Solver  # noqa: F401
