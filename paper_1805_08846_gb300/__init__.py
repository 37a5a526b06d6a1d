"""GB300-native dimension-split wave-propagation step (CUDACLAW, arXiv 1805.08846).

``Solver`` / ``Ensemble`` wrap the C ABI of ``include/claw.h``; the CUDA
library is built in-tree by ``paper_1805_08846_gb300.build``.  Importing this
package does not load the library; the first solver call does, and raises if
it cannot.
"""
from .solver import Ensemble, Solver  # noqa: F401
from ._lib import ClawError  # noqa: F401
