"""GB300-native level-crossing-probability (LCP) maps of local divergence.

The library computes, for an ensemble of 2D vector fields on a uniform grid,
the probability that the divergence isocontour crosses each cell, under the
independent-Gaussian model of Ouermi et al. (arXiv 2510.01190, Sec. 3.1), plus
the classical Monte Carlo estimator it replaces (Sec. 3.2, Sec. 4).

All arithmetic runs in hand-written sm_103a CUDA kernels behind the C ABI in
``include/lcp.h``; this package only marshals arguments (``_binding``).  The
CUDA library is loaded on first use and its absence is an error: there is no
CPU fallback.
"""

from ._binding import *  # noqa: F401,F403
from ._binding import __all__  # noqa: F401
from . import surrogate  # noqa: E402,F401  (learned surrogate: moments, features, network kernels)
