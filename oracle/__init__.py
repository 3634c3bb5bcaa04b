"""FP64 CPU oracle for the level-crossing-probability (LCP) map of local divergence.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously-correct
statement of what the GPU library computes, written from Ouermi et al.,
"Efficient Probabilistic Visualization of Local Divergence of 2D Vector Fields
with Independent Gaussian Uncertainty" (arXiv 2510.01190).  Only the test
suite, the smoke check in ``__graft_entry__`` and the CPU-baseline leg of
``bench.py`` may import it.  The product path (``paper_2510_01190_gb300``)
never imports, links or executes anything in here, and this package imports
nothing from the product: the two share no code.

Every public function cites the passage it follows.  See ``lcp_oracle`` for the
functions and the readings taken where the paper is silent.

Parity status
-------------
All functions are pinned by ``tests/test_oracle_pins.py`` against closed forms,
the paper's Fig. 2 worked example, exact rational arithmetic, brute-force
sampling with an independent random generator, and (for Philox4x32-10) an
independent open-source implementation.  ``exact_empirical_lcp`` is pinned by
brute-force enumeration on small ensembles.  ``surrogate`` (moments,
divergence cumulants, features, the network and Adam of the learned surrogate)
is pinned by ``tests/test_oracle_surrogate.py``: exact rational moments, the
divergence's exact distribution enumerated over every stencil combination,
hand-evaluated networks, a finite-difference gradient check and Adam's
first-step property.  ``viz`` (the colour map and the isocontour segments)
is pinned by ``tests/test_oracle_viz.py``: exact integer byte formulas on dyadic
inputs, the stops' own colours, special values, and marching squares against
hand-drawn cases and the crossing mask.  ``volume`` (the 3D extension) is
pinned by ``tests/test_oracle_volume.py``: exactness on linear fields, exact
rational arithmetic, the reduction of z-invariant fields to the 2D oracle, axis
permutation, and brute-force sampling with an independent generator.
"""

from .lcp_oracle import *  # noqa: F401,F403
from . import surrogate  # noqa: F401,E402
from . import viz  # noqa: F401,E402
from . import volume  # noqa: F401,E402
