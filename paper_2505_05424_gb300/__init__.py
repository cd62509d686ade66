"""GB300-native (sm_103a) inexact proximal ALM for staggered-grid dynamic optimal transport.

The solver itself lives in the CUDA library behind the C ABI declared in
include/dot.h; this package holds its thin Python binding and the seeded
synthetic-input generators.  Importing the package does not load the CUDA
library; the first solver call does, and fails loudly when it is missing.
"""
__all__ = ["workloads"]
