"""GB300-native ROM-based inexact FETI-DP hot path for lattice structures.

The compute path lives in the CUDA shared library built from ``csrc/``
(C ABI declared in ``include/fetidp.h``); :mod:`.binding` marshals
arguments to it.  Importing this package has no side effects: the
library is loaded on first use of :mod:`.binding`.
"""

__all__ = ["workloads", "binding"]
