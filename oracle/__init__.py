"""Plain FP64 CPU oracle for RT-DetMCD (De Ketelaere, Hubert, Raymaekers,
Rousseeuw, Vranckx, "Real-time outlier detection for large datasets by
RT-DetMCD", arXiv 1910.05615).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline leg of bench.py may import this package.  The product path (the
CUDA library and its Python binding) never imports, calls or links it, and it
shares no code, table or helper with that path.

The oracle follows the paper's steps in its own order and notation with plain
numpy/scipy primitives (sort, Cholesky, eigh, chi-squared distribution
functions) in float64.  Where the paper is silent or ambiguous the reading
taken is stated at the function that implements it.
"""
from .rtdetmcd import *  # noqa: F401,F403
