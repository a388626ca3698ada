"""dtwgb: all-pairs windowed DTW and k-medoids on GB300 (sm_103a).

After "Fast dynamic time warping and clustering in C++" (arXiv 2307.04904).
The computation lives in the CUDA library built from ``csrc/`` (C ABI in
``include/dtwgb.h``); ``api`` is its Python binding and ``synth`` makes seeded
synthetic inputs.  Importing the package does not load the library: the first
call does, and raises if it has not been built.
"""

from .api import (DTWError, dtw_pairwise, dtw_pairwise_host, dtw_query,  # noqa: F401
                  kmedoids_fit, load)

__all__ = ["DTWError", "dtw_pairwise", "dtw_pairwise_host", "dtw_query", "kmedoids_fit", "load"]
