"""libsgrcolor: data-driven speculative-greedy graph coloring on GB300 (sm_103a).

The hot path is the C-ABI library built from ``csrc/`` (see
``include/sgrcolor.h``); ``paper_1606_06025_gb300.sgrcolor`` is its thin
Python binding.  Importing the binding loads (and if needed builds) the
library; there is no CPU fallback.
"""
