"""GB300-native recursive Green-function (KNIT slice-sweep) transport library.

The compute path is the C-ABI library ``libknit`` (hand-written CUDA for
sm_103a, declared in ``include/knit.h``); ``paper_1010_2627_gb300.knit`` is its
thin ctypes binding.  ``paper_1010_2627_gb300.inputs`` builds synthetic
lattices and instance lists.  Importing the package loads nothing; the
binding loads the library on first use and fails loudly if it is missing.
"""
__all__ = ["inputs", "knit"]
