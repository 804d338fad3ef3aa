"""GB300-native (sm_103a) implementation of the hot path of the deep-learning-guided memetic
graph colouring method DLMCOL (Goudet, Grelier, Hao, arXiv 2109.05948).

The compute lives in the CUDA library ``libdlmcol.so`` (sources in ``csrc/``, C-ABI in
``include/dlmcol.h``); ``paper_2109_05948_gb300.dlmcol`` is its thin ctypes binding.
"""
__all__ = ["inputs", "dlmcol"]
