"""GB300-native DDG two-level Schwarz PCG (Edwards & Bridson, arXiv 1504.00907).

The numerical work runs in ``libddg.so`` (hand-written sm_103a CUDA kernels
behind the C ABI of ``include/ddg.h``); :mod:`.ddg` is its Python binding.
Importing the package does not load the library; ``ddg.load()`` does.
"""
__all__ = ["ddg", "build"]
