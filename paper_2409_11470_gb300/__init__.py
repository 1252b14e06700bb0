"""GB300-native hot path of adaptive particle refinement (APR) for compressible SPH.

Nealon & Price, arXiv 2409.11470.  The computation lives in the CUDA library
``libapr.so`` (sources in ``csrc/``, C ABI in ``include/apr.h``); this package
builds it (``build``) and binds it (``binding``).  Importing ``binding`` fails
loudly if the library has not been built.
"""
__all__ = ["build", "binding"]
