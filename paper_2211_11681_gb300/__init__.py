"""GB300 (sm_103a) samplet S-format algebra: the masked product C = P_S(A B) of
samplet-compressed kernel matrices (Harbrecht, Multerer, Schenk, Schwab, arXiv 2211.11681,
Sec. 4.1), S-format addition, and the Newton-Schulz / Taylor scaling-and-squaring drivers
built on it.

The compute path is libsformat.so (CUDA, C ABI in include/sformat.h); ``sformat`` is its
Python binding.  ``build.build()`` compiles it in tree.
"""
__all__ = ["sformat", "build"]
