"""GB300-native numeric sparse LU (Gilbert-Peierls over BTF + nested dissection).

The compute path is the CUDA library ``libbasker_gb300.so`` reached through the
C ABI in ``include/basker.h``; ``paper_1601_05725_gb300.basker`` is its thin
binding.  Importing this package loads nothing: the library is loaded on first
use and a missing library is an error, never a fallback.
"""
__all__ = ["inputs", "basker"]
