"""GB300-native polyhedral-homotopy path tracking (hot path of T. Chen,
"GPU-accelerated path tracker for polyhedral homotopy").

The compute path is libhpt.so (CUDA for sm_103a behind the C ABI in
include/hpt.h); ``paper_2111_14317_gb300.hpt`` is its Python binding.  Build
the library with ``paper_2111_14317_gb300.build.build()``.
"""
__all__ = ["build", "hpt"]
