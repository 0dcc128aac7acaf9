"""GB300-native spectral D-bar CGO solver (Klein & McLaughlin, arXiv 1508.02363).

The compute path is the CUDA library ``libdbar_gb300.so`` (C ABI in
``include/dbar.h``); ``paper_1508_02363_gb300.dbar`` is its Python binding.
Build the library with ``python -m paper_1508_02363_gb300.build``.
"""
__all__ = ["build", "dbar"]
