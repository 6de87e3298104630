"""GB300-native Wilson-Dirac conjugate gradient (arXiv 2111.14958 hot path).

The compute path is the CUDA library ``libwdcg.so`` (C ABI in ``include/wd.h``), bound through
:mod:`paper_2111_14958_gb300.wd`. Importing :mod:`paper_2111_14958_gb300.wd` raises if the library
is not built; nothing here falls back to the CPU.
"""
__all__ = ["wd", "build"]
