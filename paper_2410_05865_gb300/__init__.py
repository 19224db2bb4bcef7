"""GB300-native fourth-order cut-cell multigrid Poisson solver (arXiv 2410.05865).

The solver lives in ``libccmg.so`` (C ABI: ``include/ccmg.h``); ``ccmg`` is its
Python binding.  Build with ``paper_2410_05865_gb300.build.build()``.
"""
__all__ = ["ccmg", "build"]
