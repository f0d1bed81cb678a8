"""GB300-native discrete DMK evaluation pass (arXiv 2308.00292).

The compute path lives in ``libdmk.so`` (CUDA kernels for sm_103a behind a C
ABI declared in ``include/dmk.h``); ``paper_2308_00292_gb300.dmk`` is the thin
ctypes binding.  Importing the package does not load the library.
"""
__all__ = ["dmk", "inputs"]
