"""GB300-native image-source-method RIR simulation (arXiv 1810.11359).

The compute path is the C-ABI CUDA library ``libism`` (csrc/, include/ism.h);
``paper_1810_11359_gb300.ism`` is the thin ctypes binding over it.  Importing
the package does not load the library; the first call does, and raises if the
library has not been built (there is no CPU fallback).
"""
__all__ = ["ism", "workloads"]
