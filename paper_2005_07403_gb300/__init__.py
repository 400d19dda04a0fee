"""GB300-native batched 2x2 SVD (Novakovic, arXiv 2005.07403).

The compute path is a CUDA shared library for sm_103a with a C ABI
(``include/svd2.h``); ``paper_2005_07403_gb300.svd2`` is its thin Python
binding.  Importing the package loads nothing: the library is loaded on the
first call, and a missing library is an error (there is no CPU fallback).
"""
__all__ = ["inputs"]
