"""Certified quantization-based bounds on the p-Wasserstein metric for GB300.

The computation lives in ``libqwb.so`` (CUDA kernels for sm_103a plus a host
network simplex) behind the C ABI of ``include/qwb.h``; ``api`` is its Python
binding (``from paper_2506_00976_gb300 import api``).  Importing the package
does not load the library; the first call does, and raises if it is not built.
"""
