"""GB300-native propagation of the hierarchical equations of motion (HEOM) for
excitonic energy transfer with trapping, after Kreisbeck et al.,
arXiv:1012.4382.

The compute path is the C-ABI library ``libheom.so`` (CUDA kernels for
sm_103a); :mod:`paper_1012_4382_gb300.heom` is its thin ctypes binding.
Importing the package does not load the library; the binding loads it on
first use and raises if it is missing.
"""
__all__ = ["heom", "workloads"]
