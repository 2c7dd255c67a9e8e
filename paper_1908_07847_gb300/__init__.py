"""GB300-native training of the one-hidden-layer sigmoid network of arXiv 1908.07847.

The compute path is a C-ABI shared library of hand-written sm_103a CUDA kernels
(``csrc/``, declared in ``include/mlp_gb300.h``); ``binding`` wraps it with the
same names.  Importing this package does not load the library; ``binding.lib()``
does, and raises if it has not been built.
"""
__all__ = ["binding", "inputs"]
