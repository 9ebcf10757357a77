"""GB300-native MG-GLAM derivative-coupling field solvers (arXiv:2110.00566).

The compute path is the CUDA library ``libmgglam.so`` built from ``csrc/``
for sm_103a; ``binding`` is a thin ctypes layer over its C-ABI.  Importing
this package does not load the library; the first call into ``binding``
does, and raises if the library is missing -- there is no CPU fallback.
"""
__all__ = ["binding", "inputs"]
