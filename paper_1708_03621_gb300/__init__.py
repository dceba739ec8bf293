"""GB300-native plane-wave Hamiltonian hot path (JDFTx method, arXiv:1708.03621).

The compute path is libjdft.so (hand-written sm_103a CUDA behind the C ABI in
include/jdft.h); ``jdft`` is its ctypes binding.  Build with
``python -m paper_1708_03621_gb300.build``.
"""
from . import jdft  # noqa: F401
