"""B300-native forward/adjoint of the Pauli-measurement oracle of rank-adaptive
matrix-free atomic quantum state tomography.

The compute path is the C-ABI library ``libqst.so`` (hand-written sm_103a CUDA,
declared in ``include/qst.h``); ``paper_2607_19577_b300.qst`` is its thin
ctypes binding.  Importing this package loads nothing; ``qst`` loads the
library on first use and fails loudly if it is missing.
"""
__all__ = ["qst", "synth"]
