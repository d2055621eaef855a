"""GB300-native batched time-domain LISA log-likelihood (arXiv:2501.08261).

The compute path is the C-ABI CUDA library built from ``csrc/`` (sm_103a);
``api`` is a thin ctypes binding with the same entry-point names.
"""
