"""Batched LAD-LASSO coordinate descent for one GB300 (sm_103a).

The compute path is the CUDA library `libladlasso.so` built from `csrc/`;
`ladlasso.py` is its ctypes binding (argument marshalling only).  There is
no CPU fallback: calls fail loudly when the library is not built.
"""
