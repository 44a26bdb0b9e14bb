"""GB300-native Lindblad master-equation and quantum-trajectory solvers.

The compute path is the C-ABI library `_lib/libqtl.so` (hand-written sm_103a
CUDA, declared in include/qtl.h); `paper_2504_21440_gb300.qtl` is its thin
ctypes binding.  Nothing is imported here, so the package can be inspected
without a GPU.
"""
