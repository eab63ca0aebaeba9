"""GB300-native DCT-based t-SVD / t-SVT / TNN-C completion (arXiv 1902.03070).

The compute path is the C-ABI library libtnn.so (hand-written sm_103a CUDA
kernels); `paper_1902_03070_gb300.tnn` is its thin ctypes binding.  There is no
CPU fallback: importing the binding fails loudly when the library is missing.
"""
__all__ = ["inputs"]
