"""hegpu: homomorphic convolution and average pooling over RNS-CKKS ciphertexts holding a
row-major packed image sharded across several ciphertexts, on one GB300 (sm_103a).

The compute path is the C-ABI library libhegpu.so (include/hegpu.h); `hegpu` is its thin
ctypes binding.  Build with ``python -m paper_2306_09189_gb300.build``.
"""
from . import hegpu  # noqa: F401
