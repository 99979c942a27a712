"""GB300 (sm_103a) implementation of SecPE's encrypted prompt-ensemble
aggregation and encrypted Argmax on RNS-CKKS (arXiv 2502.00847).

The compute path is the CUDA library libsecpe.so (C ABI in include/secpe.h);
`secpe` is its ctypes binding.  Importing this package does not load the
library; `secpe.lib()` does, and raises if it is not built.
"""
