"""GB300-native encrypted sparse x sparse matmul (CKKS SpMSpM, CSR x CSC).

The compute path is the C-ABI library libspfhe.so (sm_103a CUDA kernels,
declared in include/spfhe.h); `paper_2604_11659_gb300.spfhe` is its thin
ctypes binding.  Submodules load lazily so that `synthetic` (plaintext
workload generators) can be imported without a GPU.
"""
__all__ = ["spfhe", "synthetic"]
