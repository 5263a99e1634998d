"""GB300-native DNN-SP2-PT: density matrix and first-order response on sm_103a.

The computation lives in libdmpt.so (CUDA kernels behind the C ABI of
include/dmpt.h); ``dmpt`` is its ctypes binding.  Import is light: the
library is loaded on first use.
"""

__all__ = ["dmpt", "workloads"]
