"""GB300-native EC-ElGamal plaintext-ciphertext matrix multiplication.

The compute path is the C-ABI CUDA library ``libpcmm.so`` (sources in
``csrc/``, declarations in ``include/pcmm.h``); ``pcmm`` is its thin ctypes
binding.  Importing this package loads nothing: ``pcmm.lib()`` loads the
library on first use and raises if it has not been built.
"""
__all__ = ["pcmm", "inputs"]
