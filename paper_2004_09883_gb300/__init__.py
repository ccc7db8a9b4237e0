"""GB300-native complex FFT function block (complex64 C2C, sm_103a CUDA).

The compute path is the C-ABI shared library ``libfbfft.so`` built from
``csrc/``; ``fbfft`` is its thin ctypes binding.  Importing this package does
not load the library: ``from paper_2004_09883_gb300 import fbfft`` does, and it
raises if the library is missing.
"""
__all__ = ["fbfft", "inputs"]
