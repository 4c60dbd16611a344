"""afft: a single-GPU (GB300, sm_103a) 3-D FFT library after AccFFT's pencil stages.

The compute path lives in the CUDA shared library built from ``csrc/``; the
``afft`` module is its ctypes binding (argument marshalling only).  Importing
this package does not load the library; the first call into ``afft`` does,
and raises if it is missing -- there is no CPU fallback.
"""
__all__ = ["afft", "synth"]
