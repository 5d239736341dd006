"""usFFT sampling-and-detection on one GB300 GPU (sm_103a).

The compute path is the CUDA library ``libusfft.so`` (C ABI declared in include/usfft.h);
``binding`` marshals arguments to it through ctypes.  Importing this package loads
nothing: the library is loaded on first use and a missing library is an error (there is
no CPU fallback).
"""
__all__ = ["binding"]
