"""GB300 (sm_103a) library for the hot path of HICU (calibrationless MRI).

The computation lives in libhicu.so (CUDA C++, C ABI in include/hicu.h);
``hicu`` is its thin ctypes binding and ``autograd`` wraps the convolution
pair as a torch.autograd.Function.  Build with ``python -m
paper_2004_08962_gb300.build``.
"""
from . import hicu  # noqa: F401
