"""GB300-native block-preconditioned VIE-FFT engine (arXiv 2501.13512).

Modules:
  inputs  seeded synthetic workloads (geometry + incidence), no method arithmetic
  build   compiles csrc/*.cu into libvie.so for sm_103a
  vie     ctypes binding of the C ABI declared in include/vie.h
The CUDA library is loaded lazily by ``vie.load()``.
"""
__version__ = "0.1.0"
