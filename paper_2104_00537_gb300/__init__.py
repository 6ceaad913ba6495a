"""GB300-native WCSPH hot path (DualSPHysics paper, arXiv 2104.00537).

The compute path is the CUDA library ``libsph.so`` (built from ``csrc/``) behind
a C ABI declared in ``include/sph.h``; ``sph`` is its thin ctypes binding.
Importing this package does not load the library; ``sph.load()`` does.
"""
