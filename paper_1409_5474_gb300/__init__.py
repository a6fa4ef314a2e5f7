"""GB300-native direct-summation Hermite N-body core.

Submodules:
- ``ic``: seeded synthetic inputs (Plummer spheres, cluster batches, request streams);
- ``nbody``: ctypes binding of the C-ABI library ``libnbody.so`` (CUDA kernels for sm_103a);
- ``build``: compiles ``libnbody.so`` from ``csrc/``.

Importing the package loads nothing compiled; ``nbody`` loads the CUDA library
on first use and raises if it is missing.
"""
