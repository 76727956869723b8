"""GB300-native hierarchical-GMM point-cloud registration (arXiv 1807.02587).

The compute path is the CUDA library ``_lib/libhgmm.so`` (sources under
``csrc/``, C ABI in ``include/hgmm.h``); ``binding`` is its thin ctypes
binding and ``synth`` the seeded synthetic inputs.  Importing ``binding``
requires the compiled library; this package module itself imports nothing
heavy so that the input generators stay usable without it.
"""
__all__ = ["binding", "synth", "build_ext"]
