"""GB300-native implementation of V3DG's online per-frame path (LOD-cut selection + splatting).

The compute path is the CUDA library ``libv3dg.so`` (C ABI in include/v3dg.h); this package is its
Python binding.  PyTorch is used only for device memory (the library's allocator callback) and
streams.
"""
from .api import Context, camera_struct, hierarchy_struct  # noqa: F401
from ._native import V3dgError  # noqa: F401
