"""GB300-native (sm_103a) differentiable rasterizer for composed, editable 3D Gaussians.

The path of iVR-GS (arXiv 2504.17954): composition and edits (Sec. 4.5, 4.6), EWA projection
with Blinn-Phong shading (Sec. 3, Sec. 4.3), tile binning by radix sort, front-to-back
compositing (Sec. 3), and its reverse mode. The compute lives in libivrgs.so (CUDA, C ABI in
include/ivrgs.h); this package marshals arguments to it.
"""
from . import _native
from ._native import IvrgsError
from .rasterizer import (Gaussians, Rasterizer, RenderFunction, camera_structs, compose_edit, pack_mixed, render,
                         reorder_spatial, vq_compress)

__all__ = ["_native", "IvrgsError", "Gaussians", "Rasterizer", "RenderFunction", "camera_structs", "compose_edit",
           "pack_mixed", "render", "reorder_spatial", "vq_compress"]
