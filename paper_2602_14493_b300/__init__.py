"""Gaussian Mesh Renderer (arXiv 2602.14493) hot path for B300 (sm_103a).

Mesh-to-Gaussian conversion (Sec. 2.2) fused with EWA projection, tile
binning sorted by (tile, depth, face), front-to-back alpha compositing, and
the hand-written backward pass, as CUDA kernels behind the C ABI of
include/gmr.h (libgmr.so, built in-tree). PyTorch supplies device memory and
streams only.
"""

from ._lib import GmrError, load as load_library
from .render import GMRRender, GMRRenderWithT, Renderer, camera_array, copy_h2d, pixel_offsets, render

__all__ = ["GMRRender", "GMRRenderWithT", "Renderer", "GmrError", "camera_array", "copy_h2d", "load_library",
           "pixel_offsets", "render"]
