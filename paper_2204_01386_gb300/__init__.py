"""GB300-native HardSoftRas (the soft rasterizer of arXiv 2204.01386, Sec. 3.4):
forward and hand-written adjoint as CUDA kernels for sm_103a behind a C ABI
(include/dressi.h), with a thin Python binding."""
from .binding import DressiError, load  # noqa: F401
from .render import DressiFn, PackedScene, Renderer, decode_layer_ids, make_params, make_views, render  # noqa: F401

__all__ = ["DressiError", "DressiFn", "PackedScene", "Renderer", "decode_layer_ids", "load", "make_params", "make_views",
           "render"]
