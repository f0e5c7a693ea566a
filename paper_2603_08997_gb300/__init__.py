"""GB300 (sm_103a) implementation of the 3DGS rasterizer inside the
post-densification refinement loop, with the SkipGS per-view backward gate.

Compute lives in libgsr.so (CUDA kernels behind the C ABI in include/gsr.h);
`gsr` is the ctypes binding, `raster` the buffers and call sequence,
`refine` the gated loop, `autograd` the torch.autograd.Function wrapper.
"""
from . import gsr  # noqa: F401
from .raster import AdamState, Gate, GaussianModel, RasterSettings, Renderer, Views  # noqa: F401
