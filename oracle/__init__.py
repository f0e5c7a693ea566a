"""FP64 CPU oracle of the 3DGS rasterizer + SkipGS gate.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline / reference arm may import this package; the product path
never does, and the two share no code.

* ``gs_oracle.c`` (built into ``liboracle.so``): projection (Eq. cov, Eq. proj,
  SH colour), tile binning and the stable key sort, tiled and brute-force
  compositing (Eq. blend, Eq. alpha) and the analytic adjoint.
* ``loss.py``: Eq. (loss), L = (1-lambda) L1 + lambda (1 - SSIM), lambda = 0.2,
  and its gradient.
* ``adam.py``: Adam (Kingma & Ba), as the paper's optimizer.
* ``gate.py``: Algorithm 1 (SkipGS gating) with Eq. (view-ema), (deviation),
  (gate), (rhocum), (rhocum_check), (rhohat), (rhomincalib).
"""
from .core import (  # noqa: F401
    RasterConfig, build, lib, project, bin_sort, render, render_brute, raster_bwd, project_bwd,
    forward, backward, sh_basis, num_threads, set_num_threads, camera_struct, tile_grid,
)
from .loss import loss_and_grad, ssim_map, gaussian_window  # noqa: F401
from .adam import AdamConfig, adam_step, param_groups  # noqa: F401
from .gate import GateConfig, Gate  # noqa: F401
