"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This package draws random scenes, cameras and view sequences only.  It holds
none of the method's arithmetic (no projection, blending, loss, gradient or
gate step), so both sides of every parity test can consume it.
"""
from .scenes import (  # noqa: F401
    Camera, Scene, sh_coeff_count, dc_from_rgb,
    camera_pinhole, camera_look_at, ring_cameras,
    scene_cube, scene_ball, perturb_scene, scene_tiny, sparse_start,
    case_c1, case_c2, case_c3, case_c4, case_c4_ring, case_c5, view_sequence,
    C4_RESOLUTIONS, projected_records, opaque_stack_records, dl_dimage, pre_sequence,
)
