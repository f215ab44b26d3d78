"""Seeded synthetic inputs for the k-shell renderer.

This package only *makes inputs*: nested triangle-mesh shells with UVs, texel
arrays and pinhole cameras.  It contains none of the renderer's arithmetic
(no projection, rasterization, sampling, SH evaluation or compositing), so the
CUDA path and the CPU oracle can both be fed from it without sharing code.

The paper's scenes (Shelly, DTU, custom captures) and its baked assets are not
available; these generators stand in for them with the same structure: k
nested, smooth, closed shells around a unit-size object, UV atlases, SH
textures and views on a hemisphere or sphere (Sec. 3 "Support Surfaces as
Shells", Sec. 3 "Texturing Meshes", Sec. 4 Tab. 2).
"""

from .scenes import (  # noqa: F401
    FMT_RGBA_F32,
    FMT_SH_F16,
    FMT_SH_U8,
    BAKED_STRIDES,
    baked_layout,
    baked_values_to_bytes,
    baked_sh_texture,
    ntex_init,
    Camera,
    Shell,
    Scene,
    icosphere,
    latlong_shell,
    displaced_shells,
    concentric_icospheres,
    look_at,
    fibonacci_cameras,
    rgba_texture,
    sh_texture,
    sh_channels,
    config_scene,
    CONFIGS,
)
