"""GB300-native (sm_103a) k-shell renderer of Volumetric Surfaces
(arXiv 2409.02482): forward, texel-gradient backward and a persistent
multi-item batch, behind the C ABI in include/vs.h (libvs.so).

Importing the package does not load the library; the first call does, and
raises if it has not been built.
"""

from .render import (Context, ShellObject, VSRender, camera_struct, make_workspace,  # noqa: F401
                     read_stats, render, render_backward, render_batch, render_layers, workspace_size,
                     VS_FLAG_ALPHA_ATTEN, VS_FLAG_LOSS_L1, VS_FLAG_LOSS_L2, VS_TEX_RGBA_F32, VS_TEX_SH_F16,
                     VS_TEX_SH_U8, baked_layout)
from .render import BatchItems, NeuralTexture  # noqa: F401
from .render import autotune_batch, get_batch_tuning, set_batch_tuning, tune_search, tuning  # noqa: F401
