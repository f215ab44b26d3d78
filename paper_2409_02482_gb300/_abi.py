"""ctypes mirror of include/vs.h.

Argument marshalling only: every step of rendering and differentiation runs
in the CUDA kernels of libvs.so.  There is no fallback: if the library is
missing, loading raises.
"""

from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvs.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "vs.h")

VS_OK = 0
VS_ERR_INVALID_ARG = -1
VS_ERR_CUDA = -2
VS_ERR_UNSUPPORTED = -3
VS_ERR_WORKSPACE = -4
VS_ERR_OVERFLOW = -5
VS_ERR_TIMEOUT = -6
STATUS_NAMES = {0: "VS_OK", -1: "VS_ERR_INVALID_ARG", -2: "VS_ERR_CUDA", -3: "VS_ERR_UNSUPPORTED",
                -4: "VS_ERR_WORKSPACE", -5: "VS_ERR_OVERFLOW", -6: "VS_ERR_TIMEOUT"}

VS_TEX_RGBA_F32 = 0
VS_TEX_SH_F16 = 1
VS_TEX_SH_U8 = 2
VS_FLAG_LOSS_L2 = 1 << 0
VS_FLAG_LOSS_L1 = 1 << 2
VS_FLAG_ALPHA_ATTEN = 1 << 1
VS_FLAG_TEST_STALL = 1 << 30
VS_MAX_SHELLS = 16
VS_LAYER_FLOATS = 12


class vs_shell_desc(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_void_p), ("num_verts", ctypes.c_int32),
                ("uv", ctypes.c_void_p), ("tris", ctypes.c_void_p), ("num_tris", ctypes.c_int32),
                ("texels", ctypes.c_void_p), ("tex_w", ctypes.c_int32), ("tex_h", ctypes.c_int32),
                ("format", ctypes.c_int32), ("sh_degree", ctypes.c_int32),
                ("texel_pitch", ctypes.c_int32), ("band_shift", ctypes.c_int32),
                ("value_min", ctypes.c_float), ("value_max", ctypes.c_float),
                ("grad_pitch", ctypes.c_int32)]


class vs_camera(ctypes.Structure):
    _fields_ = [("world_to_cam", ctypes.c_float * 12), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("znear", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class vs_batch_item(ctypes.Structure):
    _fields_ = [("obj", ctypes.c_void_p), ("cam", vs_camera), ("out_rgba", ctypes.c_void_p),
                ("hits", ctypes.c_void_p), ("grad_rgb", ctypes.c_void_p),
                ("grad_texels", ctypes.POINTER(ctypes.c_void_p)), ("loss", ctypes.c_void_p)]


class vs_tuning(ctypes.Structure):
    _fields_ = [("raster_tris", ctypes.c_int32), ("shade_pixels", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


VS_TUNING_DEFAULT_RASTER_TRIS = 256
VS_TUNING_DEFAULT_SHADE_PIXELS = 256
vs_cost_fn = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.POINTER(vs_tuning), ctypes.c_void_p)


class vs_ntex_config(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("features", ctypes.c_int32), ("log2_table", ctypes.c_int32),
                ("base_res", ctypes.c_int32), ("growth", ctypes.c_float), ("hidden", ctypes.c_int32),
                ("out_ch", ctypes.c_int32), ("tensor_cores", ctypes.c_int32)]


class vs_stats(ctypes.Structure):
    _fields_ = [("device_status", ctypes.c_int32), ("fragments", ctypes.c_uint64),
                ("tris_front", ctypes.c_uint64), ("tris_culled_back", ctypes.c_uint64),
                ("tris_culled_near", ctypes.c_uint64), ("tris_culled_guard", ctypes.c_uint64),
                ("tris_large", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("tris_clipped", ctypes.c_uint64), ("kernel_class", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


# vs_stats.kernel_class: 1 + texel class (+ 16 for the clipping / layers variant)
KCLASS_ANY, KCLASS_RGBA, KCLASS_SH0, KCLASS_U80, KCLASS_FULL = 1, 2, 3, 7, 16

_P = ctypes.c_void_p
_I = ctypes.c_int32
_U = ctypes.c_uint32
_SZ = ctypes.c_size_t

SIGNATURES = {
    "vs_create": ([ctypes.POINTER(_P), ctypes.c_int], _I),
    "vs_destroy": ([_P], _I),
    "vs_last_error": ([], ctypes.c_char_p),
    "vs_load_shells": ([_P, ctypes.POINTER(vs_shell_desc), _I, ctypes.POINTER(_P)], _I),
    "vs_free_shells": ([_P, _P], _I),
    "vs_workspace_size": ([_P, ctypes.POINTER(_P), ctypes.POINTER(vs_camera), _I, _U,
                           ctypes.POINTER(_SZ)], _I),
    "vs_render": ([_P, _P, ctypes.POINTER(vs_camera), _P, _P, _P, _P, _SZ, _U, _P], _I),
    "vs_render_layers": ([_P, _P, ctypes.POINTER(vs_camera), _P, _P, _P, _P, _P, _SZ, _U, _P], _I),
    "vs_render_backward": ([_P, _P, ctypes.POINTER(vs_camera), _P, _P, _P,
                            ctypes.POINTER(_P), _P, _P, _SZ, _U, _P], _I),
    "vs_render_batch": ([_P, ctypes.POINTER(vs_batch_item), _I, _P, _I, _P, _SZ, _U, _P], _I),
    "vs_read_stats": ([_P, _P, _I, ctypes.POINTER(vs_stats)], _I),
    "vs_render_noalloc": ([_P, _P, ctypes.POINTER(vs_camera), _P, _P, _P, _U, _P], _I),
    "vs_baked_layout": ([_I, _I, _I, _I, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_I), ctypes.POINTER(_I),
                         ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_int64)], _I),
    "vs_ntex_layout": ([ctypes.POINTER(vs_ntex_config), ctypes.POINTER(ctypes.c_int64),
                        ctypes.POINTER(ctypes.c_int64)], _I),
    "vs_ntex_workspace_size": ([ctypes.POINTER(vs_ntex_config), _I, _I, ctypes.POINTER(_SZ)], _I),
    "vs_ntex_forward": ([_P, ctypes.POINTER(vs_ntex_config), _P, _I, _I, _P, _I, _I, _I, _P, _SZ, _P], _I),
    "vs_ntex_backward": ([_P, ctypes.POINTER(vs_ntex_config), _P, _I, _I, _P, _I, _I, _P, _P, _SZ, _P], _I),
    "vs_adam_step": ([_P, _P, _P, _P, _P, ctypes.c_int64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                      ctypes.c_float, _I, _P], _I),
    "vs_set_batch_tuning": ([_P, _I, _I, ctypes.POINTER(vs_tuning)], _I),
    "vs_get_batch_tuning": ([_P, _I, _I, ctypes.POINTER(vs_tuning)], _I),
    "vs_tune_search": ([ctypes.POINTER(vs_tuning), _I, vs_cost_fn, _P, ctypes.POINTER(vs_tuning),
                        ctypes.POINTER(_I)], _I),
    "vs_autotune_batch": ([_P, ctypes.POINTER(vs_batch_item), _I, _P, _I, _P, _SZ, _U, _P, _I,
                           ctypes.POINTER(vs_tuning)], _I),
}

_lib = None


def header_functions():
    """Names of the functions include/vs.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vs_[a-z_]+)\s*\(", text)))


def load(path: str = LIB_PATH):
    """Load libvs.so (built by __graft_entry__.build()); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libvs.so not found at {path}: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


class VSError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def check(status: int):
    if status != VS_OK:
        raise VSError(status, load().vs_last_error().decode(errors="replace"))
    return status
