"""FP64 CPU oracle of the k-shell renderer -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path:
it is a separate C++ library (``vs_oracle.cpp``) reached through ``ctypes``,
fed by the seeded generators of the ``synth`` package.

Every function states the paper passage it follows; the discrete readings of
the silent parts (snapping, fill rule, depth key, addressing) are listed at
the top of ``vs_oracle.cpp``.
"""

from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

from .build import LIB_PATH, build_oracle

FMT_RGBA_F32 = 0
FMT_SH_F16 = 1
FMT_SH_U8 = 2

_lib = None


class OCam(ctypes.Structure):
    _fields_ = [("w2c", ctypes.c_float * 12), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("znear", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class OShell(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_void_p), ("uv", ctypes.c_void_p), ("tris", ctypes.c_void_p),
                ("nv", ctypes.c_int32), ("nt", ctypes.c_int32), ("tex", ctypes.c_void_p),
                ("tw", ctypes.c_int32), ("th", ctypes.c_int32), ("fmt", ctypes.c_int32),
                ("degree", ctypes.c_int32), ("pitch", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("band_shift", ctypes.c_int32), ("vmin", ctypes.c_double), ("vmax", ctypes.c_double)]


_DTYPES = {np.dtype(np.float32): 0, np.dtype(np.float16): 1, np.dtype(np.float64): 2}


def lib():
    global _lib
    if _lib is None:
        path = os.environ.get("VS_ORACLE_LIB", LIB_PATH)   # e.g. a mutated copy
        if path == LIB_PATH and not os.path.exists(LIB_PATH):
            build_oracle()
        _lib = ctypes.CDLL(path)
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def ocam(cam) -> OCam:
    c = OCam()
    w2c = np.ascontiguousarray(cam.world_to_cam, dtype=np.float32).reshape(-1)
    for i in range(12):
        c.w2c[i] = float(w2c[i])
    c.fx, c.fy, c.cx, c.cy, c.znear = cam.fx, cam.fy, cam.cx, cam.cy, cam.znear
    c.width, c.height = cam.width, cam.height
    return c


class _ShellRefs:
    """Keeps contiguous copies alive while the C side holds pointers."""

    def __init__(self, shells, shape_only: bool = False):
        # shape_only: the texel values are not passed (NULL): for the calls
        # that never read them (raster statistics, footprint counts), so a
        # shape-only texture (e.g. a broadcast array) is not materialised
        self.keep = []
        self.arr = (OShell * len(shells))()
        for i, s in enumerate(shells):
            pos = np.ascontiguousarray(s.pos, np.float32)
            uv = np.ascontiguousarray(s.uv, np.float32)
            tris = np.ascontiguousarray(s.tris, np.int32)
            tex = s.tex if shape_only else np.ascontiguousarray(s.tex)
            self.keep += [pos, uv, tris, tex]
            o = self.arr[i]
            o.pos, o.uv, o.tris = _ptr(pos).value, _ptr(uv).value, _ptr(tris).value
            o.nv, o.nt = pos.shape[0], tris.shape[0]
            o.tex = None if shape_only else _ptr(tex).value
            o.fmt, o.degree = s.fmt, s.degree
            if s.fmt == FMT_SH_U8:
                assert tex.dtype == np.uint8 and tex.ndim == 1
                o.tw, o.th, o.pitch, o.dtype = s.tex_w, s.tex_h, 0, -1
                o.band_shift, o.vmin, o.vmax = s.band_shift, s.vmin, s.vmax
            else:
                o.th, o.tw, o.pitch = tex.shape[0], tex.shape[1], tex.shape[2]
                o.dtype = _DTYPES[tex.dtype]


def sample_baked(shell, m: int, u: float, v: float) -> np.ndarray:
    """Decoded bilinear sample of SH coefficient m (RGBA) of a FMT_SH_U8
    shell at UV (u, v)."""
    tex = np.ascontiguousarray(shell.tex, np.uint8)
    out = np.zeros(4, np.float64)
    r = lib().oracle_sample_baked(_ptr(tex), ctypes.c_int32(shell.tex_w), ctypes.c_int32(shell.tex_h),
                                  ctypes.c_int32(shell.degree), ctypes.c_int32(shell.band_shift),
                                  ctypes.c_double(shell.vmin), ctypes.c_double(shell.vmax), ctypes.c_int32(m),
                                  ctypes.c_double(u), ctypes.c_double(v), _ptr(out))
    if r != 0:
        raise ValueError("coefficient out of range")
    return out


def footprint_texels_baked(scene, cam, hits: np.ndarray) -> np.ndarray:
    """Distinct texels per (shell, band) [k, 4] touched by the bilinear
    footprints of a view's fragments (baked shells; zeros otherwise)."""
    refs = _ShellRefs(scene.shells)
    hits = np.ascontiguousarray(hits, np.int32)
    out = np.zeros((scene.k, 4), np.int64)
    c = ocam(cam)
    lib().oracle_footprint_texels_baked(refs.arr, ctypes.c_int32(scene.k), ctypes.byref(c), _ptr(hits), _ptr(out))
    return out


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


# --- vertex stage -------------------------------------------------------------

def setup_vertices(pos: np.ndarray, cam):
    """Pinned FP32 transform + 1/256 px snap + depth key, per vertex.

    Returns (xy int64 [V,2], invw float32 [V], q uint32 [V], flags int32 [V])
    with flags bit 0 = nearer than znear, bit 1 = outside the guard band.
    """
    pos = np.ascontiguousarray(pos, np.float32)
    n = pos.shape[0]
    xy = np.zeros((n, 2), np.int64)
    invw = np.zeros(n, np.float32)
    q = np.zeros(n, np.uint32)
    flags = np.zeros(n, np.int32)
    c = ocam(cam)
    lib().oracle_setup_vertices(_ptr(pos), ctypes.c_int32(n), ctypes.byref(c), _ptr(xy), _ptr(invw),
                                _ptr(q), _ptr(flags))
    return xy, invw, q, flags


# --- raster (per shell nearest hit) ---------------------------------------------

def raster(pos, tris, cam, brute: bool = False, threads: Optional[int] = None,
           coverage: bool = False):
    """Per-shell nearest-hit raster (Fig. 3c: first intersection per surface).

    Returns (keys uint64 [H,W], cover int32 [H,W] or None, stats int64 [5] =
    front, back/degenerate, behind the near plane, off the guard band,
    clipped at the near plane).
    keys = (depth key << 32) | (2^32 - 1 - triangle); 0 = miss.
    """
    pos = np.ascontiguousarray(pos, np.float32)
    tris = np.ascontiguousarray(tris, np.int32)
    H, W = cam.height, cam.width
    keys = np.zeros((H, W), np.uint64)
    cover = np.zeros((H, W), np.int32) if coverage else None
    stats = np.zeros(5, np.int64)
    c = ocam(cam)
    lib().oracle_raster(_ptr(pos), ctypes.c_int32(pos.shape[0]), _ptr(tris),
                        ctypes.c_int32(tris.shape[0]), ctypes.byref(c), ctypes.c_int32(int(brute)),
                        ctypes.c_int32(threads or default_threads()), _ptr(keys),
                        _ptr(cover) if cover is not None else None, _ptr(stats))
    return keys, cover, stats


def hits_from_keys(keys: np.ndarray) -> np.ndarray:
    low = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
    return np.where(keys == 0, -1, 0xFFFFFFFF - low).astype(np.int32)


def raster_scene(scene, cam, threads: Optional[int] = None, brute: bool = False):
    """hits int32 [k,H,W] (-1 = miss), keys uint64 [k,H,W], stats [k,5]."""
    hs, ks, st = [], [], []
    for s in scene.shells:
        keys, _, stats = raster(s.pos, s.tris, cam, brute=brute, threads=threads)
        ks.append(keys)
        hs.append(hits_from_keys(keys))
        st.append(stats)
    return np.stack(hs), np.stack(ks), np.stack(st)


# --- shading / compositing ----------------------------------------------------------

ALPHA_ATTEN = 2   # flag: transparency attenuation (Sec. 3 "Transparency Attenuation")


def shade(scene, cam, hits: np.ndarray, bg=(0.0, 0.0, 0.0), threads: Optional[int] = None, flags: int = 0):
    """Bilinear texel fetch, SH decode and front-to-back compositing (Eq. 6);
    flags & ALPHA_ATTEN scales each alpha by 2 sigmoid(10 |v . n|) - 1.

    Returns (rgba float64 [H,W,4] = (C + T bg, 1 - T), fragments per shell).
    """
    refs = _ShellRefs(scene.shells)
    H, W = cam.height, cam.width
    hits = np.ascontiguousarray(hits, np.int32)
    assert hits.shape == (scene.k, H, W)
    out = np.zeros((H, W, 4), np.float64)
    bgv = np.ascontiguousarray(bg, np.float64)
    frags = np.zeros(scene.k, np.int64)
    c = ocam(cam)
    lib().oracle_shade(refs.arr, ctypes.c_int32(scene.k), ctypes.byref(c), _ptr(bgv), _ptr(hits),
                       _ptr(out), ctypes.c_int32(threads or default_threads()), _ptr(frags),
                       ctypes.c_int32(flags), None)
    return out, frags


LAYER_FIELDS = ("nx", "ny", "nz", "u", "v", "alpha", "weight", "r", "g", "b", "pad0", "pad1")


def layers(scene, cam, hits: np.ndarray, bg=(0.0, 0.0, 0.0), threads: Optional[int] = None, flags: int = 0):
    """Per-shell render buffers of Figs. S1/S3 before blending: float64
    [k, H, W, 12] = unit face normal, uv, opacity, blending weight T_i alpha_i
    (the layer's contribution), rgb, 0, 0 -- zero where a shell has no
    fragment.  Also returns the composite (rgba) like shade()."""
    refs = _ShellRefs(scene.shells)
    H, W = cam.height, cam.width
    hits = np.ascontiguousarray(hits, np.int32)
    out = np.zeros((H, W, 4), np.float64)
    lay = np.zeros((scene.k, H, W, 12), np.float64)
    bgv = np.ascontiguousarray(bg, np.float64)
    frags = np.zeros(scene.k, np.int64)
    c = ocam(cam)
    lib().oracle_shade(refs.arr, ctypes.c_int32(scene.k), ctypes.byref(c), _ptr(bgv), _ptr(hits),
                       _ptr(out), ctypes.c_int32(threads or default_threads()), _ptr(frags),
                       ctypes.c_int32(flags), _ptr(lay))
    return lay, out


def render(scene, cam, bg=(0.0, 0.0, 0.0), threads: Optional[int] = None, flags: int = 0):
    """Full oracle render: (rgba [H,W,4] f64, hits [k,H,W] i32, frags [k])."""
    hits, _, _ = raster_scene(scene, cam, threads=threads)
    rgba, frags = shade(scene, cam, hits, bg=bg, threads=threads, flags=flags)
    return rgba, hits, frags


def backward(scene, cam, hits: np.ndarray, grad_rgb: np.ndarray, bg=(0.0, 0.0, 0.0),
             flags: int = 0, with_scale: bool = False, gmag: Optional[np.ndarray] = None,
             aw_err: float = 0.0, only: Optional[int] = None, weight_err: float = 0.0):
    """dL/d(texel values) given dL/d(output rgb) -- the texture-fitting
    gradient of Sec. 3 "Texturing Meshes".  Returns one FP64 array per shell,
    shaped like its texture.

    with_scale: also return the gradient's per-texel error scales as
    (grads, (S_w, S_1, S_y)): over the (fragment, tap) terms that reach a
    texel value, S_w sums |w| M and S_1 sums M, M being the term's product
    without the tap weight w, with every factor taken by absolute value and
    every difference as the sum of its terms' absolute values; S_y sums
    |w| M with the SH basis value left out (SH coefficient values only; see
    oracle_backward).  An FP32 evaluation errs by a small multiple of
    epsilon times S_w, plus its tap-weight error times S_1, plus its
    absolute SH-basis error times S_y.  gmag [H, W, 3]:
    the size of each pixel's output gradient before cancellation (default
    |grad_rgb|; l2_loss_scale for the L2 loss).  aw_err: with ALPHA_ATTEN,
    an absolute error of each alpha_w that the scales allow for.
    weight_err: a tap-weight error the scales allow for; S_1 then also
    reaches the texels beside a footprint whose texel coordinate lies
    within weight_err of a texel-centre line (where a lower-precision
    evaluation may shift the footprint by one texel).  only:
    compute shell `only`'s arrays alone (the others are None), which bounds
    the host memory of large textures.  The scales do not change the
    gradient."""
    refs = _ShellRefs(scene.shells)
    H, W = cam.height, cam.width
    hits = np.ascontiguousarray(hits, np.int32)
    g = np.ascontiguousarray(grad_rgb, np.float64)
    assert g.shape == (H, W, 3)
    want = [only is None or i == only for i in range(scene.k)]

    def arrays():
        return [np.zeros(s.tex.shape, np.float64) if w else None for s, w in zip(scene.shells, want)]

    def pointers(arrs):
        return (ctypes.c_void_p * scene.k)(*[a.ctypes.data if a is not None else None for a in arrs])

    grads = arrays()
    ptrs = pointers(grads)
    scales = arrays() if with_scale else None
    reach = arrays() if with_scale else None
    sptrs = pointers(scales) if with_scale else None
    rptrs = pointers(reach) if with_scale else None
    ysc = arrays() if with_scale else None
    yptrs = pointers(ysc) if with_scale else None
    gm = None
    if gmag is not None:
        gm = np.ascontiguousarray(gmag, np.float64)
        assert gm.shape == (H, W, 3)
    bgv = np.ascontiguousarray(bg, np.float64)
    c = ocam(cam)
    r = lib().oracle_backward(refs.arr, ctypes.c_int32(scene.k), ctypes.byref(c), _ptr(bgv), _ptr(hits),
                              _ptr(g), ptrs, ctypes.c_int32(flags),
                              _ptr(gm) if gm is not None else ctypes.c_void_p(0), sptrs, rptrs,
                              ctypes.c_double(aw_err), ctypes.c_double(weight_err), yptrs)
    if r != 0:
        raise ValueError("the baked byte format (FMT_SH_U8) has no gradient")
    return (grads, (scales, reach, ysc)) if with_scale else grads


def l2_loss_grad(rgba: np.ndarray, target_rgb: np.ndarray):
    """L = mean over pixels and RGB channels of (C - target)^2; returns (L, dL/dC)."""
    d = rgba[..., :3] - target_rgb
    n = d.size
    return float((d * d).sum() / n), 2.0 * d / n


def l2_loss_scale(rgba: np.ndarray, target_rgb: np.ndarray):
    """Size of each pixel's L2-loss gradient before cancellation,
    2 (|C| + |target|) / n: the gmag of backward's error scale when the
    gradient is formed from a computed colour and a target."""
    return 2.0 * (np.abs(rgba[..., :3]) + np.abs(target_rgb)) / (rgba[..., :3].size)


def l1_loss_grad(rgba: np.ndarray, target_rgb: np.ndarray):
    """The pixel-wise L1 colour loss the textures are fitted with (Sec. 3
    "Texturing Meshes"): L = mean over pixels and RGB channels of
    |C - target|; returns (L, dL/dC) with the subgradient 0 where C equals
    the target."""
    d = rgba[..., :3] - target_rgb
    n = d.size
    return float(np.abs(d).sum() / n), np.sign(d) / n


def footprint_texels(scene, cam, hits: np.ndarray) -> np.ndarray:
    """Distinct texels read by each shell's bilinear footprints."""
    refs = _ShellRefs(scene.shells, shape_only=True)
    hits = np.ascontiguousarray(hits, np.int32)
    out = np.zeros(scene.k, np.int64)
    c = ocam(cam)
    lib().oracle_footprint_texels(refs.arr, ctypes.c_int32(scene.k), ctypes.byref(c), _ptr(hits),
                                  _ptr(out))
    return out


# --- single steps, for the pins -------------------------------------------------------

def sh_basis(degree: int, v: Sequence[float]) -> np.ndarray:
    vv = np.ascontiguousarray(v, np.float64)
    out = np.zeros(16, np.float64)
    lib().oracle_sh_basis(ctypes.c_int32(degree), _ptr(vv), _ptr(out))
    return out[: (degree + 1) ** 2]


def sample(tex: np.ndarray, u: float, v: float, nch: Optional[int] = None) -> np.ndarray:
    """Bilinear sample of the raw texel values at UV (u, v) (Fig. 5)."""
    tex = np.ascontiguousarray(tex)
    th, tw, pitch = tex.shape
    nch = pitch if nch is None else nch
    out = np.zeros(nch, np.float64)
    lib().oracle_sample(_ptr(tex), ctypes.c_int32(_DTYPES[tex.dtype]), ctypes.c_int32(tw), ctypes.c_int32(th),
                        ctypes.c_int32(pitch), ctypes.c_int32(nch), ctypes.c_double(u),
                        ctypes.c_double(v), _ptr(out))
    return out


def interp_uv(X, Y, invw, uv, px: int, py: int) -> np.ndarray:
    Xa = np.ascontiguousarray(X, np.int64)
    Ya = np.ascontiguousarray(Y, np.int64)
    iw = np.ascontiguousarray(invw, np.float64)
    uva = np.ascontiguousarray(uv, np.float32).reshape(-1)
    out = np.zeros(2, np.float64)
    lib().oracle_interp_uv(_ptr(Xa), _ptr(Ya), _ptr(iw), _ptr(uva), ctypes.c_int64(px),
                           ctypes.c_int64(py), _ptr(out))
    return out


def ray_dir(cam, x: int, y: int) -> np.ndarray:
    out = np.zeros(3, np.float64)
    c = ocam(cam)
    lib().oracle_ray_dir(ctypes.byref(c), ctypes.c_int32(x), ctypes.c_int32(y), _ptr(out))
    return out
