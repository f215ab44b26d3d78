"""Python binding of the k-shell renderer: the C-ABI names, torch tensors in.

PyTorch only supplies device memory and streams here; all rendering and
differentiation runs in libvs.so's CUDA kernels (see include/vs.h).
"""

from __future__ import annotations

import ctypes
from typing import List, Optional, Sequence

import torch

from . import _abi
from ._abi import (VS_FLAG_ALPHA_ATTEN, VS_FLAG_LOSS_L1, VS_FLAG_LOSS_L2, VS_TEX_RGBA_F32, VS_TEX_SH_F16, VS_TEX_SH_U8, check,
                   vs_batch_item, vs_ntex_config,
                   vs_camera, vs_cost_fn, vs_shell_desc, vs_stats, vs_tuning)

__all__ = ["Context", "ShellObject", "camera_struct", "workspace_size", "make_workspace",
           "render", "render_layers", "render_backward", "render_batch", "read_stats", "VSRender",
           "NeuralTexture",
           "tuning", "set_batch_tuning", "get_batch_tuning", "tune_search", "autotune_batch",
           "VS_FLAG_ALPHA_ATTEN", "VS_FLAG_LOSS_L1", "VS_FLAG_LOSS_L2", "VS_TEX_RGBA_F32", "VS_TEX_SH_F16", "VS_TEX_SH_U8",
           "baked_layout"]


def _ptr(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def camera_struct(cam) -> vs_camera:
    """vs_camera from any object with world_to_cam (3x4), fx, fy, cx, cy,
    znear, width, height (e.g. synth.Camera)."""
    c = vs_camera()
    m = torch.as_tensor(cam.world_to_cam, dtype=torch.float32).reshape(-1).tolist()
    for i in range(12):
        c.world_to_cam[i] = m[i]
    c.fx, c.fy, c.cx, c.cy, c.znear = (float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy),
                                       float(cam.znear))
    c.width, c.height = int(cam.width), int(cam.height)
    return c


class Context:
    """vs_create / vs_destroy."""

    def __init__(self, device: int = 0):
        self.lib = _abi.load()
        self.device = device
        self.handle = ctypes.c_void_p()
        check(self.lib.vs_create(ctypes.byref(self.handle), device))

    def close(self):
        if self.handle:
            self.lib.vs_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ShellObject:
    """vs_load_shells over device tensors (kept alive by this object).

    Each shell: dict(pos=[V,3] f32, uv=[V,2] f32, tris=[T,3] i32,
    tex=[H,W,pitch] f32 (RGBA) or f16 (SH), fmt, degree, and optionally
    grad_pitch: FP32 values per texel of its gradient arrays, default the
    texel pitch); baked shells
    (VS_TEX_SH_U8): tex = the u8 band buffer (vs_baked_layout) and tex_w,
    tex_h, band_shift, vmin, vmax."""

    def __init__(self, ctx: Context, shells: Sequence[dict]):
        self.ctx = ctx
        self.shells = [dict(s) for s in shells]
        k = len(self.shells)
        arr = (vs_shell_desc * k)()
        for i, s in enumerate(self.shells):
            for key in ("pos", "uv", "tris", "tex"):
                t = s[key]
                if not (t.is_cuda and t.is_contiguous()):
                    raise ValueError(f"shell {i}: {key} must be a contiguous CUDA tensor")
            d = arr[i]
            d.pos, d.num_verts = s["pos"].data_ptr(), s["pos"].shape[0]
            d.uv = s["uv"].data_ptr()
            d.tris, d.num_tris = s["tris"].data_ptr(), s["tris"].shape[0]
            d.texels = s["tex"].data_ptr()
            d.format = int(s["fmt"])
            d.sh_degree = int(s.get("degree", 0))
            if d.format == VS_TEX_SH_U8:
                d.tex_w, d.tex_h, d.texel_pitch = int(s["tex_w"]), int(s["tex_h"]), 0
                d.band_shift = int(s.get("band_shift", 0))
                d.value_min, d.value_max = float(s.get("vmin", -15.0)), float(s.get("vmax", 15.0))
            else:
                d.tex_h, d.tex_w, d.texel_pitch = s["tex"].shape
                d.grad_pitch = int(s.get("grad_pitch", 0))
        self.handle = ctypes.c_void_p()
        check(ctx.lib.vs_load_shells(ctx.handle, arr, k, ctypes.byref(self.handle)))

    @property
    def k(self) -> int:
        return len(self.shells)

    @property
    def textures(self) -> List[torch.Tensor]:
        return [s["tex"] for s in self.shells]

    def grad_shapes(self) -> List[tuple]:
        """Shape of each shell's FP32 gradient array: [H, W, grad_pitch]."""
        out = []
        for s in self.shells:
            h, w, p = s["tex"].shape
            out.append((h, w, int(s.get("grad_pitch", 0)) or p))
        return out

    def zero_grads(self) -> List[torch.Tensor]:
        """Zeroed FP32 gradient arrays, one per shell."""
        return [torch.zeros(sh, dtype=torch.float32, device=s["tex"].device)
                for sh, s in zip(self.grad_shapes(), self.shells)]

    @classmethod
    def from_scene(cls, ctx: Context, scene, device="cuda", grad_pitch: Optional[int] = None) -> "ShellObject":
        """Upload a synth.Scene (numpy arrays) to the device.  grad_pitch: the
        gradient arrays' values per texel for the FP16/FP32 shells (None =
        the texel pitch; "tight" = the format's value count)."""
        shells = []
        for s in scene.shells:
            d = dict(pos=torch.from_numpy(s.pos).to(device).contiguous(),
                     uv=torch.from_numpy(s.uv).to(device).contiguous(),
                     tris=torch.from_numpy(s.tris).to(device).contiguous(),
                     tex=torch.from_numpy(s.tex).to(device).contiguous(),
                     fmt=s.fmt, degree=s.degree)
            if s.fmt == VS_TEX_SH_U8:
                d.update(tex_w=s.tex_w, tex_h=s.tex_h, band_shift=s.band_shift, vmin=s.vmin, vmax=s.vmax)
            elif grad_pitch is not None:
                d["grad_pitch"] = s.channels if grad_pitch == "tight" else int(grad_pitch)
            shells.append(d)
        return cls(ctx, shells)

    def free(self):
        if self.handle:
            self.ctx.lib.vs_free_shells(self.ctx.handle, self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def workspace_size(ctx: Context, objs: Sequence[ShellObject], cams: Sequence, flags: int = 0) -> int:
    n = len(objs)
    oarr = (ctypes.c_void_p * n)(*[o.handle.value for o in objs])
    carr = (vs_camera * n)(*[camera_struct(c) for c in cams])
    out = ctypes.c_size_t()
    check(ctx.lib.vs_workspace_size(ctx.handle, oarr, carr, n, flags, ctypes.byref(out)))
    return out.value


def make_workspace(ctx: Context, objs, cams, flags: int = 0, device="cuda") -> torch.Tensor:
    """Zero-filled workspace tensor of the required size."""
    return torch.zeros(workspace_size(ctx, objs, cams, flags), dtype=torch.uint8, device=device)


def render(ctx: Context, obj: ShellObject, cam, ws: torch.Tensor, bg=(0.0, 0.0, 0.0),
           out: Optional[torch.Tensor] = None, hits: Optional[torch.Tensor] = None,
           want_hits: bool = True, flags: int = 0, stream=None):
    """vs_render: returns (rgba [H,W,4] f32, hits [k,H,W] i32 or None)."""
    H, W = int(cam.height), int(cam.width)
    dev = ws.device
    if out is None:
        out = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    if hits is None and want_hits:
        hits = torch.empty((obj.k, H, W), dtype=torch.int32, device=dev)
    c = camera_struct(cam)
    bgv = (ctypes.c_float * 3)(*bg)
    check(ctx.lib.vs_render(ctx.handle, obj.handle, ctypes.byref(c), bgv, _ptr(out), _ptr(hits),
                            _ptr(ws), ws.numel(), flags, _stream(stream)))
    return out, hits


def render_layers(ctx: Context, obj: ShellObject, cam, ws: torch.Tensor, bg=(0.0, 0.0, 0.0), flags: int = 0,
                  stream=None):
    """vs_render_layers: (rgba [H,W,4], hits [k,H,W], layers [k,H,W,12]) --
    per shell: unit face normal, u, v, opacity, blending weight, rgb, 0, 0."""
    H, W = int(cam.height), int(cam.width)
    dev = ws.device
    out = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    hits = torch.empty((obj.k, H, W), dtype=torch.int32, device=dev)
    layers = torch.empty((obj.k, H, W, _abi.VS_LAYER_FLOATS), dtype=torch.float32, device=dev)
    c = camera_struct(cam)
    bgv = (ctypes.c_float * 3)(*bg)
    check(ctx.lib.vs_render_layers(ctx.handle, obj.handle, ctypes.byref(c), bgv, _ptr(out), _ptr(hits),
                                   _ptr(layers), _ptr(ws), ws.numel(), flags, _stream(stream)))
    return out, hits, layers


def render_backward(ctx: Context, obj: ShellObject, cam, ws: torch.Tensor, hits: torch.Tensor,
                    grad_rgb: torch.Tensor, grads: Optional[List[torch.Tensor]] = None,
                    bg=(0.0, 0.0, 0.0), loss: Optional[torch.Tensor] = None, flags: int = 0,
                    stream=None) -> List[torch.Tensor]:
    """vs_render_backward: accumulates into (and returns) FP32 texel grads."""
    if grads is None:
        grads = obj.zero_grads()
    c = camera_struct(cam)
    bgv = (ctypes.c_float * 3)(*bg)
    gptrs = (ctypes.c_void_p * obj.k)(*[g.data_ptr() for g in grads])
    check(ctx.lib.vs_render_backward(ctx.handle, obj.handle, ctypes.byref(c), bgv, _ptr(hits),
                                     _ptr(grad_rgb.contiguous()), gptrs, _ptr(loss), _ptr(ws),
                                     ws.numel(), flags, _stream(stream)))
    return grads


class BatchItems:
    """Host-side vs_batch_item array (built once, reusable across calls)."""

    def __init__(self, items: Sequence[dict]):
        n = len(items)
        self.arr = (vs_batch_item * n)()
        self.keep = []
        for j, it in enumerate(items):
            b = self.arr[j]
            b.obj = it["obj"].handle.value
            b.cam = camera_struct(it["cam"])
            b.out_rgba = it["out"].data_ptr()
            b.hits = it["hits"].data_ptr() if it.get("hits") is not None else None
            b.grad_rgb = it["grad_rgb"].data_ptr() if it.get("grad_rgb") is not None else None
            if it.get("grads") is not None:
                g = (ctypes.c_void_p * len(it["grads"]))(*[t.data_ptr() for t in it["grads"]])
                self.keep.append(g)
                b.grad_texels = ctypes.cast(g, ctypes.POINTER(ctypes.c_void_p))
            b.loss = it["loss"].data_ptr() if it.get("loss") is not None else None
        self.n = n


def render_batch(ctx: Context, items, ws: torch.Tensor, bg=(0.0, 0.0, 0.0), do_backward: bool = False,
                 flags: int = 0, stream=None):
    """vs_render_batch over a BatchItems (or a list of item dicts: obj, cam,
    out, hits, grad_rgb, grads, loss)."""
    if not isinstance(items, BatchItems):
        items = BatchItems(items)
    bgv = (ctypes.c_float * 3)(*bg)
    check(ctx.lib.vs_render_batch(ctx.handle, items.arr, items.n, bgv, int(do_backward), _ptr(ws),
                                  ws.numel(), flags, _stream(stream)))
    return items


def baked_layout(tex_w: int, tex_h: int, degree: int, band_shift: int):
    """vs_baked_layout: ([(offset, w, h, stride) per band], total bytes)."""
    off = (ctypes.c_int64 * 4)()
    w, h, st = (ctypes.c_int32 * 4)(), (ctypes.c_int32 * 4)(), (ctypes.c_int32 * 4)()
    total = ctypes.c_int64()
    check(_abi.load().vs_baked_layout(tex_w, tex_h, degree, band_shift, off, w, h, st, ctypes.byref(total)))
    return [(off[i], w[i], h[i], st[i]) for i in range(degree + 1)], total.value


def tuning(raster_tris: int = 256, shade_pixels: int = 256, blocks_per_sm: int = 0) -> vs_tuning:
    """A vs_tuning (work-unit sizes and grid of vs_render_batch)."""
    return vs_tuning(raster_tris, shade_pixels, blocks_per_sm, 0)


def set_batch_tuning(ctx: Context, t: vs_tuning, do_backward: bool = False, k_max: int = 0):
    check(ctx.lib.vs_set_batch_tuning(ctx.handle, int(do_backward), k_max, ctypes.byref(t)))


def get_batch_tuning(ctx: Context, do_backward: bool = False, k_max: int = 1) -> vs_tuning:
    t = vs_tuning()
    check(ctx.lib.vs_get_batch_tuning(ctx.handle, int(do_backward), k_max, ctypes.byref(t)))
    return t


def tune_search(start: vs_tuning, max_blocks_per_sm: int, cost) -> tuple:
    """vs_tune_search with a Python cost(tuning) -> float; returns
    (best vs_tuning, number of cost calls)."""
    cb = vs_cost_fn(lambda t, _user: float(cost(t.contents)))
    best, n = vs_tuning(), ctypes.c_int32(0)
    check(_abi.load().vs_tune_search(ctypes.byref(start), max_blocks_per_sm, cb, None, ctypes.byref(best),
                                     ctypes.byref(n)))
    return best, n.value


def autotune_batch(ctx: Context, items, ws: torch.Tensor, bg=(0.0, 0.0, 0.0), do_backward: bool = False,
                   flags: int = 0, stream=None, repeats: int = 2) -> vs_tuning:
    """vs_autotune_batch: times launch shapes on this batch and keeps the
    fastest in the context.  Outputs are overwritten and gradients/losses
    accumulate over the tuning launches."""
    if not isinstance(items, BatchItems):
        items = BatchItems(items)
    bgv = (ctypes.c_float * 3)(*bg)
    best = vs_tuning()
    check(ctx.lib.vs_autotune_batch(ctx.handle, items.arr, items.n, bgv, int(do_backward), _ptr(ws), ws.numel(),
                                    flags, _stream(stream), repeats, ctypes.byref(best)))
    return best


class NeuralTexture:
    """vs_ntex_*: a hash-grid + MLP texture evaluated at texel centres, its
    adjoint and Adam, over device tensors kept here (params, grads, Adam
    moments, workspace).  `params` may be set from a numpy vector in the
    vs_ntex_layout order."""

    def __init__(self, ctx: Context, levels=16, features=2, log2_table=19, base_res=16, growth=1.5,
                 hidden=64, out_ch=28, tex_w=1024, tex_h=1024, device="cuda", tensor_cores=False):
        self.ctx = ctx
        self.cfg = vs_ntex_config(levels, features, log2_table, base_res, float(growth), hidden, out_ch,
                                  int(tensor_cores))
        self.tex_w, self.tex_h = int(tex_w), int(tex_h)
        off = (ctypes.c_int64 * 7)()
        total = ctypes.c_int64()
        check(ctx.lib.vs_ntex_layout(ctypes.byref(self.cfg), off, ctypes.byref(total)))
        self.offsets, self.count = list(off), total.value
        self.params = torch.zeros(self.count, dtype=torch.float32, device=device)
        self.grads = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        nb = ctypes.c_size_t()
        check(ctx.lib.vs_ntex_workspace_size(ctypes.byref(self.cfg), self.tex_w, self.tex_h, ctypes.byref(nb)))
        self.ws = torch.zeros(max(nb.value, 256), dtype=torch.uint8, device=device)

    def status(self) -> int:
        """The workspace's status word (synchronises): 0, or 1 when a
        bounded wait of the tensor-core layers ran out."""
        return int(self.ws[:4].view(torch.int32).item())

    def forward(self, texels: torch.Tensor, ch0: int = 0, stream=None):
        """Write channels [ch0, ch0 + C) of texels [H, W, pitch] (f32 or f16)."""
        dtype = {torch.float32: 0, torch.float16: 1}[texels.dtype]
        assert texels.is_contiguous() and texels.shape[:2] == (self.tex_h, self.tex_w)
        check(self.ctx.lib.vs_ntex_forward(self.ctx.handle, ctypes.byref(self.cfg), _ptr(self.params), self.tex_w,
                                           self.tex_h, _ptr(texels), dtype, texels.shape[2], ch0, _ptr(self.ws),
                                           self.ws.numel(), _stream(stream)))

    def backward(self, grad_texels: torch.Tensor, ch0: int = 0, stream=None):
        """Add dL/d(params) for dL/d(texels) (f32 [H, W, pitch]) into grads."""
        assert grad_texels.dtype == torch.float32 and grad_texels.is_contiguous()
        check(self.ctx.lib.vs_ntex_backward(self.ctx.handle, ctypes.byref(self.cfg), _ptr(self.params), self.tex_w,
                                            self.tex_h, _ptr(grad_texels), grad_texels.shape[2], ch0,
                                            _ptr(self.grads), _ptr(self.ws), self.ws.numel(), _stream(stream)))

    def adam(self, lr: float, beta1=0.9, beta2=0.99, eps=1e-15, stream=None):
        """One Adam step with the accumulated grads (then zero them yourself)."""
        self.step += 1
        check(self.ctx.lib.vs_adam_step(self.ctx.handle, _ptr(self.params), _ptr(self.grads), _ptr(self.m),
                                        _ptr(self.v), self.count, lr, beta1, beta2, eps, self.step, _stream(stream)))


def read_stats(ws: torch.Tensor, reset: bool = False, stream=None) -> dict:
    st = vs_stats()
    check(_abi.load().vs_read_stats(_ptr(ws), _stream(stream), int(reset), ctypes.byref(st)))
    return st.as_dict()


class VSRender(torch.autograd.Function):
    """Differentiable render w.r.t. the texel arrays.

    forward(ctx_, obj, cam, ws, bg, flags, *textures) -> rgba [H,W,4]; the
    hit buffer is saved and the backward recomputes transmittance from it
    (vs_render_backward, same flags).  Gradients come back in FP32 and
    autograd casts them to each texture's dtype.
    """

    @staticmethod
    def forward(fctx, vctx: Context, obj: ShellObject, cam, ws: torch.Tensor, bg, flags, *textures):
        out, hits = render(vctx, obj, cam, ws, bg=bg, flags=flags)
        fctx.vctx, fctx.obj, fctx.cam, fctx.ws, fctx.bg, fctx.flags = vctx, obj, cam, ws, bg, flags
        fctx.save_for_backward(hits)
        return out

    @staticmethod
    def backward(fctx, grad_out):
        (hits,) = fctx.saved_tensors
        g = grad_out[..., :3].contiguous().float()
        grads = render_backward(fctx.vctx, fctx.obj, fctx.cam, fctx.ws, hits, g, bg=fctx.bg,
                                flags=fctx.flags)
        out = []
        for gr, t in zip(grads, fctx.obj.textures):   # gradient pitch -> texel pitch
            p, gp = t.shape[2], gr.shape[2]
            out.append(gr if gp == p else (gr[..., :p] if gp > p else torch.nn.functional.pad(gr, (0, p - gp))))
        return (None, None, None, None, None, None, *out)
