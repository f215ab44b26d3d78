"""vs_render_noalloc: the forward entry point for callers that cannot allocate
device memory -- a render loop that must not allocate once it is running, or
a host framework that owns and pools every byte of device memory and lends
none out -- and so cannot pass a workspace.  It keeps its scratch in a fixed
device array shared by every call.  These checks call it through the C ABI
and compare it with vs_render on two calls in a row: the second call must not
see the first call's leftovers.  Both entry points run the same kernels on the
same inputs, so colours must agree bit for bit, not just to a tolerance.  The
calls cover a hit buffer and none, and a close-up whose near plane cuts the
shells (the generic kernels with clipping).  A request larger than the fixed
array is refused before anything runs.

This file is collected last on purpose: it must pass on its own in a fresh
process and after every other test.
"""

import ctypes

import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _call_noalloc(lib, ctx, obj, cam, bg, out, hits):
    import paper_2409_02482_gb300 as vs
    c = vs.camera_struct(cam)
    bgv = (ctypes.c_float * 3)(*bg)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.vs_render_noalloc(ctx.handle, obj.handle, ctypes.byref(c), bgv,
                                 ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(hits.data_ptr()) if hits is not None else None,
                                 0, stream)


def test_noalloc_matches_vs_render_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2409_02482_gb300 as vs
    from paper_2409_02482_gb300 import _abi
    lib = _abi.load()
    ctx = vs.Context(0)
    (scene, cams), = synth.config_scene("c1")
    obj = vs.ShellObject.from_scene(ctx, scene)
    # views in a row with different sizes, so stale scratch from one call
    # would show up in the next; the last is a close-up with the near plane
    # through the shells (clipping kernels), rendered without a hit buffer
    views = [(cams[0], True),
             (synth.look_at((1.0, 2.5, 1.2), width=200, height=150), True),
             (synth.look_at((0.0, -1.45, 0.25), width=96, height=80, fov_y_deg=60.0, znear=0.6), True),
             (synth.look_at((0.9, -0.9, 0.6), width=77, height=64, fov_y_deg=70.0, znear=0.55), False),
             (cams[0], False)]
    bg = (0.3, 0.2, 0.1)
    clipped = 0
    for cam, with_hits in views:
        ws = vs.make_workspace(ctx, [obj], [cam])
        ref_out, ref_hits = vs.render(ctx, obj, cam, ws, bg=bg)
        clipped += vs.read_stats(ws)["tris_clipped"]
        out = torch.full((cam.height, cam.width, 4), float("nan"), device="cuda")
        hits = (torch.full((obj.k, cam.height, cam.width), -7, dtype=torch.int32, device="cuda")
                if with_hits else None)
        assert _call_noalloc(lib, ctx, obj, cam, bg, out, hits) == _abi.VS_OK, lib.vs_last_error()
        torch.cuda.synchronize()
        if with_hits:
            assert torch.equal(hits, ref_hits)
        # same kernels, same inputs, same arithmetic: identical bits
        assert torch.equal(out, ref_out), (out - ref_out).abs().max().item()
        assert (ref_hits >= 0).any()
    assert clipped > 0, "the close-ups must exercise near-plane clipping"


def test_noalloc_refuses_requests_beyond_its_fixed_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2409_02482_gb300 as vs
    from paper_2409_02482_gb300 import _abi
    lib = _abi.load()
    ctx = vs.Context(0)
    (scene, _), = synth.config_scene("c1")
    obj = vs.ShellObject.from_scene(ctx, scene)
    big = synth.look_at((0.0, -3.0, 0.5), width=4096, height=4096)    # 3 x 4096^2 x 8 B > 16 MiB
    out = torch.empty((4, 4), device="cuda")
    st = _call_noalloc(lib, ctx, obj, big, (0.0, 0.0, 0.0), out, None)
    assert st == _abi.VS_ERR_OVERFLOW
    assert b"bytes of scratch" in lib.vs_last_error()
