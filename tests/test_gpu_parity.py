"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: hit IDs bit-exact; colours within 1e-5 max-abs for FP32 texels and
2e-3 for FP16 texel storage (against the oracle fed the same FP16 values --
the compute error -- and, separately reported, the FP32 values before
rounding -- the storage error); gradients checked texel value by texel
value against their own bar (assert_grad_bar); batched forward
bit-identical to the per-view launches.
"""

import math

import numpy as np
import pytest
import torch

import oracle
import synth
from synth import FMT_RGBA_F32, FMT_SH_F16, Scene, Shell

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5
TOL_F16 = 2e-3
# baked bytes: the oracle reads the same bytes, so only the FP32 arithmetic
# differs (sums of up to 16 decoded values of magnitude <= 15 per channel)
TOL_U8 = 2e-4


@pytest.fixture(scope="module")
def vs():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2409_02482_gb300 as vs
    return vs


@pytest.fixture(scope="module")
def ctx(vs):
    return vs.Context(0)


# Per-texel gradient bar.  For every texel value, the oracle's error scales
# (oracle.backward(with_scale=True)) are S_w = sum of |w| M and S_1 = sum of M
# over the (fragment, tap) terms that reach it, M the term's magnitude
# without cancellation.  The GPU's gradient must satisfy
#     |g_gpu - g_ref| <= tol * S_w + ETA_W * S_1 + SH_ERR * S_y
# with tol = 1e-5 (FP32 textures) or 2e-3 (FP16 storage): the first term is
# the bar on the sum of contributions; the second covers the tap weights,
# which the GPU forms from FP32 texel coordinates (reading A16: the integer
# part split off, the in-triangle offset within ~8 texels carrying ~4
# roundings) and the oracle in FP64 -- their difference is a few 1e-6 at
# most, so ETA_W = 2^-17.  Values nothing reaches are exactly zero on both
# sides.  Returns the worst err / (1e-5 S_w + ETA_W S_1) over all values.
ETA_W = 2.0 ** -17
# The SH basis of the GPU comes from an FP32 ray direction (components off by
# ~3e-7 after the camera rotation and the normalisation) and FP32 products;
# a basis value near zero is a difference of such terms (e.g. x^2 - y^2), so
# its error is absolute: up to ~3e-6 for l = 3 (2.89 xyz).  The bar adds
# SH_ERR times the oracle's S_y (the coefficient terms without the basis
# value).
SH_ERR = 2.0 ** -18


def assert_grad_bar_by_shell(scene, terms, got, tol, nch=None):
    """assert_grad_bar for large textures, one shell at a time (bounded host
    memory): terms = [(cam, hits, dL, gmag or None)], whose oracle adjoints
    are summed; got = the GPU's gradient tensors.  Returns the worst ratio."""
    worst = 0.0
    for i in range(scene.k):
        ref = sw = s1 = sy = None
        for cam, hits, dL, gmag in terms:
            rg, (rw, r1, ry) = oracle.backward(scene, cam, hits, dL, with_scale=True, gmag=gmag, only=i,
                                               weight_err=ETA_W)
            if ref is None:
                ref, sw, s1, sy = rg[i], rw[i], r1[i], ry[i]
            else:
                ref += rg[i]
                sw += rw[i]
                s1 += r1[i]
                sy += ry[i]
            del rg, rw, r1, ry
        worst = max(worst, assert_grad_bar([got[i]], [ref], ([sw], [s1], [sy]), tol, nch=nch))
        del ref, sw, s1, sy
    return worst


def grad_tol_of(scene):
    return TOL_F32 if all(s.fmt == FMT_RGBA_F32 for s in scene.shells) else TOL_F16


def assert_grad_bar(got, ref, scales, tol, nch=None):
    sw, s1, sy = scales
    worst = 0.0
    for gg, rg, w, r, ys in zip(got, ref, sw, s1, sy):
        g = gg.cpu().numpy() if isinstance(gg, torch.Tensor) else gg
        if nch is not None:
            assert not g[..., nch:].any(), "padding values received a gradient"
            g, rg, w, r, ys = g[..., :nch], rg[..., :nch], w[..., :nch], r[..., :nch], ys[..., :nch]
        err = np.abs(g.astype(np.float64) - rg)
        extra = ETA_W * r + SH_ERR * ys
        bar = tol * w + extra
        bad = err > bar
        if bad.any():
            idx = np.argwhere(bad)
            ratio = err[bad] / np.maximum(bar[bad], 1e-300)
            top = idx[np.argsort(-ratio)[:5]]
            detail = "; ".join(f"(y,x,c)={tuple(int(v) for v in t)} got {g[tuple(t)]:.6g} ref {rg[tuple(t)]:.6g} "
                               f"S_w {w[tuple(t)]:.3g} S_1 {r[tuple(t)]:.3g}" for t in top)
            raise AssertionError(f"{int(bad.sum())} texel values outside their bar; worst err/bar "
                                 f"{float(ratio.max()):.3g}: {detail}")
        assert not g[w == 0].any(), "a texel value nothing reaches received a gradient"
        live = w > 0
        if live.any():
            worst = max(worst, float((err[live] / (TOL_F32 * w[live] + extra[live])).max()))
    return worst


def tol_of(scene):
    if all(s.fmt == FMT_RGBA_F32 for s in scene.shells):
        return TOL_F32
    return TOL_U8 if all(s.fmt == synth.FMT_SH_U8 for s in scene.shells) else TOL_F16


def gpu_render(vs, ctx, scene, cam, bg=(0.0, 0.0, 0.0), obj=None, flags=0):
    obj = obj or vs.ShellObject.from_scene(ctx, scene)
    ws = vs.make_workspace(ctx, [obj], [cam])
    out, hits = vs.render(ctx, obj, cam, ws, bg=bg, flags=flags)
    st = vs.read_stats(ws)
    assert st["device_status"] == 0
    return out.cpu().numpy(), hits.cpu().numpy(), st, obj, ws


def check_forward(vs, ctx, scene, cam, bg=(0.0, 0.0, 0.0), tol=None, flags=0):
    out, hits, st, obj, ws = gpu_render(vs, ctx, scene, cam, bg, flags=flags)
    ref, ref_hits, frags = oracle.render(scene, cam, bg=bg, flags=flags)
    mism = (hits != ref_hits).sum()
    assert mism == 0, f"{mism} hit IDs differ"
    err = np.abs(out - ref).max()
    assert err <= (tol or tol_of(scene)), f"max colour error {err}"
    assert st["fragments"] == frags.sum()
    assert st["tris_culled_near"] == 0 and st["tris_culled_guard"] == 0
    return err, obj, ws, hits


# ----------------------------------------------------------------------------
# forward
# ----------------------------------------------------------------------------

def test_c1_full_size_rgba_f32(vs, ctx):
    (scene, cams), = synth.config_scene("c1")
    err, *_ = check_forward(vs, ctx, scene, cams[0], bg=(0.3, 0.2, 0.1), tol=TOL_F32)
    print(f"c1 max err {err:.3e}")


@pytest.mark.parametrize("w,h", [(77, 53), (256, 1), (1, 200), (131, 257)])
def test_ragged_images(vs, ctx, w, h):
    (scene, _), = synth.config_scene("c1", scale=0.25)
    cam = synth.look_at((2.0, -2.0, 1.0), width=w, height=h)
    check_forward(vs, ctx, scene, cam, tol=TOL_F32)


@pytest.mark.parametrize("name,scale", [("c2", 0.01), ("c3", 0.004), ("c5", 0.0005)])
def test_sh_configs_scaled(vs, ctx, name, scale):
    (scene, cams), = synth.config_scene(name, scale=scale, views=3)
    errs = []
    for cam in cams:
        err, *_ = check_forward(vs, ctx, scene, cam, bg=(0.2, 0.2, 0.2))
        errs.append(err)
    print(f"{name} compute error vs oracle on the same FP16 values: {max(errs):.3e}")
    assert max(errs) < 1e-4      # FP32 compute error is far below the FP16 bar


def test_fp16_storage_error_is_within_bar(vs, ctx):
    """The error against the FP32 values before FP16 rounding (storage
    error) stays within 2e-3."""
    (scene, cams), = synth.config_scene("c2", scale=0.01, views=2)
    rng = np.random.default_rng(0)
    master = []
    for s in scene.shells:
        m = (0.3 * rng.standard_normal(s.tex.shape)).astype(np.float32)
        master.append(m)
        s.tex = m.astype(np.float16)
    for cam in cams:
        out, hits, st, obj, ws = gpu_render(vs, ctx, scene, cam)
        ref32 = Scene([Shell(s.pos, s.uv, s.tris, m, s.fmt, s.degree) for s, m in zip(scene.shells, master)])
        ref, _ = oracle.shade(ref32, cam, hits)
        err = np.abs(out - ref).max()
        print(f"storage error {err:.3e}")
        assert err <= TOL_F16


@pytest.mark.parametrize("k", [1, 2, 9, 16])
def test_many_and_few_shells(vs, ctx, k):
    shells = []
    rng = np.random.default_rng(k)
    geo = synth.displaced_shells(k, 10, seed=3, spacing=0.03)
    for i, (p, u, t) in enumerate(geo):
        if i % 2:
            shells.append(Shell(p, u, t, synth.sh_texture(32, 32, i % 4, rng), FMT_SH_F16, i % 4))
        else:
            shells.append(Shell(p, u, t, synth.rgba_texture(16, 16, rng), FMT_RGBA_F32))
    cam = synth.look_at((2.5, -1.5, 1.0), width=96, height=72)
    check_forward(vs, ctx, Scene(shells), cam, bg=(0.5, 0.5, 0.5))


def test_texel_pitch_padding_and_vector_widths(vs, ctx):
    """Padded texel pitches select wider loads; results do not change."""
    scene, cams = synth.config_scene("c4", scale=0.002, views=1)[0]
    cam = cams[0]
    base, *_ = gpu_render(vs, ctx, scene, cam)
    for pitch in (14, 16, 20):
        padded = Scene([Shell(s.pos, s.uv, s.tris,
                              np.concatenate([s.tex, np.zeros(s.tex.shape[:2] + (pitch - s.tex.shape[2],),
                                                              np.float16)], axis=2),
                              s.fmt, s.degree) for s in scene.shells])
        out, *_ = gpu_render(vs, ctx, padded, cam)
        assert np.array_equal(out, base)


def test_nothing_visible(vs, ctx):
    (scene, _), = synth.config_scene("c1", scale=0.25)
    cam = synth.look_at((0.0, -3.0, 0.0), target=(0.0, -6.0, 0.0), width=64, height=48)
    out, hits, st, *_ = gpu_render(vs, ctx, scene, cam, bg=(0.25, 0.5, 1.0))
    assert np.all(hits == -1)
    assert np.all(out == np.array([0.25, 0.5, 1.0, 0.0], np.float32))
    assert st["fragments"] == 0


def test_degenerate_and_back_facing_triangles(vs, ctx):
    pos, uv, tris = synth.icosphere(2, 1.0)
    extra = np.array([[0, 0, 0], [1, 1, 2], [5, 5, 5]], np.int32)          # zero-area
    flipped = tris[:40][:, [0, 2, 1]]                                        # back-facing copies
    t2 = np.concatenate([tris, extra, flipped]).astype(np.int32)
    rng = np.random.default_rng(0)
    scene = Scene([Shell(pos, uv, t2, synth.rgba_texture(32, 32, rng), FMT_RGBA_F32)])
    cam = synth.look_at((0.5, -2.5, 0.8), width=80, height=80)
    err, obj, ws, hits = check_forward(vs, ctx, scene, cam, tol=TOL_F32)


def test_large_triangles_take_the_cooperative_path(vs, ctx):
    """A few triangles that cover most of the image (screen boxes far above
    the per-thread limit) next to tiny ones."""
    pos, uv, tris = synth.icosphere(0, 1.0)     # 20 faces, each hundreds of pixels
    rng = np.random.default_rng(1)
    geo2 = synth.icosphere(3, 0.7)
    scene = Scene([Shell(pos, uv, tris, synth.rgba_texture(64, 64, rng), FMT_RGBA_F32),
                   Shell(*geo2, synth.rgba_texture(64, 64, rng), FMT_RGBA_F32)])
    cam = synth.look_at((0.3, -2.2, 0.5), width=640, height=480)
    err, obj, ws, hits = check_forward(vs, ctx, scene, cam, tol=TOL_F32)
    st = vs.read_stats(ws)
    assert st["device_status"] == 0


def test_bad_triangle_indices_are_reported_not_faulted(vs, ctx):
    pos, uv, tris = synth.icosphere(1, 1.0)
    bad = tris.copy()
    bad[3, 1] = 10_000_000
    rng = np.random.default_rng(0)
    scene = Scene([Shell(pos, uv, bad, synth.rgba_texture(8, 8, rng), FMT_RGBA_F32)])
    cam = synth.look_at((0.0, -3.0, 0.0), width=32, height=32)
    obj = vs.ShellObject.from_scene(ctx, scene)
    ws = vs.make_workspace(ctx, [obj], [cam])
    vs.render(ctx, obj, cam, ws)
    st = vs.read_stats(ws, reset=True)
    assert st["device_status"] == -1       # VS_ERR_INVALID_ARG
    # the context is still usable afterwards
    (scene2, cams2), = synth.config_scene("c1", scale=0.1)
    check_forward(vs, ctx, scene2, cams2[0], tol=TOL_F32)


def test_host_side_errors(vs, ctx):
    from paper_2409_02482_gb300._abi import VSError
    (scene, cams), = synth.config_scene("c1", scale=0.1)
    obj = vs.ShellObject.from_scene(ctx, scene)
    ws = vs.make_workspace(ctx, [obj], cams[:1])
    with pytest.raises(VSError, match="WORKSPACE"):   # below the visibility words alone
        vs.render(ctx, obj, cams[0], ws[: 8 * obj.k * int(cams[0].width) * int(cams[0].height) // 2])
    with pytest.raises(VSError, match="WORKSPACE"):
        vs.render(ctx, obj, cams[0], ws[1:])


# ----------------------------------------------------------------------------
# backward
# ----------------------------------------------------------------------------

# FP32 alpha_w = 2 sigmoid(10 |v.n|) - 1 (GPU: __expf, rsqrtf) against the
# oracle's FP64: a few ulps of the sigmoid near 1/2..1, doubled, plus the
# normal's and the dot product's rounding -- well under 2^-20 absolute.
AW_ERR = 2.0 ** -20


def check_backward(vs, ctx, scene, cam, bg, tol=None, flags=0):
    """Standalone adjoint of one view against the oracle's, every texel value
    within its own bar (assert_grad_bar; tol defaults to the format's)."""
    obj = vs.ShellObject.from_scene(ctx, scene)
    ws = vs.make_workspace(ctx, [obj], [cam])
    out, hits = vs.render(ctx, obj, cam, ws, bg=bg, flags=flags)
    g = torch.randn((cam.height, cam.width, 3), device="cuda",
                    generator=torch.Generator("cuda").manual_seed(1))
    grads = vs.render_backward(ctx, obj, cam, ws, hits, g, bg=bg, flags=flags)
    ref, sc = oracle.backward(scene, cam, hits.cpu().numpy(), g.cpu().numpy().astype(np.float64), bg=bg,
                              flags=flags, with_scale=True, aw_err=AW_ERR, weight_err=ETA_W)
    worst = assert_grad_bar(grads, ref, sc, tol or grad_tol_of(scene))
    assert vs.read_stats(ws)["device_status"] == 0
    return worst, obj, ws, hits, grads


def test_backward_rgba_matches_oracle(vs, ctx):
    (scene, cams), = synth.config_scene("c1", scale=0.25)
    w, *_ = check_backward(vs, ctx, scene, cams[0], (0.2, 0.3, 0.4))
    print(f"rgba grad worst err / per-texel 1e-5 bar {w:.2e}")


@pytest.mark.parametrize("name,scale", [("c2", 0.005), ("c4", 0.001), ("c5", 0.0004)])
def test_backward_sh_matches_oracle(vs, ctx, name, scale):
    sc, cams = synth.config_scene(name, scale=scale, views=1)[0]
    w, *_ = check_backward(vs, ctx, sc, cams[0], (0.1, 0.1, 0.1))
    print(f"{name} sh grad worst err / per-texel 1e-5 bar {w:.2e}")


def test_backward_l2_loss_flag(vs, ctx):
    (scene, cams), = synth.config_scene("c3", scale=0.002, views=1)
    cam = cams[0]
    (target_scene, _), = synth.config_scene("c3", scale=0.002, views=1, tex_seed=1)
    target, _, _ = oracle.render(target_scene, cam)
    obj = vs.ShellObject.from_scene(ctx, scene)
    ws = vs.make_workspace(ctx, [obj], [cam])
    out, hits = vs.render(ctx, obj, cam, ws)
    tgt = torch.from_numpy(target[..., :3].astype(np.float32)).cuda()
    loss = torch.zeros(1, device="cuda")
    grads = vs.render_backward(ctx, obj, cam, ws, hits, tgt, loss=loss, flags=vs.VS_FLAG_LOSS_L2)
    ref_rgba, ref_hits, _ = oracle.render(scene, cam)
    t64 = target[..., :3].astype(np.float32).astype(np.float64)
    L, dL = oracle.l2_loss_grad(ref_rgba, t64)
    ref, sc = oracle.backward(scene, cam, ref_hits, dL, with_scale=True,
                              gmag=oracle.l2_loss_scale(ref_rgba, t64), weight_err=ETA_W)
    assert abs(loss.item() - L) <= 1e-5 * L + 1e-9
    w = assert_grad_bar(grads, ref, sc, grad_tol_of(scene))
    print(f"l2 loss grad worst err / per-texel 1e-5 bar {w:.2e}")


def test_backward_l1_loss_flag(vs, ctx):
    """The L1 colour loss of Sec. 3 "Texturing Meshes": loss value and
    gradients against the oracle."""
    BG_EXACT = (0.25, 0.5, 0.75)   # exact in FP32: background residuals are 0 on both sides
    (scene, cams), = synth.config_scene("c3", scale=0.002, views=1)
    cam = cams[0]
    (target_scene, _), = synth.config_scene("c3", scale=0.002, views=1, tex_seed=5)
    target, _, _ = oracle.render(target_scene, cam, bg=BG_EXACT)
    tgt64 = target[..., :3].astype(np.float32).astype(np.float64)
    ref_rgba, ref_hits, _ = oracle.render(scene, cam, bg=BG_EXACT)
    # no residual so close to zero that FP32 and FP64 could disagree on its
    # sign (the colours agree to ~2e-7; target seed 5 keeps them >= 3e-5)
    d = np.abs(ref_rgba[..., :3] - tgt64)
    assert not np.any((d > 0) & (d < 1e-5))
    obj = vs.ShellObject.from_scene(ctx, scene)
    ws = vs.make_workspace(ctx, [obj], [cam])
    out, hits = vs.render(ctx, obj, cam, ws, bg=BG_EXACT)
    tgt = torch.from_numpy(target[..., :3].astype(np.float32)).cuda()
    loss = torch.zeros(1, device="cuda")
    grads = vs.render_backward(ctx, obj, cam, ws, hits, tgt, bg=BG_EXACT, loss=loss,
                               flags=vs.VS_FLAG_LOSS_L1)
    L, dL = oracle.l1_loss_grad(ref_rgba, tgt64)
    ref, sc = oracle.backward(scene, cam, ref_hits, dL, bg=BG_EXACT, with_scale=True, weight_err=ETA_W)
    assert abs(loss.item() - L) <= 1e-5 * L + 1e-9
    w = assert_grad_bar(grads, ref, sc, grad_tol_of(scene))
    print(f"l1 loss grad worst err / per-texel 1e-5 bar {w:.2e}")
    assert vs.read_stats(ws)["device_status"] == 0


@pytest.mark.parametrize("attenuate", [False, True])
def test_autograd_function(vs, ctx, attenuate):
    flags = vs.VS_FLAG_ALPHA_ATTEN if attenuate else 0
    (scene, cams), = synth.config_scene("c1", scale=0.25)
    cam = cams[0]
    obj = vs.ShellObject.from_scene(ctx, scene)
    ws = vs.make_workspace(ctx, [obj], [cam])
    tex = [t.clone().requires_grad_(True) for t in obj.textures]
    obj2 = vs.ShellObject(ctx, [dict(s, tex=t) for s, t in zip(obj.shells, tex)])
    out = vs.VSRender.apply(ctx, obj2, cam, ws, (0.0, 0.0, 0.0), flags, *tex)
    w = torch.randn_like(out[..., :3])
    (out[..., :3] * w).sum().backward()
    out2, hits = vs.render(ctx, obj, cam, ws, flags=flags)
    assert torch.equal(out, out2)
    ref = vs.render_backward(ctx, obj, cam, ws, hits, w, flags=flags)
    for t, r in zip(tex, ref):
        # same kernel, same hits: only the order of the float atomics differs
        assert (t.grad - r).abs().max().item() <= 1e-5 * r.abs().max().item()


# ----------------------------------------------------------------------------
# near-plane clipping (close-up views)
# ----------------------------------------------------------------------------

def _closeup_cameras():
    return [synth.look_at((0.0, -1.45, 0.25), width=96, height=80, fov_y_deg=60.0, znear=0.6),
            synth.look_at((0.9, -0.9, 0.6), width=77, height=64, fov_y_deg=70.0, znear=0.55),
            synth.look_at((0.2, 0.3, 1.2), width=64, height=64, fov_y_deg=50.0, znear=0.4)]


@pytest.mark.parametrize("fmt", ["rgba", "sh", "baked"])
def test_clipped_close_ups_match_oracle(vs, ctx, fmt):
    """Cameras close to the shells with the near plane through them: hit IDs
    bit-exact (clipped parts rasterized from the same cut points), colours
    within the format's bar, clipped triangles counted."""
    if fmt == "rgba":
        geo = synth.concentric_icospheres([1.0, 0.9, 0.8], subdiv=3)
        rng = np.random.default_rng(40)
        sc = Scene([Shell(p, u, t, rng.uniform(0.1, 0.9, (32, 32, 4)).astype(np.float32), FMT_RGBA_F32)
                    for p, u, t in geo])
    elif fmt == "sh":
        (sc, _), = synth.config_scene("c2", scale=0.004, views=1)
    else:
        sc = _baked_scene(3, 30, 64, 2, 1, seed=7)
    clipped = 0
    for cam in _closeup_cameras():
        out, hits, st, obj, ws = gpu_render(vs, ctx, sc, cam, bg=(0.1, 0.2, 0.3))
        ref, ref_hits, frags = oracle.render(sc, cam, bg=(0.1, 0.2, 0.3))
        assert np.array_equal(hits, ref_hits), f"{(hits != ref_hits).sum()} hit IDs differ"
        assert np.abs(out - ref).max() <= tol_of(sc)
        assert st["fragments"] == frags.sum()
        ostats = oracle.raster_scene(sc, cam)[2].sum(0)
        assert st["tris_clipped"] == ostats[4] and st["tris_culled_near"] == ostats[2]
        clipped += st["tris_clipped"]
    assert clipped > 100


def test_clipped_batch_and_backward_match(vs, ctx):
    """Clipped views in a batch are bit-identical to vs_render, and the
    adjoint of a clipped close-up matches the oracle's."""
    geo = synth.concentric_icospheres([1.0, 0.9], subdiv=3)
    rng = np.random.default_rng(41)
    sc = Scene([Shell(p, u, t, rng.uniform(0.1, 0.9, (16, 16, 4)).astype(np.float32), FMT_RGBA_F32)
                for p, u, t in geo])
    cams = _closeup_cameras()
    items, objs, ws = _batch_setup(vs, ctx, [(sc, cams)], True)
    vs.render_batch(ctx, items, ws, do_backward=True)
    assert vs.read_stats(ws)["device_status"] == 0
    plain = [torch.zeros_like(g) for g in items[0]["grads"]]
    for it in items:
        ws1 = vs.make_workspace(ctx, [it["obj"]], [it["cam"]])
        out, hits = vs.render(ctx, it["obj"], it["cam"], ws1)
        assert torch.equal(out, it["out"]) and torch.equal(hits, it["hits"])
        vs.render_backward(ctx, it["obj"], it["cam"], ws1, hits, it["grad_rgb"], grads=plain)
    for a, b in zip(items[0]["grads"], plain):
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-6 * b.abs().max().item())
    w, *_ = check_backward(vs, ctx, sc, cams[0], (0.2, 0.3, 0.4))
    print(f"clipped close-up grad worst err / per-texel 1e-5 bar {w:.2e}")


# ----------------------------------------------------------------------------
# per-layer buffers (Figs. S1/S3)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["c2", "baked", "closeup"])
def test_layer_buffers_match_oracle(vs, ctx, case):
    if case == "c2":
        (sc, cams), = synth.config_scene("c2", scale=0.004, views=2)
        cam, flags = cams[1], vs.VS_FLAG_ALPHA_ATTEN
    elif case == "baked":
        sc, cam, flags = _baked_scene(3, 24, 64, 3, 1, seed=2), synth.look_at((1.0, -2.5, 1.0), width=70, height=56), 0
    else:
        geo = synth.concentric_icospheres([1.0, 0.9], subdiv=3)
        rng = np.random.default_rng(43)
        sc = Scene([Shell(p, u, t, rng.uniform(0.1, 0.9, (16, 16, 4)).astype(np.float32), FMT_RGBA_F32)
                    for p, u, t in geo])
        cam, flags = _closeup_cameras()[0], 0
    obj = vs.ShellObject.from_scene(ctx, sc)
    ws = vs.make_workspace(ctx, [obj], [cam])
    out, hits, lay = vs.render_layers(ctx, obj, cam, ws, bg=(0.1, 0.2, 0.3), flags=flags)
    assert vs.read_stats(ws)["device_status"] == 0
    plain, plain_hits = vs.render(ctx, obj, cam, ws, bg=(0.1, 0.2, 0.3), flags=flags)
    assert torch.equal(hits, plain_hits)
    assert (out - plain).abs().max().item() <= 1e-6
    ref_lay, ref = oracle.layers(sc, cam, hits.cpu().numpy(), bg=(0.1, 0.2, 0.3), flags=flags)
    lay = lay.cpu().numpy()
    tol = tol_of(sc)
    assert np.abs(lay[..., 0:3] - ref_lay[..., 0:3]).max() <= 1e-5      # normals
    assert np.abs(lay[..., 3:5] - ref_lay[..., 3:5]).max() <= 1e-5      # uv
    assert np.abs(lay[..., 5:10] - ref_lay[..., 5:10]).max() <= tol     # opacity, weight, rgb
    assert np.all(lay[..., 10:] == 0)


# ----------------------------------------------------------------------------
# transparency attenuation (Sec. 3): alpha * (2 sigmoid(10 |v . n|) - 1)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("name,scale", [("c1", 1.0), ("c2", 0.01), ("c5", 0.0005)])
def test_alpha_atten_forward_matches_oracle(vs, ctx, name, scale):
    (scene, cams), = synth.config_scene(name, scale=scale, views=2)[:1]
    cam = cams[-1]
    bg = (0.3, 0.2, 0.1)
    err, obj, ws, hits = check_forward(vs, ctx, scene, cam, bg=bg, flags=vs.VS_FLAG_ALPHA_ATTEN)
    plain, plain_hits, *_ = gpu_render(vs, ctx, scene, cam, bg, obj=obj)
    assert np.array_equal(plain_hits, hits)                 # visibility is unchanged
    out, *_ = gpu_render(vs, ctx, scene, cam, bg, obj=obj, flags=vs.VS_FLAG_ALPHA_ATTEN)
    assert np.abs(out - plain).max() > 1e-2                 # and the flag does something
    print(f"{name} attenuated colour err {err:.2e}")


@pytest.mark.parametrize("name,scale", [("c1", 0.25), ("c2", 0.005), ("c5", 0.0004)])
def test_alpha_atten_backward_matches_oracle(vs, ctx, name, scale):
    (sc, cams), = synth.config_scene(name, scale=scale, views=1)[:1]
    w, *_ = check_backward(vs, ctx, sc, cams[0], (0.2, 0.3, 0.4), flags=vs.VS_FLAG_ALPHA_ATTEN)
    print(f"{name} attenuated grad worst err / per-texel 1e-5 bar {w:.2e}")


# ----------------------------------------------------------------------------
# the baked format: RGBA SH bytes, per-band resolutions (Sec. 3 "Mixed
# Resolutions", "Squeezing and Quantization", "Baking Textures")
# ----------------------------------------------------------------------------

def _baked_scene(k, n_lat, tex, degree, shift, seed=0):
    shells = []
    for i, (pos, uv, tris) in enumerate(synth.displaced_shells(k, n_lat, seed=seed)):
        buf = synth.baked_sh_texture(tex, tex, degree, shift, np.random.default_rng(100 * seed + i))
        shells.append(Shell(pos, uv, tris, buf, synth.FMT_SH_U8, degree, tex_w=tex, tex_h=tex, band_shift=shift))
    return Scene(shells)


@pytest.mark.parametrize("degree,shift", [(0, 0), (1, 1), (2, 0), (3, 1), (3, 2)])
def test_baked_forward_matches_oracle(vs, ctx, degree, shift):
    sc = _baked_scene(3, 24, 64, degree, shift, seed=degree)
    for cam in (synth.look_at((0.3, -3.2, 1.1), width=97, height=61),
                synth.look_at((-2.0, 1.5, 2.0), width=64, height=64)):
        err, *_ = check_forward(vs, ctx, sc, cam, bg=(0.2, 0.1, 0.3), tol=TOL_U8)
        print(f"baked deg {degree} shift {shift}: max colour error {err:.2e}")


def test_baked_c2b_views_match_oracle(vs, ctx):
    (sc, cams), = synth.config_scene("c2b", scale=0.01, views=3)
    for cam in cams:
        err, *_ = check_forward(vs, ctx, sc, cam, tol=TOL_U8)
        print(f"c2b scaled view: max colour error {err:.2e}")


def test_baked_with_attenuation_matches_oracle(vs, ctx):
    sc = _baked_scene(2, 20, 32, 2, 1, seed=5)
    cam = synth.look_at((2.5, -1.5, 1.0), width=80, height=72)
    check_forward(vs, ctx, sc, cam, bg=(0.0, 0.3, 0.1), tol=TOL_U8, flags=vs.VS_FLAG_ALPHA_ATTEN)


def test_baked_batches_bit_identical_to_plain(vs, ctx):
    """A baked-only batch (compiled for the class) and a batch mixing baked,
    FP16 SH and FP32 RGBA objects (decided per shell) both give vs_render's
    bits."""
    baked = [(_baked_scene(3, 20, 64, 3, 1, seed=s), [synth.look_at((0.5 * s, -3.0, 1.0), width=70, height=50)])
             for s in range(3)]
    sh = synth.config_scene("c4", scale=0.001, views=1)[:2]
    (c1, c1cams), = synth.config_scene("c1", scale=0.25)
    for objs_cams in (baked, baked + sh + [(c1, c1cams)]):
        items, objs, ws = _batch_setup(vs, ctx, objs_cams, False)
        vs.render_batch(ctx, items, ws, bg=(0.1, 0.2, 0.3))
        assert vs.read_stats(ws)["device_status"] == 0
        for it in items:
            ws1 = vs.make_workspace(ctx, [it["obj"]], [it["cam"]])
            out, hits = vs.render(ctx, it["obj"], it["cam"], ws1, bg=(0.1, 0.2, 0.3))
            assert torch.equal(out, it["out"])
            assert torch.equal(hits, it["hits"])


def test_baked_shells_have_no_gradient(vs, ctx):
    from paper_2409_02482_gb300._abi import VS_ERR_UNSUPPORTED, VSError
    sc = _baked_scene(2, 16, 32, 1, 1)
    cam = synth.look_at((0.0, -3.0, 0.5), width=32, height=32)
    obj = vs.ShellObject.from_scene(ctx, sc)
    ws = vs.make_workspace(ctx, [obj], [cam])
    out, hits = vs.render(ctx, obj, cam, ws)
    g = torch.zeros((32, 32, 3), device="cuda")
    grads = [torch.zeros(1024, device="cuda") for _ in range(obj.k)]
    with pytest.raises(VSError) as e:
        vs.render_backward(ctx, obj, cam, ws, hits, g, grads=grads)
    assert e.value.status == VS_ERR_UNSUPPORTED
    items = [dict(obj=obj, cam=cam, out=out, grad_rgb=g, grads=grads)]
    with pytest.raises(VSError) as e:
        vs.render_batch(ctx, items, ws, do_backward=True)
    assert e.value.status == VS_ERR_UNSUPPORTED


# ----------------------------------------------------------------------------
# batch
# ----------------------------------------------------------------------------

def _batch_setup(vs, ctx, objs_cams, do_bwd, with_targets=False, grad_pitch=None):
    items, objs = [], []
    for sc, cams in objs_cams:
        obj = vs.ShellObject.from_scene(ctx, sc, grad_pitch=grad_pitch)
        objs.append(obj)
        grads = obj.zero_grads() if do_bwd else None
        for cam in cams:
            it = dict(obj=obj, cam=cam, scene=sc,
                      out=torch.empty((cam.height, cam.width, 4), device="cuda"),
                      hits=torch.empty((obj.k, cam.height, cam.width), dtype=torch.int32, device="cuda"),
                      grads=grads)
            if do_bwd:
                it["grad_rgb"] = torch.randn((cam.height, cam.width, 3), device="cuda",
                                             generator=torch.Generator("cuda").manual_seed(len(items)))
                it["loss"] = torch.zeros(1, device="cuda")
            items.append(it)
    ws = vs.make_workspace(ctx, [it["obj"] for it in items], [it["cam"] for it in items])
    return items, objs, ws


def test_batch_in_workspace_sized_runs(vs, ctx):
    """A workspace too small for the whole batch runs it as consecutive
    launches over runs of items: forward bit-identical to the one-launch
    batch, fused gradients equal up to float-atomic order, one table upload
    + persistent kernel per run; a workspace smaller than one item is
    refused before anything runs."""
    from paper_2409_02482_gb300._abi import VSError
    (sc, cams), = synth.config_scene("c2", scale=0.004, views=5)
    items, objs, ws = _batch_setup(vs, ctx, [(sc, cams)], True)
    vs.render_batch(ctx, items, ws, do_backward=True, flags=vs.VS_FLAG_LOSS_L2)
    ref_out = [it["out"].clone() for it in items]
    ref_hits = [it["hits"].clone() for it in items]
    ref_g = [g.clone() for g in items[0]["grads"]]
    one = vs.workspace_size(ctx, [objs[0]], cams[:1])
    small = ws[: 2 * one + 4096].clone().zero_()   # about two items per run
    for g in items[0]["grads"]:
        g.zero_()
    for it in items:
        it["out"].fill_(float("nan"))
        it["hits"].fill_(-9)
    vs.read_stats(small, reset=True)
    vs.render_batch(ctx, items, small, do_backward=True, flags=vs.VS_FLAG_LOSS_L2)
    st = vs.read_stats(small)
    assert st["device_status"] == 0
    assert st["launches"] >= 3 * 2      # at least three runs: upload + kernel each
    for it, o, h in zip(items, ref_out, ref_hits):
        assert torch.equal(it["out"], o) and torch.equal(it["hits"], h)
    for a, b in zip(items[0]["grads"], ref_g):
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-6 * b.abs().max().item())
    with pytest.raises(VSError, match="WORKSPACE"):
        vs.render_batch(ctx, items, ws[: one // 2], do_backward=True, flags=vs.VS_FLAG_LOSS_L2)


def test_batch_forward_bit_identical_to_plain(vs, ctx):
    objs_cams = synth.config_scene("c4", scale=0.003, views=2)[:6]
    items, objs, ws = _batch_setup(vs, ctx, objs_cams, False)
    bg = (0.1, 0.2, 0.3)
    vs.render_batch(ctx, items, ws, bg=bg)
    st = vs.read_stats(ws, reset=True)
    assert st["device_status"] == 0
    total = 0
    for it in items:
        ws1 = vs.make_workspace(ctx, [it["obj"]], [it["cam"]])
        out, hits = vs.render(ctx, it["obj"], it["cam"], ws1, bg=bg)
        assert torch.equal(out, it["out"])
        assert torch.equal(hits, it["hits"])
        total += vs.read_stats(ws1)["fragments"]
    assert st["fragments"] == total
    # and against the oracle for two of them
    for it in items[:2]:
        ref, ref_hits, _ = oracle.render(it["scene"], it["cam"], bg=bg)
        assert np.array_equal(it["hits"].cpu().numpy(), ref_hits)
        assert np.abs(it["out"].cpu().numpy() - ref).max() <= TOL_F16


def test_batch_results_do_not_depend_on_item_order(vs, ctx):
    """The library runs a batch's items grouped by object in a chain of
    nearby cameras, whatever the caller's order: items of three objects
    given interleaved, and the same items reversed, land in their own
    buffers -- colours and hits bit-identical to the grouped order, texel
    gradients equal up to float-atomic order, per-item losses equal."""
    objs_cams = synth.config_scene("c4", scale=0.002, views=3)[:3]
    items, objs, ws = _batch_setup(vs, ctx, objs_cams, True)
    vs.render_batch(ctx, items, ws, do_backward=True, flags=vs.VS_FLAG_LOSS_L2)
    ref = [(it["out"].clone(), it["hits"].clone(), it["loss"].clone()) for it in items]
    ref_g = [[g.clone() for g in o_grads] for o_grads in (its["grads"] for its in items[::3])]
    inter = [items[v + 3 * o] for v in range(3) for o in range(3)]   # A0 B0 C0 A1 B1 C1 ...
    for order in (inter, inter[::-1]):
        for obj in objs:
            for g in _obj_grads(items, obj):
                g.zero_()
        for it in items:
            it["out"].fill_(float("nan"))
            it["hits"].fill_(-9)
            it["loss"].zero_()
        vs.render_batch(ctx, order, ws, do_backward=True, flags=vs.VS_FLAG_LOSS_L2)
        assert vs.read_stats(ws, reset=True)["device_status"] == 0
        for it, (o, h, l) in zip(items, ref):
            assert torch.equal(it["out"], o) and torch.equal(it["hits"], h)
            assert torch.allclose(it["loss"], l, rtol=1e-5)
        for it, gs in zip(items[::3], ref_g):
            for a, b in zip(it["grads"], gs):
                assert torch.allclose(a, b, rtol=1e-4, atol=1e-6 * b.abs().max().item())


def _obj_grads(items, obj):
    return next(it["grads"] for it in items if it["obj"] is obj)


@pytest.mark.parametrize("mode", ["plain", "attenuate", "l1"])
def test_batch_fused_backward_matches_plain(vs, ctx, mode):
    flags = {"plain": 0, "attenuate": vs.VS_FLAG_ALPHA_ATTEN, "l1": vs.VS_FLAG_LOSS_L1}[mode]
    objs_cams = synth.config_scene("c4", scale=0.002, views=2)[:4]
    items, objs, ws = _batch_setup(vs, ctx, objs_cams, True)
    vs.render_batch(ctx, items, ws, do_backward=True, flags=flags)
    assert vs.read_stats(ws)["device_status"] == 0
    for obj, (sc, cams) in zip(objs, objs_cams):
        its = [it for it in items if it["obj"] is obj]
        plain = [torch.zeros_like(g) for g in its[0]["grads"]]
        for it in its:
            ws1 = vs.make_workspace(ctx, [obj], [it["cam"]])
            out, hits = vs.render(ctx, obj, it["cam"], ws1, flags=flags)
            assert torch.equal(out, it["out"])
            vs.render_backward(ctx, obj, it["cam"], ws1, hits, it["grad_rgb"], grads=plain, flags=flags)
        for a, b in zip(its[0]["grads"], plain):
            assert torch.allclose(a, b, rtol=1e-4, atol=1e-6 * b.abs().max().item())


@pytest.mark.parametrize("raster_tris,shade_pixels,blocks", [(32, 32, 1), (2048, 4096, 0), (64, 1024, 2)])
def test_batch_tuning_changes_launch_shape_not_results(vs, ctx, raster_tris, shade_pixels, blocks):
    """Any unit size and grid gives the same forward bits as vs_render, and
    the same fused gradients up to float-atomic order."""
    objs_cams = synth.config_scene("c4", scale=0.002, views=2)[:3]
    items, objs, ws = _batch_setup(vs, ctx, objs_cams, True)
    kmax = max(o.k for o in objs)
    t = vs.tuning(raster_tris, shade_pixels, blocks)
    vs.set_batch_tuning(ctx, t, do_backward=True, k_max=kmax)
    vs.set_batch_tuning(ctx, t, do_backward=False, k_max=kmax)
    try:
        got = vs.get_batch_tuning(ctx, do_backward=True, k_max=kmax)
        assert (got.raster_tris, got.shade_pixels, got.blocks_per_sm) == (raster_tris, shade_pixels, blocks)
        vs.render_batch(ctx, items, ws, do_backward=True)
        assert vs.read_stats(ws)["device_status"] == 0
        for obj in objs:
            its = [it for it in items if it["obj"] is obj]
            plain = [torch.zeros_like(g) for g in its[0]["grads"]]
            for it in its:
                ws1 = vs.make_workspace(ctx, [obj], [it["cam"]])
                out, hits = vs.render(ctx, obj, it["cam"], ws1)
                assert torch.equal(out, it["out"])
                assert torch.equal(hits, it["hits"])
                vs.render_backward(ctx, obj, it["cam"], ws1, hits, it["grad_rgb"], grads=plain)
            for a, b in zip(its[0]["grads"], plain):
                assert torch.allclose(a, b, rtol=1e-4, atol=1e-6 * b.abs().max().item())
        # forward-only batch with the same shape
        for it in items:
            it["out"].fill_(float("nan"))
        vs.render_batch(ctx, items, ws)
        ref, ref_hits, _ = oracle.render(items[0]["scene"], items[0]["cam"])
        assert np.array_equal(items[0]["hits"].cpu().numpy(), ref_hits)
        assert np.abs(items[0]["out"].cpu().numpy() - ref).max() <= TOL_F16
    finally:
        vs.set_batch_tuning(ctx, vs.tuning(), do_backward=True, k_max=0)
        vs.set_batch_tuning(ctx, vs.tuning(), do_backward=False, k_max=0)


def test_autotune_batch_picks_and_keeps_a_valid_shape(vs, ctx):
    objs_cams = synth.config_scene("c4", scale=0.002, views=2)[:4]
    items, objs, ws = _batch_setup(vs, ctx, objs_cams, True)
    kmax = max(o.k for o in objs)
    try:
        best = vs.autotune_batch(ctx, items, ws, do_backward=True, repeats=1)
        assert best.raster_tris in (64, 128, 256, 512, 1024)
        assert best.shade_pixels in (64, 128, 256, 512, 1024)
        assert best.blocks_per_sm >= 1
        kept = vs.get_batch_tuning(ctx, do_backward=True, k_max=kmax)
        assert kept.as_dict() == best.as_dict()
        assert vs.read_stats(ws, reset=True)["device_status"] == 0
        # the tuned launch still renders what vs_render renders
        vs.render_batch(ctx, items, ws, do_backward=True)
        assert vs.read_stats(ws)["device_status"] == 0
        for it in items[:3]:
            ws1 = vs.make_workspace(ctx, [it["obj"]], [it["cam"]])
            out, _ = vs.render(ctx, it["obj"], it["cam"], ws1)
            assert torch.equal(out, it["out"])
        from paper_2409_02482_gb300._abi import VSError
        with pytest.raises(VSError):
            vs.autotune_batch(ctx, items, ws, repeats=0)
    finally:
        vs.set_batch_tuning(ctx, vs.tuning(), do_backward=True, k_max=0)


def test_batch_stall_hook_times_out_and_context_survives(vs, ctx):
    objs_cams = synth.config_scene("c4", scale=0.001, views=1)[:2]
    items, objs, ws = _batch_setup(vs, ctx, objs_cams, False)
    vs.render_batch(ctx, items, ws, flags=1 << 30)
    st = vs.read_stats(ws, reset=True)
    assert st["device_status"] == -6          # VS_ERR_TIMEOUT
    vs.render_batch(ctx, items, ws)
    st = vs.read_stats(ws, reset=True)
    assert st["device_status"] == 0
    ref, ref_hits, _ = oracle.render(items[0]["scene"], items[0]["cam"])
    assert np.array_equal(items[0]["hits"].cpu().numpy(), ref_hits)


def test_batch_graph_capture_replays(vs, ctx):
    objs_cams = synth.config_scene("c4", scale=0.001, views=2)[:3]
    items, objs, ws = _batch_setup(vs, ctx, objs_cams, False)
    bi = vs.BatchItems(items)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        vs.render_batch(ctx, bi, ws, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    first = [it["out"].clone() for it in items]
    for it in items:
        it["out"].zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        vs.render_batch(ctx, bi, ws, stream=torch.cuda.current_stream())
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for a, it in zip(first, items):
        assert torch.equal(a, it["out"])
    assert vs.read_stats(ws)["device_status"] == 0


# ----------------------------------------------------------------------------
# full-size workloads (the launch configuration the benchmark times)
# ----------------------------------------------------------------------------

# ----------------------------------------------------------------------------
# compiled texel classes: the kernels the fused step runs on aligned texels
# (256-bit SH loads, per-pixel SH basis, triangle records, cooperative
# scatter), checked against the oracle and shown to be the ones that ran
# ----------------------------------------------------------------------------

def _class_scene(fmt, deg, pitch, k=3, n_lat=20, tex=64, seed=0):
    rng = np.random.default_rng(50 + deg)
    shells = []
    for pos, uv, tris in synth.displaced_shells(k, n_lat, seed=seed):
        if fmt == FMT_RGBA_F32:
            shells.append(Shell(pos, uv, tris, synth.rgba_texture(tex, tex, rng), FMT_RGBA_F32))
        else:
            shells.append(Shell(pos, uv, tris, synth.sh_texture(tex, tex, deg, rng, sigma=0.4, pitch=pitch),
                                FMT_SH_F16, deg))
    return Scene(shells)


# (format, SH degree, texel pitch with 32-byte-aligned texels, kernel class)
CLASS_CASES = [(FMT_RGBA_F32, 0, 4, 2), (FMT_SH_F16, 0, 8, 3), (FMT_SH_F16, 1, 16, 4), (FMT_SH_F16, 2, 32, 5),
               (FMT_SH_F16, 3, 64, 6)]


@pytest.mark.parametrize("fmt,deg,pitch,kclass", CLASS_CASES)
def test_class_kernels_match_oracle(vs, ctx, fmt, deg, pitch, kclass):
    """Fused batch (forward + adjoint of two views into shared gradients) and
    the plain render / render_backward pair, both on the class kernels,
    against the oracle: hits exact, colours and gradients to FP32 rounding."""
    sc = _class_scene(fmt, deg, pitch)
    cams = [synth.look_at((0.3, -2.6, 0.9), width=96, height=72),
            synth.look_at((-1.9, -1.2, -0.7), width=80, height=88)]
    bg = (0.1, 0.2, 0.3)
    items, objs, ws = _batch_setup(vs, ctx, [(sc, cams)], True)
    vs.render_batch(ctx, items, ws, bg=bg, do_backward=True)
    st = vs.read_stats(ws, reset=True)
    assert st["device_status"] == 0
    assert st["kernel_class"] == kclass
    nch = 4 if fmt == FMT_RGBA_F32 else 1 + 3 * (deg + 1) ** 2
    ref_sum = None
    for it in items:
        ref, ref_hits, _ = oracle.render(sc, it["cam"], bg=bg)
        assert np.array_equal(it["hits"].cpu().numpy(), ref_hits)
        assert np.abs(it["out"].cpu().numpy() - ref).max() <= 2e-5
        rg, rs = oracle.backward(sc, it["cam"], ref_hits, it["grad_rgb"].cpu().numpy().astype(np.float64), bg=bg,
                                 with_scale=True, weight_err=ETA_W)
        if ref_sum is None:
            ref_sum, scale_sum = rg, rs
        else:
            ref_sum = [a + b for a, b in zip(ref_sum, rg)]
            scale_sum = tuple([a + b for a, b in zip(x, y)] for x, y in zip(scale_sum, rs))
        # plain pair on the same class kernels, this view alone
        ws1 = vs.make_workspace(ctx, [objs[0]], [it["cam"]])
        out1, hits1 = vs.render(ctx, objs[0], it["cam"], ws1, bg=bg)
        assert torch.equal(out1, it["out"]) and torch.equal(hits1, it["hits"])
        g1 = vs.render_backward(ctx, objs[0], it["cam"], ws1, hits1, it["grad_rgb"], bg=bg)
        assert vs.read_stats(ws1)["kernel_class"] == kclass
        w1 = assert_grad_bar(g1, rg, rs, grad_tol_of(sc), nch=nch)
    w2 = assert_grad_bar(items[0]["grads"], ref_sum, scale_sum, grad_tol_of(sc), nch=nch)
    print(f"class {kclass} grad worst err / per-texel 1e-5 bar: plain {w1:.2e}, fused batch {w2:.2e}")


@pytest.mark.parametrize("deg,pitch,gpitch,kclass", [(2, 32, 28, 5), (3, 64, 52, 6), (1, 16, 13, 1)])
def test_gradient_pitch_without_padding(vs, ctx, deg, pitch, gpitch, kclass):
    """Gradient arrays with their own pitch (here the value count: no
    padding) while the texels keep theirs: the fused batch and the plain
    adjoint against the oracle, per texel value.  A 16-byte-aligned gradient
    pitch keeps the class kernels; an odd one (13 floats) runs the generic
    kernels with scalar reductions."""
    sc = _class_scene(FMT_SH_F16, deg, pitch)
    cams = [synth.look_at((0.3, -2.6, 0.9), width=96, height=72),
            synth.look_at((-1.9, -1.2, -0.7), width=80, height=88)]
    bg = (0.1, 0.2, 0.3)
    items, objs, ws = _batch_setup(vs, ctx, [(sc, cams)], True, grad_pitch=gpitch)
    assert items[0]["grads"][0].shape[2] == gpitch
    vs.render_batch(ctx, items, ws, bg=bg, do_backward=True)
    st = vs.read_stats(ws, reset=True)
    assert st["device_status"] == 0 and st["kernel_class"] == kclass
    nch = 1 + 3 * (deg + 1) ** 2
    ref_sum = scale_sum = None
    for it in items:
        ref, ref_hits, _ = oracle.render(sc, it["cam"], bg=bg)
        assert np.array_equal(it["hits"].cpu().numpy(), ref_hits)
        rg, rs = oracle.backward(sc, it["cam"], ref_hits, it["grad_rgb"].cpu().numpy().astype(np.float64), bg=bg,
                                 with_scale=True, weight_err=ETA_W)
        ws1 = vs.make_workspace(ctx, [objs[0]], [it["cam"]])
        g1 = vs.render_backward(ctx, objs[0], it["cam"], ws1, it["hits"], it["grad_rgb"], bg=bg)
        assert g1[0].shape[2] == gpitch
        assert_grad_bar(g1, rg, rs, TOL_F16, nch=nch)
        if ref_sum is None:
            ref_sum, scale_sum = rg, rs
        else:
            ref_sum = [a + b for a, b in zip(ref_sum, rg)]
            scale_sum = tuple([a + b for a, b in zip(x, y)] for x, y in zip(scale_sum, rs))
    w = assert_grad_bar(items[0]["grads"], ref_sum, scale_sum, TOL_F16, nch=nch)
    print(f"grad pitch {gpitch}: worst err / per-texel 1e-5 bar {w:.2e}")


def test_unaligned_texels_take_the_generic_kernels(vs, ctx):
    """A pitch that breaks 32-byte alignment keeps SH degree 2 on the generic
    kernels, with the same results."""
    sc = _class_scene(FMT_SH_F16, 2, 28)
    cam = synth.look_at((0.3, -2.6, 0.9), width=64, height=48)
    w, obj, ws, hits, grads = check_backward(vs, ctx, sc, cam, (0.1, 0.2, 0.3))
    assert vs.read_stats(ws)["kernel_class"] == 1


def test_c2_full_size_views(vs, ctx):
    (scene, cams), = synth.config_scene("c2", views=100)
    obj = vs.ShellObject.from_scene(ctx, scene)
    for cam in (cams[0], cams[57]):
        err, *_ = check_forward(vs, ctx, scene, cam, bg=(0.0, 0.0, 0.0), tol=TOL_F16)
        print(f"c2 full view err {err:.3e}")


def test_c2_full_size_fused_batch_matches_oracle(vs, ctx):
    """The benchmark's configuration at full size: c2 (7 shells x ~200k
    faces, 2048^2 SH2 FP16 texels at pitch 32), views in one fused forward +
    adjoint batch with the L2 loss, on the compiled SH2 class with the
    autotuned launch shape.  Hits of every view exact, colours within the
    FP16 SH bar, the gradients summed over the batch within each texel
    value's own bar, against the oracle."""
    (scene, cams), = synth.config_scene("c2", views=100, pitch=32)
    views = [cams[0], cams[57]]
    obj = vs.ShellObject.from_scene(ctx, scene)
    H, W = views[0].height, views[0].width
    tgt = np.random.default_rng(5).random((len(views), H, W, 3)).astype(np.float32)
    targets = torch.from_numpy(tgt).cuda()
    grads = [torch.zeros(t.shape, dtype=torch.float32, device="cuda") for t in obj.textures]
    losses = torch.zeros(len(views), device="cuda")
    items = [dict(obj=obj, cam=c, out=torch.empty((H, W, 4), device="cuda"),
                  hits=torch.empty((obj.k, H, W), dtype=torch.int32, device="cuda"), grad_rgb=targets[i],
                  grads=grads, loss=losses[i:i + 1]) for i, c in enumerate(views)]
    bi = vs.BatchItems(items)
    ws = vs.make_workspace(ctx, [obj] * len(views), views)
    vs.autotune_batch(ctx, bi, ws, do_backward=True, flags=vs.VS_FLAG_LOSS_L2)
    for g in grads:
        g.zero_()
    vs.read_stats(ws, reset=True)
    vs.render_batch(ctx, bi, ws, do_backward=True, flags=vs.VS_FLAG_LOSS_L2)
    st = vs.read_stats(ws)
    assert st["device_status"] == 0
    assert st["kernel_class"] == 1 + 2 + 2   # SH degree 2 class
    terms = []
    for i, it in enumerate(items):
        ref, ref_hits, _ = oracle.render(scene, it["cam"])
        assert np.array_equal(it["hits"].cpu().numpy(), ref_hits)
        err = np.abs(it["out"].cpu().numpy() - ref).max()
        assert err <= TOL_F16
        t64 = tgt[i].astype(np.float64)
        _, dL = oracle.l2_loss_grad(ref, t64)
        terms.append((it["cam"], ref_hits, dL, oracle.l2_loss_scale(ref, t64)))
    w = assert_grad_bar_by_shell(scene, terms, grads, TOL_F16, nch=28)
    print(f"c2 full-size fused batch grad worst err / per-texel 1e-5 bar {w:.2e}")



# ----------------------------------------------------------------------------
# the remaining configurations at full size, one view each
# ----------------------------------------------------------------------------

def _host_mem_available_gb():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    return 0.0


def test_c3_full_size_fused_view_matches_oracle(vs, ctx):
    """The texture-fitting configuration at full size: 9 shells x ~500k
    faces, 2048^2 SH2 FP16 texels (pitch 32, the SH2 class), one 1024^2 view
    in a fused forward + adjoint batch with the L2 loss against a target
    rendered by the oracle from the second seeded texture set; FP32
    gradients without padding (pitch 28).  Hits exact, colours within the
    FP16 bar, every texel value of the gradient within its own bar."""
    (scene, cams), = synth.config_scene("c3", views=64, pitch=32)
    (tscene, _), = synth.config_scene("c3", views=64, pitch=32, tex_seed=1)
    cam = cams[37]
    target = oracle.render(tscene, cam)[0][..., :3]
    del tscene
    obj = vs.ShellObject.from_scene(ctx, scene, grad_pitch=28)
    H, W = cam.height, cam.width
    tgt32 = target.astype(np.float32)
    grads = obj.zero_grads()
    loss = torch.zeros(1, device="cuda")
    it = dict(obj=obj, cam=cam, out=torch.empty((H, W, 4), device="cuda"),
              hits=torch.empty((obj.k, H, W), dtype=torch.int32, device="cuda"),
              grad_rgb=torch.from_numpy(tgt32).cuda(), grads=grads, loss=loss)
    ws = vs.make_workspace(ctx, [obj], [cam])
    vs.render_batch(ctx, [it], ws, do_backward=True, flags=vs.VS_FLAG_LOSS_L2)
    st = vs.read_stats(ws)
    assert st["device_status"] == 0 and st["kernel_class"] == 1 + 2 + 2
    ref, ref_hits, frags = oracle.render(scene, cam)
    assert np.array_equal(it["hits"].cpu().numpy(), ref_hits)
    assert st["fragments"] == frags.sum()
    assert np.abs(it["out"].cpu().numpy() - ref).max() <= TOL_F16
    t64 = tgt32.astype(np.float64)
    L, dL = oracle.l2_loss_grad(ref, t64)
    assert abs(loss.item() - L) <= 1e-5 * L
    w = assert_grad_bar_by_shell(scene, [(cam, ref_hits, dL, oracle.l2_loss_scale(ref, t64))], grads, TOL_F16,
                                 nch=28)
    print(f"c3 full-size view: {frags.sum()} fragments, grad worst err / per-texel 1e-5 bar {w:.2e}")


def test_c4_full_size_uneven_items_match_oracle(vs, ctx):
    """The uneven multi-object configuration at full size (32 objects, k in
    {3, 5, 7, 9}, 10k-1M faces per shell, 1024^2 SH1 FP16 texels at pitch
    16, the SH1 class): the two objects with the most faces, one view each
    at different resolutions, in ONE fused forward + adjoint batch with the
    L2 loss against uniform targets.  Per item: hits exact, colours within
    the FP16 bar, the loss against the oracle's, every texel value of the
    gradient within its own bar."""
    objs_cams = synth.config_scene("c4", views=8, pitch=16)
    order = sorted(range(len(objs_cams)), key=lambda o: -sum(s.tris.shape[0] for s in objs_cams[o][0].shells))
    picks = []
    for o in order[:2]:
        sc, cams = objs_cams[o]
        cam = max(cams, key=lambda c: c.width * c.height) if not picks else min(cams, key=lambda c: c.width * c.height)
        picks.append((sc, cam))
    del objs_cams
    rng = np.random.default_rng(21)
    items = []
    for sc, cam in picks:
        obj = vs.ShellObject.from_scene(ctx, sc)
        H, W = cam.height, cam.width
        tgt = rng.random((H, W, 3), dtype=np.float32)
        items.append(dict(obj=obj, cam=cam, scene=sc, tgt=tgt, out=torch.empty((H, W, 4), device="cuda"),
                          hits=torch.empty((obj.k, H, W), dtype=torch.int32, device="cuda"),
                          grad_rgb=torch.from_numpy(tgt).cuda(), grads=obj.zero_grads(),
                          loss=torch.zeros(1, device="cuda")))
    ws = vs.make_workspace(ctx, [it["obj"] for it in items], [it["cam"] for it in items])
    vs.render_batch(ctx, items, ws, do_backward=True, flags=vs.VS_FLAG_LOSS_L2)
    st = vs.read_stats(ws)
    assert st["device_status"] == 0 and st["kernel_class"] == 1 + 2 + 1
    for it in items:
        sc, cam = it["scene"], it["cam"]
        ref, ref_hits, frags = oracle.render(sc, cam)
        assert np.array_equal(it["hits"].cpu().numpy(), ref_hits)
        assert np.abs(it["out"].cpu().numpy() - ref).max() <= TOL_F16
        t64 = it["tgt"].astype(np.float64)
        L, dL = oracle.l2_loss_grad(ref, t64)
        assert abs(it["loss"].item() - L) <= 1e-5 * L
        w = assert_grad_bar_by_shell(sc, [(cam, ref_hits, dL, oracle.l2_loss_scale(ref, t64))], it["grads"],
                                     TOL_F16, nch=13)
        print(f"c4 full-size item k={sc.k} {cam.width}x{cam.height}: "
              f"{frags.sum()} fragments, grad worst err / per-texel bar {w:.2e}")


def test_c5_full_size_view_matches_oracle(vs, ctx):
    """The large configuration at full size: 9 shells x ~2M faces, 4096^2
    SH3 FP16 texels (pitch 64, the SH3 class; ~19 GB), one 3840x2160 view.
    The fused forward + adjoint batch (L2 loss, gradient pitch 52): hits
    exact, colours within the FP16 bar, loss against the oracle's.  The
    standalone adjoint with an output gradient on a random 1 % of the pixels
    (the oracle's FP64 adjoint skips the rest): every texel value within its
    own bar."""
    if _host_mem_available_gb() < 64 or torch.cuda.mem_get_info()[0] < 80 * 2 ** 30:
        pytest.skip("needs ~64 GB of host and ~80 GB of device memory")
    (scene, cams), = synth.config_scene("c5", views=256, pitch=64)
    cam = cams[101]
    obj = vs.ShellObject.from_scene(ctx, scene, grad_pitch=52)
    H, W = cam.height, cam.width
    rng = np.random.default_rng(9)
    tgt32 = rng.random((H, W, 3), dtype=np.float32)
    grads = obj.zero_grads()
    loss = torch.zeros(1, device="cuda")
    it = dict(obj=obj, cam=cam, out=torch.empty((H, W, 4), device="cuda"),
              hits=torch.empty((obj.k, H, W), dtype=torch.int32, device="cuda"),
              grad_rgb=torch.from_numpy(tgt32).cuda(), grads=grads, loss=loss)
    ws = vs.make_workspace(ctx, [obj], [cam])
    vs.render_batch(ctx, [it], ws, do_backward=True, flags=vs.VS_FLAG_LOSS_L2)
    st = vs.read_stats(ws, reset=True)
    assert st["device_status"] == 0 and st["kernel_class"] == 1 + 2 + 3
    ref, ref_hits, frags = oracle.render(scene, cam)
    assert np.array_equal(it["hits"].cpu().numpy(), ref_hits)
    assert st["fragments"] == frags.sum()
    assert np.abs(it["out"].cpu().numpy() - ref).max() <= TOL_F16
    L, _ = oracle.l2_loss_grad(ref, tgt32.astype(np.float64))
    assert abs(loss.item() - L) <= 1e-5 * L
    del grads, it
    g = rng.standard_normal((H, W, 3)) * (rng.random((H, W, 1)) < 0.01)
    g32 = g.astype(np.float32)
    got = vs.render_backward(ctx, obj, cam, ws, torch.from_numpy(ref_hits).cuda(), torch.from_numpy(g32).cuda())
    assert vs.read_stats(ws)["device_status"] == 0
    w = assert_grad_bar_by_shell(scene, [(cam, ref_hits, g32.astype(np.float64), None)], got, TOL_F16, nch=49)
    print(f"c5 full-size view: {frags.sum()} fragments, sampled-pixel grad worst err / per-texel 1e-5 bar {w:.2e}")
