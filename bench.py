"""Benchmark of the k-shell renderer hot path on GB300.

Workload (N = 1): 7 nested noise-displaced shells of ~200k triangles each,
2048^2 FP16 textures of one alpha logit + degree-2 RGB SH coefficients
(28 values = 56 B per texel), 100 views of 800x800 on a hemisphere at
distance 4 (the synthetic stand-in for the paper's object scenes).

One step = one texture-fitting pass over all 100 views in ONE persistent
launch (vs_render_batch, do_backward=1, VS_FLAG_LOSS_L2): rasterize every
shell with its nearest-hit test, shade and composite (forward), and
accumulate the FP32 texel gradients of the mean-squared error against
per-view target images (backward) -- every row of the hot path.  Inputs are
resident in HBM and larger than L2 (1.6 GB texels, 3.3 GB gradients, 0.8 GB
targets), so no L2 flush is needed between steps.

Printed: ONE JSON line (rank 0).  `value` = fragments composited per second
(pixel-shell pairs with a hit) over the whole job.  Extras: forward-only
batched throughput, the plain per-view launch loop and the batched/plain
ratio, images/s, the roofline of the persistent kernel, the oracle timed on
the host cores, an end-to-end number with host<->device copies, clocks.

--impl reference times the FP64 CPU oracle (the reference arm for this
build) on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fragments composited/s and fwd+bwd images/s, batched vs plain, at ≤1e-5 err"
WORKLOAD = ("k=7 noise-displaced shells x ~200k tris, 2048^2 FP16 alpha+SH2 textures, "
            "100 views 800x800 on a hemisphere at r=4")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--views", type=int, default=100)
    p.add_argument("--scale", type=float, default=1.0, help="shrink the workload (testing only)")
    p.add_argument("--pitch", type=int, default=32,
                   help="FP16 values per texel in memory (28 used; 32 = 64-byte texels)")
    p.add_argument("--grad-pitch", type=int, default=0,
                   help="FP32 values per gradient texel (0 = the texel pitch; 28 = no padding)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-uneven", action="store_true", help="skip the uneven 32-object batch")
    p.add_argument("--no-baked", action="store_true", help="skip the baked-format forward leg")
    p.add_argument("--baked-scale", type=float, default=1.0, help="shrink the baked leg (profiling only)")
    p.add_argument("--baked-views", type=int, default=100)
    p.add_argument("--no-latency", action="store_true", help="skip the single-view latency leg")
    p.add_argument("--no-c3", action="store_true", help="skip the full-size k=9 / 1024^2 fitting leg")
    p.add_argument("--no-c5", action="store_true", help="skip the full-size k=9 / 4K / SH3 leg")
    p.add_argument("--c5-views", type=int, default=256)
    p.add_argument("--c5-ws-gb", type=float, default=48.0,
                   help="workspace budget of the 4K leg (its batch runs in workspace-sized runs)")
    p.add_argument("--no-ntex", action="store_true", help="skip the neural-texture fitting leg")
    p.add_argument("--no-autotune", action="store_true",
                   help="keep the default work-unit sizes instead of autotuning them first")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = []
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            rows.append(parts)
        os.unlink(self.f.name)
        return rows

    @staticmethod
    def summarize(rows):
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        pw = [float(r[4]) for r in rows if r[4].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------
# workload
# ----------------------------------------------------------------------------
def build_workload(args, device, rank=0, world=1):
    """The C2 fitting workload of this rank: with N ranks the step's view
    list has N x args.views views, dealt round-robin (shard.view_shard), so
    every rank renders args.views views (weak scaling)."""
    import torch
    import synth
    import paper_2409_02482_gb300 as vs
    from paper_2409_02482_gb300.shard import view_shard
    (scene, cams), = synth.config_scene("c2", scale=args.scale, views=args.views * world, pitch=args.pitch)
    cams = [cams[v] for v in view_shard(len(cams), rank, world)]
    ctx = vs.Context(device.index or 0)
    obj = vs.ShellObject.from_scene(ctx, scene, device=device, grad_pitch=args.grad_pitch or None)
    H, W = cams[0].height, cams[0].width
    g = torch.Generator(device=device).manual_seed(1)
    targets = torch.rand((len(cams), H, W, 3), device=device, generator=g)
    outs = torch.empty((len(cams), H, W, 4), device=device)
    losses = torch.zeros(len(cams), device=device)
    grads = obj.zero_grads()
    items = [dict(obj=obj, cam=c, out=outs[i], grad_rgb=targets[i], grads=grads, loss=losses[i:i + 1])
             for i, c in enumerate(cams)]
    ws = vs.make_workspace(ctx, [obj] * len(cams), cams, device=device)
    return dict(scene=scene, cams=cams, ctx=ctx, obj=obj, targets=targets, outs=outs, losses=losses,
                grads=grads, items=vs.BatchItems(items), ws=ws, H=H, W=W)


def uneven_batch(ctx, device, stream, steps, autotune=True):
    """The uneven batch: 32 objects with k in {3,5,7,9}, 10k-1M faces per
    shell, 8 views each at 512^2 / 800^2 / 1024^2 / 1920x1080, 1024^2 SH1
    FP16 textures (pitch 16), fused fwd+bwd with the L2 loss -- one
    persistent launch vs the plain per-view loop of vs_render +
    vs_render_backward.  Geometry from the seeded generator; texel values
    and targets are drawn on the device (only their shape and distribution
    matter for timing)."""
    import torch
    import synth
    import paper_2409_02482_gb300 as vs
    objs = synth.config_scene("c4", views=8, pitch=16, textures=False)
    g = torch.Generator(device=device).manual_seed(4)
    items, objects = [], []
    for sc, cams in objs:
        shells = []
        for s_ in sc.shells:
            h, w, pitch = s_.tex.shape
            tex = torch.zeros((h, w, pitch), dtype=torch.float16, device=device)
            tex[..., :s_.channels] = (0.3 * torch.randn((h, w, s_.channels), device=device, generator=g)).half()
            shells.append(dict(pos=torch.from_numpy(s_.pos).to(device), uv=torch.from_numpy(s_.uv).to(device),
                               tris=torch.from_numpy(s_.tris).to(device), tex=tex, fmt=s_.fmt, degree=s_.degree))
        obj = vs.ShellObject(ctx, shells)
        objects.append(obj)
        grads = [torch.zeros(t.shape, dtype=torch.float32, device=device) for t in obj.textures]
        for cam in cams:
            items.append(dict(obj=obj, cam=cam, grads=grads,
                              out=torch.empty((cam.height, cam.width, 4), device=device),
                              grad_rgb=torch.rand((cam.height, cam.width, 3), device=device, generator=g),
                              loss=torch.zeros(1, device=device)))
    ws = vs.make_workspace(ctx, [it["obj"] for it in items], [it["cam"] for it in items], device=device)
    bi = vs.BatchItems(items)
    flags = vs.VS_FLAG_LOSS_L2

    def batched():
        vs.render_batch(ctx, bi, ws, do_backward=True, flags=flags, stream=stream)

    tuning = (vs.autotune_batch(ctx, bi, ws, do_backward=True, flags=flags, stream=stream).as_dict()
              if autotune else None)
    vs.read_stats(ws, reset=True)
    batched()
    st = vs.read_stats(ws, reset=True)
    assert st["device_status"] == 0, st
    frags = st["fragments"]
    ms_b = timed(batched, steps, 2, stream, lambda: None)
    kmax = max(o.k for o in objects)
    hmax = max(it["cam"].height * it["cam"].width for it in items)
    ws1 = torch.zeros(max(vs.workspace_size(ctx, [it["obj"]], [it["cam"]]) for it in items),
                      dtype=torch.uint8, device=device)
    hits_buf = torch.empty(kmax * hmax, dtype=torch.int32, device=device)

    def plain():
        for it in items:
            c = it["cam"]
            hits = hits_buf[: it["obj"].k * c.height * c.width].view(it["obj"].k, c.height, c.width)
            vs.render(ctx, it["obj"], c, ws1, out=it["out"], hits=hits, stream=stream)
            vs.render_backward(ctx, it["obj"], c, ws1, hits, it["grad_rgb"], grads=it["grads"],
                               loss=it["loss"], flags=flags, stream=stream)

    ms_p = timed(plain, max(1, steps // 2), 1, stream, lambda: None)
    out = {"workload": "32 objects x 8 views, k in {3,5,7,9}, 10k-1M faces/shell, 512^2..1920x1080, "
                       "1024^2 SH1 FP16, fused fwd+bwd, L2 loss",
           "items": len(items), "triangles": int(sum(sum(s.tris.shape[0] for s in sc.shells) for sc, _ in objs)),
           "fragments_per_step": frags, "batched_ms": ms_b, "plain_ms": ms_p, "batched_vs_plain": ms_p / ms_b,
           "tuning": tuning,
           "batched_fragments_per_s": frags / (ms_b * 1e-3), "batched_images_per_s": len(items) / (ms_b * 1e-3)}
    del ws, ws1, items, objects, bi
    torch.cuda.empty_cache()
    return out


def baked_leg(ctx, device, stream, steps, peak, autotune=True, scale=1.0, views=100):
    """The paper's deployed path: forward rendering of baked assets (Sec. 3
    "Baking Textures"; its Tab. 2 real-time renderer) -- the c2 geometry and
    100 views at 800x800 with RGBA SH degree 3 bytes, 2048^2 base halving per
    band (the paper's mixed resolutions), one persistent launch per step.
    Roofline bytes per fragment: the distinct texels of each band (oracle
    footprint count on views 0/49/99) times the band's real bytes per texel
    4 (2l + 1), plus geometry and the image as for the main workload."""
    import torch
    import oracle
    import synth
    import paper_2409_02482_gb300 as vs
    (sc, cams), = synth.config_scene("c2b", scale=scale, views=views)
    obj = vs.ShellObject.from_scene(ctx, sc, device=device)
    H, W = cams[0].height, cams[0].width
    outs = torch.empty((len(cams), H, W, 4), device=device)
    items = vs.BatchItems([dict(obj=obj, cam=c, out=outs[i]) for i, c in enumerate(cams)])
    ws = vs.make_workspace(ctx, [obj] * len(cams), cams, device=device)

    def step():
        vs.render_batch(ctx, items, ws, stream=stream)

    tuning = vs.autotune_batch(ctx, items, ws, stream=stream).as_dict() if autotune else None
    vs.read_stats(ws, reset=True)
    step()
    st = vs.read_stats(ws, reset=True)
    assert st["device_status"] == 0, st
    frags = st["fragments"]
    ms = timed(step, steps, 3, stream, lambda: None)
    band_bytes = np.array([4 * (2 * band + 1) for band in range(4)])
    D = F = 0
    sampled = sorted({0, len(cams) // 2, len(cams) - 1})
    for i in sampled:
        hits, _, _ = oracle.raster_scene(sc, cams[i])
        D += float((oracle.footprint_texels_baked(sc, cams[i], hits) * band_bytes).sum())
        F += int((hits >= 0).sum())
    per_frag = D / max(F, 1)
    n = len(cams)
    geo = n * sum(20 * sh.pos.shape[0] + 12 * sh.tris.shape[0] for sh in sc.shells)
    img = n * H * W * 16
    b_alg = frags * per_frag + geo + img
    achieved = b_alg / (ms * 1e-3) / 1e9
    out = {"workload": "c2 geometry (7 shells x ~200k tris), 100 views 800x800, baked RGBA SH3 bytes, "
                       "2048^2 base halving per band, forward only",
           "ms_per_step": ms, "fragments_per_step": frags, "fragments_per_s": frags / (ms * 1e-3),
           "images_per_s": n / (ms * 1e-3), "tuning": tuning,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "texel_bytes_per_fragment": per_frag,
                        "algorithmic_bytes_per_launch": b_alg, "d_sampled_views": sampled}}
    del ws, items, outs, obj
    torch.cuda.empty_cache()
    return out


def device_textures(scene, device, seed, sigma=0.3):
    """FP16 texel arrays shaped like the scene's, every real value drawn
    N(0, sigma) on the device (the generator's distribution; only shape and
    distribution matter for timing), padding zero."""
    import torch
    g = torch.Generator(device=device).manual_seed(seed)
    out = []
    for s_ in scene.shells:
        h, w, pitch = s_.tex.shape
        t = torch.zeros((h, w, pitch), dtype=torch.float16, device=device)
        for r0 in range(0, h, 1024):   # bounded FP32 temporaries
            r1 = min(h, r0 + 1024)
            t[r0:r1, :, :s_.channels] = (sigma * torch.randn((r1 - r0, w, s_.channels), device=device,
                                                              generator=g)).half()
        out.append(t)
    return out


def config_leg(name, ctx, device, stream, steps, peak, autotune=True, views=None, ws_gb=None):
    """A full-size fitting configuration besides the main one, forward + adjoint
    and forward only, as batched persistent launches:
      c3: 9 shells x ~500k faces, 2048^2 SH2 FP16 (texel pitch 32, gradient
          pitch 28), 64 views at 1024^2 on the hemisphere at 4, L2 loss
          against targets rendered from a second seeded texture set;
      c5: 9 shells x ~2M faces, 4096^2 SH3 FP16 (texel pitch 64, gradient
          pitch 52), 256 views at 3840x2160 on the sphere at 3.5, L2 loss
          against random targets; the batch runs in workspace-sized runs
          (ws_gb) -- 256 views at 4K would need ~600 MB of visibility words
          and ~1.2 GB of triangle records per view at once.
    Texel values are drawn on the device.  Roofline bytes as for the main
    workload with D from the oracle's footprint count on the middle view."""
    import torch
    import oracle
    import synth
    import paper_2409_02482_gb300 as vs
    pitch, gpitch = {"c3": (32, 28), "c5": (64, 52)}[name]
    (sc, cams), = synth.config_scene(name, views=views, pitch=pitch, textures=False)
    texs = device_textures(sc, device, seed=10)
    shells = [dict(pos=torch.from_numpy(s_.pos).to(device), uv=torch.from_numpy(s_.uv).to(device),
                   tris=torch.from_numpy(s_.tris).to(device), tex=t, fmt=s_.fmt, degree=s_.degree,
                   grad_pitch=gpitch) for s_, t in zip(sc.shells, texs)]
    obj = vs.ShellObject(ctx, shells)
    n, H, W = len(cams), cams[0].height, cams[0].width
    per_item = vs.workspace_size(ctx, [obj], cams[:1])
    full = vs.workspace_size(ctx, [obj] * n, cams)
    budget = full if ws_gb is None else min(full, max(int(ws_gb * 2 ** 30), 2 * per_item))
    ws = torch.zeros(budget, dtype=torch.uint8, device=device)
    if name == "c3":   # targets: the same views rendered from a second seeded texture set
        tex2 = device_textures(sc, device, seed=11)
        obj2 = vs.ShellObject(ctx, [dict(s_, tex=t) for s_, t in zip(shells, tex2)])
        t4 = torch.empty((n, H, W, 4), device=device)
        vs.render_batch(ctx, [dict(obj=obj2, cam=c, out=t4[i]) for i, c in enumerate(cams)], ws, stream=stream)
        targets = t4[..., :3].contiguous()
        del t4, tex2, obj2
    else:
        targets = torch.rand((n, H, W, 3), device=device, generator=torch.Generator(device=device).manual_seed(12))
    outs = torch.empty((n, H, W, 4), device=device)
    grads = obj.zero_grads()
    losses = torch.zeros(n, device=device)
    items = vs.BatchItems([dict(obj=obj, cam=c, out=outs[i], grad_rgb=targets[i], grads=grads,
                                loss=losses[i:i + 1]) for i, c in enumerate(cams)])
    fwd_items = vs.BatchItems([dict(obj=obj, cam=c, out=outs[i]) for i, c in enumerate(cams)])
    flags = vs.VS_FLAG_LOSS_L2
    tuning = None
    if autotune:   # on the items of one run (the shape carries over to every run)
        m = max(1, min(n, budget // per_item - 1))
        sub = vs.BatchItems([dict(obj=obj, cam=c, out=outs[i], grad_rgb=targets[i], grads=grads,
                                  loss=losses[i:i + 1]) for i, c in enumerate(cams[:m])])
        sub_f = vs.BatchItems([dict(obj=obj, cam=c, out=outs[i]) for i, c in enumerate(cams[:m])])
        tuning = {"fwd_bwd": vs.autotune_batch(ctx, sub, ws, do_backward=True, flags=flags,
                                               stream=stream).as_dict(),
                  "fwd": vs.autotune_batch(ctx, sub_f, ws, stream=stream).as_dict(), "tuned_on_views": m}
        for g_ in grads:
            g_.zero_()

    def step():
        vs.render_batch(ctx, items, ws, do_backward=True, flags=flags, stream=stream)

    def step_fwd():
        vs.render_batch(ctx, fwd_items, ws, stream=stream)

    vs.read_stats(ws, reset=True)
    step()
    st = vs.read_stats(ws, reset=True)
    assert st["device_status"] == 0, st
    frags, launches = st["fragments"], st["launches"]
    ms = timed(step, steps, 1, stream, lambda: None)
    ms_f = timed(step_fwd, steps, 1, stream, lambda: None)
    mid = n // 2
    hits, _, _ = oracle.raster_scene(sc, cams[mid])
    d_per_frag = float(oracle.footprint_texels(sc, cams[mid], hits).sum()) / max(int((hits >= 0).sum()), 1)
    wl = {"scene": sc, "cams": cams, "H": H, "W": W}
    b_alg, parts = algorithmic_bytes(wl, frags / n, d_per_frag, True)
    b_fwd, _ = algorithmic_bytes(wl, frags / n, d_per_frag, False)
    out = {"workload": synth.CONFIGS[name], "views": n, "image": f"{W}x{H}", "shells": obj.k,
           "tris_per_shell": int(sc.shells[0].tris.shape[0]), "texture": f"{sc.shells[0].tex.shape[1]}^2 SH"
           f"{sc.shells[0].degree} FP16, texel pitch {pitch}, gradient pitch {gpitch}",
           "workspace_bytes": budget, "workspace_bytes_one_launch": full, "launches_per_step": launches,
           "tuning": tuning, "fragments_per_step": frags,
           "fwd_bwd": {"ms_per_step": ms, "fragments_per_s": frags / (ms * 1e-3), "images_per_s": n / (ms * 1e-3),
                       "roofline": {"bound": "hbm", "achieved": b_alg / (ms * 1e-3) / 1e9, "peak": peak,
                                    "unit": "GB/s", "frac": b_alg / (ms * 1e-3) / 1e9 / peak,
                                    "algorithmic_bytes_per_step": b_alg, "bytes_breakdown": parts}},
           "fwd": {"ms_per_step": ms_f, "fragments_per_s": frags / (ms_f * 1e-3), "images_per_s": n / (ms_f * 1e-3),
                   "roofline_frac": b_fwd / (ms_f * 1e-3) / 1e9 / peak},
           "distinct_texels_per_fragment": d_per_frag, "d_sampled_views": [mid]}
    del items, fwd_items, ws, outs, targets, grads, obj, texs, shells
    torch.cuda.empty_cache()
    return out


def ntex_leg(wl, device, stream, steps, tensor_cores=False):
    """Texture fitting with neural textures on the main workload (Sec. 3
    "Texturing Meshes"): per shell two networks (opacity: 1 output; colour:
    27 SH-2 outputs), 16-level hash grids with 2^19 rows and 2 features, two
    64-wide ReLU layers (the supplement's sizes), evaluated at all 2048^2
    texel centres into the FP16 texture, then the fused render + adjoint of
    the 100 views, the networks' adjoints and Adam -- one fitting step.
    Times each part with CUDA events; random initial parameters."""
    import torch
    import synth
    import paper_2409_02482_gb300 as vs
    ctx, obj, items, ws = wl["ctx"], wl["obj"], wl["items"], wl["ws"]
    nets = []
    for i, tex in enumerate(obj.textures):
        h, w, _ = tex.shape
        pair = []
        for j, (ch0, c) in enumerate(((0, 1), (1, 27))):
            nt = vs.NeuralTexture(ctx, levels=16, features=2, log2_table=19, base_res=16, growth=1.447,
                                  hidden=64, out_ch=c, tex_w=w, tex_h=h, device=device,
                                  tensor_cores=tensor_cores)
            shapes = [("table", (16, 1 << 19, 2)), ("W0", (64, 32)), ("b0", (64,)), ("W1", (64, 64)),
                      ("b1", (64,)), ("W2", (c, 64)), ("b2", (c,))]
            nt.params.copy_(torch.from_numpy(synth.ntex_init(shapes, np.random.default_rng(100 * i + j))))
            pair.append((nt, ch0))
        nets.append(pair)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    parts = np.zeros(4)

    def step(record):
        if record:
            ev[0].record(stream)
        for pair, tex in zip(nets, obj.textures):
            for nt, ch0 in pair:
                nt.forward(tex, ch0=ch0, stream=stream)
        if record:
            ev[1].record(stream)
        for g in wl["grads"]:
            g.zero_()
        vs.render_batch(ctx, items, ws, do_backward=True, flags=vs.VS_FLAG_LOSS_L2, stream=stream)
        if record:
            ev[2].record(stream)
        for pair, g in zip(nets, wl["grads"]):
            for nt, ch0 in pair:
                nt.grads.zero_()
                nt.backward(g, ch0=ch0, stream=stream)
        if record:
            ev[3].record(stream)
        for pair in nets:
            for nt, _ in pair:
                nt.adam(1e-2, stream=stream)
        if record:
            ev[4].record(stream)

    for _ in range(2):
        step(False)
    torch.cuda.synchronize()
    for _ in range(steps):
        step(True)
        torch.cuda.synchronize()
        parts += [ev[k].elapsed_time(ev[k + 1]) for k in range(4)]
    parts /= steps
    n_tex = sum(t.shape[0] * t.shape[1] for t in obj.textures)
    out = {"workload": "main workload with neural textures: 7 shells x 2 networks (1 + 27 outputs), "
                       "16 levels x 2^19 x 2 hash grids, 2 x 64 ReLU MLP, 2048^2 grounded texels",
           "layers": "TF32 tensor cores" if tensor_cores else "FP32",
           "ms_per_step": float(parts.sum()), "ms_network_forward": float(parts[0]),
           "ms_render_fwd_bwd": float(parts[1]), "ms_network_backward": float(parts[2]),
           "ms_adam": float(parts[3]), "texels_per_step": n_tex,
           "network_evaluations_per_s": 2 * n_tex / (parts[0] * 1e-3)}
    del nets
    torch.cuda.empty_cache()
    return out


def timed(fn, steps, warmup, stream, barrier):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        fn()
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    return t0.elapsed_time(t1) / steps   # ms per step


def kernel_source_hash():
    """sha256 over the renderer's CUDA sources (kernels and the host code that
    shapes their launches; the neural-texture files take no part in them); a
    stored ncu traffic figure is used only while it matches (the kernels have
    not changed since the capture)."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2409_02482_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h")) and not name.startswith("vs_ntex"):
            h.update(name.encode())
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(f.read())
    return h.hexdigest()


def stored_traffic(n_views):
    """DRAM bytes per launch of the persistent kernel from the committed ncu
    capture (profiles/k_persistent_fwdbwd_c2_traffic.json), scaled by views,
    or None when absent or taken on other kernel sources."""
    path = os.path.join(ROOT, "profiles", "k_persistent_fwdbwd_c2_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None, "no stored capture"
    if d.get("kernel_source_sha256") != kernel_source_hash():
        return None, "kernels changed since the capture"
    per_view = (d["dram_bytes_read"] + d["dram_bytes_write"]) / d["views"]
    return per_view * n_views, f"ncu on {d['views']} views, scaled by views"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def algorithmic_bytes(wl, frags_per_view, d_per_frag, with_bwd):
    """Bytes the method itself must move per step (implementation scratch
    such as the per-shell visibility words excluded):
      texels D*s (+ FP32 gradient read-modify-write D*C*8 with backward),
      geometry read once per view (pos 12 B + uv 8 B per vertex, 12 B per
      triangle), image write 16 B/px, target read 12 B/px (backward)."""
    scene = wl["scene"]
    n = len(wl["cams"])
    s = [sh.channels * sh.tex.itemsize for sh in scene.shells]   # padding is not algorithmic
    C = [sh.channels for sh in scene.shells]
    D_total = d_per_frag * frags_per_view * n           # distinct texels over all (view, shell)
    tex = D_total * (sum(s) / len(s))
    grad = D_total * (sum(C) / len(C)) * 8 if with_bwd else 0
    geo = n * sum(20 * sh.pos.shape[0] + 12 * sh.tris.shape[0] for sh in scene.shells)
    img = n * wl["H"] * wl["W"] * (16 + (12 if with_bwd else 0))
    return tex + grad + geo + img, dict(texels=tex, grads=grad, geometry=geo, image=img)


def step_lower_bound_bytes(wl, texels_touched):
    """Per-step lower bound on the bytes of the fused step: every texel any
    view touches moved once per step (value read + FP32 gradient
    read-modify-write), the geometry read once, the images and targets of
    every view.  `texels_touched` counts the texels that received a nonzero
    gradient in one step (all shells)."""
    scene = wl["scene"]
    n = len(wl["cams"])
    s = sum(sh.channels * sh.tex.itemsize for sh in scene.shells) / len(scene.shells)
    C = sum(sh.channels for sh in scene.shells) / len(scene.shells)
    geo = sum(20 * sh.pos.shape[0] + 12 * sh.tris.shape[0] for sh in scene.shells)
    return texels_touched * (s + 8 * C) + geo + n * wl["H"] * wl["W"] * 28


def texels_per_fragment(wl, n_views=3, threads=None):
    """Distinct texels per fragment from the oracle on a few views (the D of
    the algorithmic bytes; the footprints of neighbouring pixels overlap)."""
    import oracle
    cams = wl["cams"]
    idx = np.linspace(0, len(cams) - 1, n_views).astype(int)
    D = F = 0
    for i in idx:
        hits, _, _ = oracle.raster_scene(wl["scene"], cams[i], threads=threads)
        D += int(oracle.footprint_texels(wl["scene"], cams[i], hits).sum())
        F += int((hits >= 0).sum())
    return D / max(F, 1), [int(i) for i in idx]


def cpu_baseline(wl, budget_s=20.0):
    """The oracle, as it stands, on a bounded sample of the workload: full
    fused step (raster, shade, L2 loss gradient, adjoint) for as many views
    as fit in ~budget_s.  Only the oracle's work is timed: each view's
    target image is copied to the host and widened to FP64 outside the
    clock."""
    import oracle
    threads = os.cpu_count() or 1
    dt = 0.0
    frags = 0
    views = 0
    for i, cam in enumerate(wl["cams"]):
        target = wl["targets"][i].cpu().numpy().astype(np.float64)
        t0 = time.perf_counter()
        rgba, hits, fr = oracle.render(wl["scene"], cam, threads=threads)
        _, dL = oracle.l2_loss_grad(rgba, target)
        oracle.backward(wl["scene"], cam, hits, dL)
        dt += time.perf_counter() - t0
        frags += int(fr.sum())
        views += 1
        if dt > budget_s:
            break
    return {"value": frags / dt, "unit": "fragments/s", "cores": threads, "kind": "oracle",
            "sample": f"{views} of {len(wl['cams'])} views, full fused step (raster+shade on {threads} "
                      f"threads, adjoint on 1), {dt:.1f} s of oracle time",
            "images_per_s": views / dt}


def single_view_latency(wl, stream, reps=50):
    """Frame latency of ONE view (the paper's real-time figures are per
    frame): vs_render of view 0 (forward, no hit buffer) and the fused
    forward + backward of that view as a one-item vs_render_batch, each
    timed alone with CUDA events around the call, the L2 flushed (a 256 MB
    write) before every call; median over `reps`.  Also the same forward
    replayed from a captured CUDA graph (launch overhead removed)."""
    import torch
    import paper_2409_02482_gb300 as vs
    ctx, obj, cam = wl["ctx"], wl["obj"], wl["cams"][0]
    dev = wl["targets"].device
    ws1 = vs.make_workspace(ctx, [obj], [cam], device=dev)
    out = torch.empty((wl["H"], wl["W"], 4), device=dev)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    one = vs.BatchItems([dict(obj=obj, cam=cam, out=out, grad_rgb=wl["targets"][0], grads=wl["grads"],
                              loss=wl["losses"][0:1])])

    def fwd():
        vs.render(ctx, obj, cam, ws1, out=out, want_hits=False, stream=stream)

    def fused():
        vs.render_batch(ctx, one, ws1, do_backward=True, flags=vs.VS_FLAG_LOSS_L2, stream=stream)

    def med(fn):
        for _ in range(3):
            fn()
        ts = []
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(reps):
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    ms_fwd = med(fwd)
    # a single view wants smaller work units than the 100-view batch (whose
    # tuning would leave SMs idle): the library's tuner on this one-item
    # batch, untimed, then the batch's tuning restored for the other legs
    k = obj.k
    batch_tuning = vs.get_batch_tuning(ctx, True, k)
    vs.autotune_batch(ctx, one, ws1, do_backward=True, flags=vs.VS_FLAG_LOSS_L2, stream=stream)
    one_tuning = vs.get_batch_tuning(ctx, True, k)
    ms_fused = med(fused)
    vs.set_batch_tuning(ctx, batch_tuning, True, k)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        fwd_side = lambda: vs.render(ctx, obj, cam, ws1, out=out, want_hits=False, stream=side)  # noqa: E731
        fwd_side()
        side.synchronize()
        with torch.cuda.graph(g, stream=side):
            fwd_side()
    stream.wait_stream(side)
    ms_graph = med(g.replay)
    for t in wl["grads"]:
        t.zero_()
    wl["losses"].zero_()
    del ws1, flush
    return {"view": f"view 0 of the workload ({wl['W']}x{wl['H']}, k = {obj.k})",
            "forward_ms": ms_fwd, "forward_frames_per_s": 1e3 / ms_fwd,
            "forward_graph_ms": ms_graph, "forward_graph_frames_per_s": 1e3 / ms_graph,
            "fused_fwd_bwd_ms": ms_fused, "fused_fwd_bwd_frames_per_s": 1e3 / ms_fused,
            "fused_tuning": {"raster_tris": one_tuning.raster_tris, "shade_pixels": one_tuning.shade_pixels,
                             "blocks_per_sm": one_tuning.blocks_per_sm},
            "timing": "CUDA events around each call, L2 flushed before each, median of %d" % reps}


# ----------------------------------------------------------------------------
def run_ours(args):
    import torch
    import paper_2409_02482_gb300 as vs
    ws_n, rank, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if ws_n > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)

        def barrier():
            dist.barrier()
    else:
        def barrier():
            pass
    stream = torch.cuda.current_stream()
    wl = build_workload(args, device, rank, ws_n)
    ctx, ws, items = wl["ctx"], wl["ws"], wl["items"]
    flags = vs.VS_FLAG_LOSS_L2

    def render_views(views):
        assert len(views) == len(wl["cams"])
        vs.render_batch(ctx, items, ws, do_backward=True, flags=flags, stream=stream)

    if ws_n > 1:
        # the view-sharded fitting step: this rank's views in one fused
        # launch, then one all-reduce (sum) of the FP32 texel gradients
        from paper_2409_02482_gb300.shard import ShardedFittingStep
        sharded = ShardedFittingStep(wl["grads"], render_views, args.views * ws_n)

        def step():
            sharded()
    else:
        def step():
            render_views(list(range(len(wl["cams"]))))

    def step_fwd():
        vs.render_batch(ctx, items, ws, do_backward=False, stream=stream)

    # launch shapes (work-unit sizes, grid) timed on this very batch, untimed
    # here; the tuning launches accumulate gradients and losses, so reset them
    tuning = None
    if not args.no_autotune:
        tuning = {"fwd_bwd": vs.autotune_batch(ctx, items, ws, do_backward=True, flags=flags,
                                               stream=stream).as_dict(),
                  "fwd": vs.autotune_batch(ctx, items, ws, do_backward=False, stream=stream).as_dict()}
        for g in wl["grads"]:
            g.zero_()
        wl["losses"].zero_()

    # fragments per step (device counter), status check
    vs.read_stats(ws, reset=True)
    step()
    st = vs.read_stats(ws, reset=True)
    assert st["device_status"] == 0, st
    frags = st["fragments"]
    n_views = len(wl["cams"])
    # texels the step touched (those with a nonzero gradient after this one
    # step from zero), for the per-step lower bound; untimed
    touched = sum(int((g != 0).any(dim=-1).sum().item()) for g in wl["grads"])

    launches = st["launches"]          # kernels the call enqueued, counted by the library

    sampler = ClockSampler(local)
    ms = timed(step, args.steps, args.warmup, stream, barrier)
    clock_rows = sampler.stop()
    ms_fwd = timed(step_fwd, max(3, args.steps // 2), 2, stream, barrier)

    # end to end through the public API with host buffers: every step copies
    # its targets in from pinned host memory and reads its per-view losses
    # back.  Double-buffered like a training loop's input pipeline: two
    # target / loss buffers (two item tables that differ only in those
    # pointers) alternate, step s+1's targets are copied on a second stream
    # while step s computes, and a step waits only for its own inputs.
    host_t = wl["targets"].cpu().pin_memory()
    host_loss = [torch.empty(n_views, dtype=torch.float32).pin_memory() for _ in range(2)]
    tgt = [wl["targets"], torch.empty_like(wl["targets"])]
    los = [wl["losses"], torch.zeros_like(wl["losses"])]
    bufs = [items, vs.BatchItems([dict(obj=wl["obj"], cam=c, out=wl["outs"][i], grad_rgb=tgt[1][i],
                                       grads=wl["grads"], loss=los[1][i:i + 1])
                                  for i, c in enumerate(wl["cams"])])]
    copy_stream = torch.cuda.Stream(device)
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    done = [torch.cuda.Event(), torch.cuda.Event()]
    pipe = {"s": 0}

    def prefetch(b):   # the next step's targets into buffer b, once the step that last read b is done
        copy_stream.wait_event(done[b])
        with torch.cuda.stream(copy_stream):
            tgt[b].copy_(host_t, non_blocking=True)
        ready[b].record(copy_stream)

    def step_e2e():
        b = pipe["s"] % 2
        pipe["s"] += 1
        prefetch(1 - b)
        stream.wait_event(ready[b])
        los[b].zero_()
        vs.render_batch(ctx, bufs[b], ws, do_backward=True, flags=flags, stream=stream)
        if ws_n > 1:   # the sharded step's gradient exchange
            import torch.distributed as dist
            for g in wl["grads"]:
                dist.all_reduce(g)
        host_loss[b].copy_(los[b], non_blocking=True)
        done[b].record(stream)

    for e in done:
        e.record(stream)
    prefetch(0)
    for _ in range(2):   # warm-up
        step_e2e()
    torch.cuda.synchronize()
    barrier()
    k_e2e = max(3, args.steps // 3)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(k_e2e):
        step_e2e()
    stream.wait_event(ready[pipe["s"] % 2])   # the copy issued by the last step counts too
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = t0.elapsed_time(t1) / k_e2e

    if ws_n > 1:
        import torch.distributed as dist
        t = torch.tensor([ms, ms_fwd, ms_e2e], device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, ms_fwd, ms_e2e = t.tolist()
    e2e = {"value": frags * ws_n / (ms_e2e * 1e-3), "unit": "fragments/s",
           "h2d_bytes_per_step": host_t.numel() * 4, "d2h_bytes_per_step": n_views * 4,
           "ms_per_step": ms_e2e, "pipeline": "double-buffered: the next step's H2D copy on a second stream"}

    res = {}
    # plain per-view launch loop (vs_render + vs_render_backward with the L2 flag)
    if not args.no_plain and rank == 0:
        ws1 = vs.make_workspace(ctx, [wl["obj"]], wl["cams"][:1], device=device)
        hits = torch.empty((wl["obj"].k, wl["H"], wl["W"]), dtype=torch.int32, device=device)

        def plain():
            for i, cam in enumerate(wl["cams"]):
                vs.render(ctx, wl["obj"], cam, ws1, out=wl["outs"][i], hits=hits, stream=stream)
                vs.render_backward(ctx, wl["obj"], cam, ws1, hits, wl["targets"][i], grads=wl["grads"],
                                   loss=wl["losses"][i:i + 1], flags=flags, stream=stream)

        def plain_fwd():
            for i, cam in enumerate(wl["cams"]):
                vs.render(ctx, wl["obj"], cam, ws1, out=wl["outs"][i], want_hits=False, stream=stream)

        ms_plain = timed(plain, 3, 1, stream, lambda: None)
        ms_plain_fwd = timed(plain_fwd, 3, 1, stream, lambda: None)
        # where the plain loop's time goes: device time inside the calls (an
        # event pair around each view's vs_render + vs_render_backward) against
        # the loop's span; the rest is the host's launch gaps
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * n_views)]
        torch.cuda.synchronize()
        for i, cam in enumerate(wl["cams"]):
            ev[2 * i].record(stream)
            vs.render(ctx, wl["obj"], cam, ws1, out=wl["outs"][i], hits=hits, stream=stream)
            vs.render_backward(ctx, wl["obj"], cam, ws1, hits, wl["targets"][i], grads=wl["grads"],
                               loss=wl["losses"][i:i + 1], flags=flags, stream=stream)
            ev[2 * i + 1].record(stream)
        torch.cuda.synchronize()
        busy = sum(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(n_views))
        span = ev[0].elapsed_time(ev[-1])
        # the fused kernel of the batch, launched one view at a time: fusion
        # (texels read once, no hit buffer) without the overlap of views
        singles = [vs.BatchItems([dict(obj=wl["obj"], cam=c, out=wl["outs"][i], grad_rgb=wl["targets"][i],
                                       grads=wl["grads"], loss=wl["losses"][i:i + 1])])
                   for i, c in enumerate(wl["cams"])]

        def fused_per_view():
            for one in singles:
                vs.render_batch(ctx, one, ws1, do_backward=True, flags=flags, stream=stream)

        ms_pvf = timed(fused_per_view, 3, 1, stream, lambda: None)
        res["plain_loop"] = {"fwd_bwd_ms_per_step": ms_plain, "fwd_ms_per_step": ms_plain_fwd,
                             "fwd_bwd_fragments_per_s": frags / (ms_plain * 1e-3),
                             "fwd_fragments_per_s": frags / (ms_plain_fwd * 1e-3),
                             "fwd_bwd_device_ms_in_calls": busy, "fwd_bwd_span_ms": span,
                             "fwd_bwd_gaps_ms": span - busy,
                             "fused_kernel_per_view_ms_per_step": ms_pvf}
        res["batched_vs_plain"] = {"fwd_bwd": ms_plain / ms, "fwd": ms_plain_fwd / ms_fwd,
                                   "fused_per_view_vs_plain": ms_plain / ms_pvf,
                                   "batched_vs_fused_per_view": ms_pvf / ms}
    if not args.no_latency and rank == 0:
        res["single_view_latency"] = single_view_latency(wl, stream)
    if not args.no_uneven and rank == 0:
        res["uneven_batch"] = uneven_batch(ctx, device, stream, max(3, args.steps // 10),
                                           autotune=not args.no_autotune)
    if not args.no_ntex and rank == 0:
        res["neural_texture_fitting"] = ntex_leg(wl, device, stream, max(3, args.steps // 10))
        res["neural_texture_fitting_tf32"] = ntex_leg(wl, device, stream, max(3, args.steps // 10),
                                                      tensor_cores=True)
    if not args.no_c3 and rank == 0:
        res["c3_fitting"] = config_leg("c3", ctx, device, stream, max(3, args.steps // 6), peaks()[0],
                                       autotune=not args.no_autotune)
    if not args.no_c5 and rank == 0:
        res["c5_4k"] = config_leg("c5", ctx, device, stream, 2, peaks()[0], autotune=not args.no_autotune,
                                  views=args.c5_views, ws_gb=args.c5_ws_gb)
    if not args.no_baked and rank == 0:
        res["baked_forward"] = baked_leg(ctx, device, stream, max(5, args.steps // 3), peaks()[0],
                                         autotune=not args.no_autotune, scale=args.baked_scale,
                                         views=args.baked_views)

    if rank != 0:
        if ws_n > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    # roofline of the persistent kernel (the only compute kernel of a step)
    peak, peak_kind = peaks()
    d_per_frag, sampled = texels_per_fragment(wl)
    b_alg, parts = algorithmic_bytes(wl, frags / n_views, d_per_frag, True)
    b_fwd, _ = algorithmic_bytes(wl, frags / n_views, d_per_frag, False)
    achieved = b_alg / (ms * 1e-3) / 1e9
    traffic, traffic_note = stored_traffic(n_views)
    achieved_fwd = b_fwd / (ms_fwd * 1e-3) / 1e9
    b_lb = step_lower_bound_bytes(wl, touched)

    out = {
        "metric": METRIC,
        "value": frags * ws_n / (ms * 1e-3),
        "unit": "fragments/s",
        "n_gpus": ws_n,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "step": "batched fused fwd+bwd, L2 loss vs target images, "
                   "one persistent launch", "texel_storage": "f16", "views": n_views,
                   "image": f"{wl['W']}x{wl['H']}", "shells": wl["obj"].k,
                   "tris_per_shell": [int(s.tris.shape[0]) for s in wl["scene"].shells],
                   "l2": "inputs larger than L2 (no flush)",
                   "parallelism": (f"views sharded over {ws_n} ranks ({n_views} each), one gradient "
                                   f"all-reduce per step" if ws_n > 1 else "1 GPU"),
                   "tuning": tuning or "default (256 tris, 256 px, occupancy maximum)"},
        "images_per_s": n_views * ws_n / (ms * 1e-3),
        "fragments_per_step": frags,
        "fwd_only": {"fragments_per_s": frags * ws_n / (ms_fwd * 1e-3), "images_per_s": n_views * ws_n / (ms_fwd * 1e-3),
                     "ms_per_step": ms_fwd,
                     "roofline_frac": achieved_fwd / peak, "achieved_gbs": achieved_fwd},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "traffic_note": traffic_note,
                     "peak_kind": f"{peak_kind} hbm_gbs",
                     "kernel": "vsd::k_persistent", "algorithmic_bytes_per_launch": b_alg,
                     "bytes_breakdown": parts, "distinct_texels_per_fragment": d_per_frag,
                     "d_sampled_views": sampled,
                     "step_lower_bound": {"texels_touched": touched, "bytes": b_lb,
                                          "frac": b_lb / (ms * 1e-3) / 1e9 / peak,
                                          "note": "each touched texel moved once per step (no per-view "
                                                  "re-reads); per-view bytes are the roofline above"}},
        "gpu_launches": launches * args.steps,
        "launches_per_step": launches,
        "kernels": ["vsd::k_upload (item table, %d)" % (launches - 1), "vsd::k_persistent<true> (1)"],
        "e2e": e2e,
        "clocks": ClockSampler.summarize(clock_rows),
    }
    out.update(res)
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl)
    print(json.dumps(out))
    if ws_n > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on this machine's host cores, same
    metric/unit/config, each step a bounded sample (one view's fused step)."""
    ws_n, rank, local = dist_env()
    if rank != 0:
        return
    import synth
    import oracle
    (scene, cams), = synth.config_scene("c2", scale=args.scale, views=args.views)
    H, W = cams[0].height, cams[0].width
    rng = np.random.default_rng(1)
    threads = os.cpu_count() or 1

    def one(i):
        cam = cams[i % len(cams)]
        rgba, hits, fr = oracle.render(scene, cam, threads=threads)
        _, dL = oracle.l2_loss_grad(rgba, rng.random((H, W, 3)))
        oracle.backward(scene, cam, hits, dL)
        return int(fr.sum())

    for i in range(args.warmup):
        one(i)
    t0 = time.perf_counter()
    frags = sum(one(args.warmup + i) for i in range(args.steps))
    dt = time.perf_counter() - t0
    v = frags / dt
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "fragments/s", "n_gpus": ws_n,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "step": "one view's fused fwd+bwd per step (bounded sample)"},
           "cpu_baseline": {"value": v, "unit": "fragments/s", "cores": threads, "kind": "oracle",
                            "sample": f"{args.steps} views, one per step"},
           "e2e": {"value": v, "unit": "fragments/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        if a.steps == 30 and "--steps" not in sys.argv:
            a.steps = 5
        run_reference(a)
    else:
        run_ours(a)
