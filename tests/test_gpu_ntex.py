"""The neural texture on the GPU (through the C ABI) against the FP64
oracle: forward at texel centres, adjoint into the hash tables and MLP,
Adam; and the whole fitting loop of Sec. 3 "Texturing Meshes" -- network ->
grounded texels -> fused render + adjoint -> network adjoint -> Adam --
reducing an image loss."""

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import ntex
from synth import FMT_SH_F16, Scene, Shell

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vs():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2409_02482_gb300 as vs
    return vs


@pytest.fixture(scope="module")
def ctx(vs):
    return vs.Context(0)


CFG = ntex.NtexConfig(levels=8, features=2, log2_table=12, base_res=4, growth=1.6, hidden=64, out_ch=28)


def _params(cfg, seed):
    p = synth.ntex_init(cfg.shapes(), np.random.default_rng(seed))
    lay, _ = cfg.layout()
    off, shp = lay[0][1], lay[0][2]
    n = int(np.prod(shp))
    # tables well away from zero so that every level matters in the check
    p[off:off + n] = np.random.default_rng(seed + 1).normal(0, 0.5, n).astype(np.float32)
    return p


def _net(vs, ctx, cfg, params, W, H):
    nt = vs.NeuralTexture(ctx, cfg.levels, cfg.features, cfg.log2_table, cfg.base_res, cfg.growth, cfg.hidden,
                          cfg.out_ch, tex_w=W, tex_h=H)
    nt.params.copy_(torch.from_numpy(params))
    return nt


@pytest.mark.parametrize("W,H", [(70, 50), (600, 500)])
def test_ntex_forward_matches_oracle(vs, ctx, W, H):
    params = _params(CFG, 1)
    nt = _net(vs, ctx, CFG, params, W, H)
    ref, _ = ntex.forward(CFG, params.astype(np.float64), W, H)
    tex = torch.full((H, W, 32), 7.0, device="cuda")
    nt.forward(tex, ch0=2)
    got = tex.cpu().numpy()
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(got[..., 2:30] - ref).max() <= 1e-4 * scale
    assert np.all(got[..., :2] == 7.0) and np.all(got[..., 30:] == 7.0)
    tex16 = torch.zeros((H, W, 28), dtype=torch.float16, device="cuda")
    nt.forward(tex16)
    assert np.abs(tex16.float().cpu().numpy() - ref).max() <= 2e-3 * scale


def test_ntex_tensor_core_mode_is_close(vs, ctx):
    """TF32 layers (10-bit mantissa inputs, FP32 accumulation) against the
    exact FP32 mode.  Texels agree to the TF32 rounding level.  Gradients are
    compared per parameter block in norm: the backward recomputes the forward
    activations in TF32, so the few hidden pre-activations that TF32 moves
    across zero flip their ReLU mask and add or drop a whole cotangent term.
    With random-sign cotangents the error norm grows like the square root of
    that flip fraction; running this configuration through TF32-rounded GEMM
    inputs in FP64 gives about 2% normwise (4.5% of a block's largest
    entry), and exact activations give 5e-4.  The bar is 4x the former.  b2
    is a plain sum of the cotangent and must agree to FP32 rounding."""
    W, H = 120, 90
    params = _params(CFG, 7)
    nt = _net(vs, ctx, CFG, params, W, H)
    tc = vs.NeuralTexture(ctx, CFG.levels, CFG.features, CFG.log2_table, CFG.base_res, CFG.growth, CFG.hidden,
                          CFG.out_ch, tex_w=W, tex_h=H, tensor_cores=True)
    tc.params.copy_(nt.params)
    a = torch.zeros((H, W, 28), device="cuda")
    b = torch.zeros_like(a)
    nt.forward(a)
    tc.forward(b)
    assert (a - b).abs().max().item() <= 1e-2 * max(1.0, a.abs().max().item())
    assert (a - b).norm().item() <= 2e-3 * a.norm().item()
    g = torch.randn((H, W, 28), device="cuda", generator=torch.Generator("cuda").manual_seed(8))
    nt.backward(g)
    tc.backward(g)
    lay, _ = CFG.layout()
    for name, off, shp in lay:
        n = int(np.prod(shp))
        r, q = nt.grads[off:off + n], tc.grads[off:off + n]
        bar = 1e-5 if name == "b2" else 8e-2
        assert (q - r).norm().item() <= bar * r.norm().item(), name
    assert tc.status() == 0 and nt.status() == 0


# the benchmark's networks: 16 levels x 2 features, 2^19-row tables, two
# 64-wide hidden layers, 1 (opacity) or 27 (SH-2 colour) outputs, 2048^2 texels
BENCH_CFG = dict(levels=16, features=2, log2_table=19, base_res=16, growth=1.447, hidden=64)


@pytest.mark.parametrize("tensor_cores", [False, True])
@pytest.mark.parametrize("out_ch", [1, 27])
def test_ntex_bench_configuration_matches_oracle(vs, ctx, out_ch, tensor_cores):
    """The benchmark's neural texture at full size (one 2048^2 texture),
    forward into FP32 texels and the adjoint of a gradient on 4096 sampled
    texels, against the oracle evaluated on those texels.  FP32 layers: the
    texels within 1e-4 and every parameter block's gradient within 1e-4 of
    its largest entry.  TF32 layers (tcgen05): within the bars derived for
    TF32 (see test_ntex_tensor_core_mode_is_close), and the status word
    clear (no bounded wait ran out)."""
    cfg = ntex.NtexConfig(out_ch=out_ch, **BENCH_CFG)
    W = H = 2048
    params = synth.ntex_init(cfg.shapes(), np.random.default_rng(40 + out_ch))
    lay, _ = cfg.layout()
    off, shp = lay[0][1], lay[0][2]
    n = int(np.prod(shp))
    params[off:off + n] = np.random.default_rng(41).normal(0, 0.5, n).astype(np.float32)
    nt = vs.NeuralTexture(ctx, cfg.levels, cfg.features, cfg.log2_table, cfg.base_res, cfg.growth, cfg.hidden,
                          cfg.out_ch, tex_w=W, tex_h=H, tensor_cores=tensor_cores)
    nt.params.copy_(torch.from_numpy(params))
    tex = torch.zeros((H, W, out_ch), device="cuda")
    nt.forward(tex)
    idx = np.sort(np.random.default_rng(42).choice(W * H, 4096, replace=False))
    ref = ntex.forward_at(cfg, params.astype(np.float64), W, H, idx)
    got = tex.reshape(-1, out_ch).cpu().numpy()[idx].astype(np.float64)
    scale = max(1.0, np.abs(ref).max())
    if tensor_cores:
        assert np.abs(got - ref).max() <= 1e-2 * scale
        assert np.linalg.norm(got - ref) <= 2e-3 * np.linalg.norm(ref)
    else:
        assert np.abs(got - ref).max() <= 1e-4 * scale
    g = np.random.default_rng(43).normal(size=(len(idx), out_ch)).astype(np.float32)
    dense = torch.zeros((H * W, out_ch), device="cuda")
    dense[torch.from_numpy(idx).cuda()] = torch.from_numpy(g).cuda()
    nt.backward(dense.reshape(H, W, out_ch))
    rg = ntex.backward(cfg, params.astype(np.float64), W, H, g.astype(np.float64), texels=idx)
    q = nt.grads.cpu().numpy().astype(np.float64)
    for name, o, sh in lay:
        k = int(np.prod(sh))
        r, v = rg[o:o + k], q[o:o + k]
        if tensor_cores:
            bar = 1e-5 if name == "b2" else 8e-2
            assert np.linalg.norm(v - r) <= bar * np.linalg.norm(r) + 1e-30, name
        else:
            assert np.abs(v - r).max() <= 1e-4 * max(np.abs(r).max(), 1e-30), name
    assert nt.status() == 0


@pytest.mark.parametrize("tensor_cores", [False, True])
def test_ntex_backward_across_chunk_boundaries(vs, ctx, tensor_cores):
    """A 1500 x 800 texture: the adjoint runs in chunks of texels (2^18 for
    FP32 layers, 2^20 for the fused TF32 kernel) that end inside a texel
    row, so the tiles of the encoding's adjoint are cut by a chunk boundary.
    A gradient on sampled texels, among them every texel within 3 of a chunk
    boundary, against the oracle on those texels."""
    W, H = 1500, 800
    params = _params(CFG, 5)
    nt = vs.NeuralTexture(ctx, CFG.levels, CFG.features, CFG.log2_table, CFG.base_res, CFG.growth, CFG.hidden,
                          CFG.out_ch, tex_w=W, tex_h=H, tensor_cores=tensor_cores)
    nt.params.copy_(torch.from_numpy(params))
    rng = np.random.default_rng(6)
    edges = [b + d for b in (1 << 18, 2 << 18, 3 << 18, 4 << 18) for d in range(-3, 3)]
    idx = np.unique(np.concatenate([rng.choice(W * H, 3000, replace=False), edges]))
    g = rng.normal(size=(len(idx), CFG.out_ch)).astype(np.float32)
    dense = torch.zeros((H * W, CFG.out_ch), device="cuda")
    dense[torch.from_numpy(idx).cuda()] = torch.from_numpy(g).cuda()
    nt.backward(dense.reshape(H, W, CFG.out_ch))
    ref = ntex.backward(CFG, params.astype(np.float64), W, H, g.astype(np.float64), texels=idx)
    got = nt.grads.cpu().numpy().astype(np.float64)
    lay, _ = CFG.layout()
    for name, off, shp in lay:
        n = int(np.prod(shp))
        r, q = ref[off:off + n], got[off:off + n]
        if tensor_cores:   # the TF32 bars of test_ntex_bench_configuration_matches_oracle
            bar = 1e-5 if name == "b2" else 8e-2
            assert np.linalg.norm(q - r) <= bar * np.linalg.norm(r) + 1e-30, name
        else:
            assert np.abs(q - r).max() <= 1e-4 * max(np.abs(r).max(), 1e-30), name
    assert nt.status() == 0


@pytest.mark.parametrize("tensor_cores", [False, True])
@pytest.mark.parametrize("levels,features,growth", [(16, 1, 1.25), (6, 3, 1.7), (8, 4, 1.7), (4, 8, 1.7)])
def test_ntex_feature_counts_match_oracle(vs, ctx, levels, features, growth, tensor_cores):
    """Feature counts other than two per level: the generic encoding gather
    and the encoding adjoint's scalar (F = 1, 3) and 16-byte vector (F = 4,
    8) reductions, forward and adjoint against the oracle.  F = 3 has no
    fused TF32 adjoint (16 % F != 0): its adjoint runs the layer GEMMs in
    either mode.  FP32 bars of test_ntex_backward_matches_oracle; TF32 bars
    of test_ntex_tensor_core_mode_is_close.  The finest level stays within
    about one lattice cell per texel, as in the benchmark's network: the
    kernels place texels on the lattice in FP32, whose rounding (N_l 2^-24
    of a cell) reaches the 1e-4 bar only at resolutions far beyond the
    texture's."""
    cfg = ntex.NtexConfig(levels=levels, features=features, log2_table=10, base_res=4, growth=growth, hidden=64,
                          out_ch=9)
    W, H = 150, 110
    params = _params(cfg, 11 + features)
    nt = vs.NeuralTexture(ctx, cfg.levels, cfg.features, cfg.log2_table, cfg.base_res, cfg.growth, cfg.hidden,
                          cfg.out_ch, tex_w=W, tex_h=H, tensor_cores=tensor_cores)
    nt.params.copy_(torch.from_numpy(params))
    tex = torch.zeros((H, W, 12), device="cuda")
    nt.forward(tex, ch0=1)
    ref, _ = ntex.forward(cfg, params.astype(np.float64), W, H)
    got = tex[..., 1:10].cpu().numpy().astype(np.float64).reshape(ref.shape)
    scale = max(1.0, np.abs(ref).max())
    if tensor_cores:
        assert np.linalg.norm(got - ref) <= 2e-3 * np.linalg.norm(ref)
    else:
        assert np.abs(got - ref).max() <= 1e-4 * scale
    g = torch.randn((H, W, 12), device="cuda", generator=torch.Generator("cuda").manual_seed(12))
    nt.backward(g, ch0=1)
    rg = ntex.backward(cfg, params.astype(np.float64), W, H, g.cpu().numpy()[..., 1:10].astype(np.float64))
    q = nt.grads.cpu().numpy().astype(np.float64)
    lay, _ = cfg.layout()
    for name, off, shp in lay:
        n = int(np.prod(shp))
        r, v = rg[off:off + n], q[off:off + n]
        if tensor_cores:
            bar = 1e-5 if name == "b2" else 8e-2
            assert np.linalg.norm(v - r) <= bar * np.linalg.norm(r) + 1e-30, name
        else:
            assert np.abs(v - r).max() <= 1e-4 * max(np.abs(r).max(), 1e-30), name
    assert nt.status() == 0


def test_ntex_backward_matches_oracle(vs, ctx):
    W, H = 70, 50
    params = _params(CFG, 2)
    nt = _net(vs, ctx, CFG, params, W, H)
    g = torch.randn((H, W, 32), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    nt.backward(g, ch0=2)
    got = nt.grads.cpu().numpy()
    ref = ntex.backward(CFG, params.astype(np.float64), W, H, g.cpu().numpy()[..., 2:30].astype(np.float64))
    lay, _ = CFG.layout()
    for name, off, shp in lay:
        n = int(np.prod(shp))
        r, q = ref[off:off + n], got[off:off + n]
        assert np.abs(q - r).max() <= 1e-4 * max(np.abs(r).max(), 1e-30), name


def test_adam_matches_oracle(vs, ctx):
    W, H = 8, 8
    params = _params(CFG, 4)
    nt = _net(vs, ctx, CFG, params, W, H)
    rng = np.random.default_rng(5)
    g = rng.normal(size=params.size).astype(np.float32)
    p, m, v = params.astype(np.float64), np.zeros(params.size), np.zeros(params.size)
    for step in (1, 2, 3):
        nt.grads.copy_(torch.from_numpy(g * step))
        nt.adam(lr=1e-2)
        p, m, v = ntex.adam(p, (g * step).astype(np.float64), m, v, step, lr=1e-2)
    assert np.abs(nt.params.cpu().numpy() - p).max() <= 1e-5
    assert np.abs(nt.m.cpu().numpy() - m).max() <= 1e-5


def test_fitting_through_the_renderer_reduces_the_loss(vs, ctx):
    """Two SH-degree-1 shells, four views: each shell's texture is a neural
    texture (one network, 13 channels: alpha logit + 12 SH coefficients)
    grounded at its 64 x 64 texel centres; 60 steps of fused render + adjoint
    against targets rendered from a random texture set, the texel gradients
    taken back through the networks, Adam."""
    geo = synth.concentric_icospheres([1.0, 0.85], subdiv=3)
    rng = np.random.default_rng(6)
    deg, tw, pitch = 1, 64, 16
    target = Scene([Shell(p, u, t, synth.sh_texture(tw, tw, deg, rng, sigma=0.8, pitch=pitch), FMT_SH_F16, deg)
                    for p, u, t in geo])
    cams = [synth.look_at(e, width=96, height=96) for e in [(0.3, -3.0, 0.8), (2.5, 1.5, 0.5),
                                                              (-2.0, 1.0, 2.0), (0.0, 2.5, -1.5)]]
    tobj = vs.ShellObject.from_scene(ctx, target)
    tws = vs.make_workspace(ctx, [tobj], cams[:1])
    targets = [vs.render(ctx, tobj, c, tws)[0][..., :3].contiguous() for c in cams]
    cfg = ntex.NtexConfig(levels=8, features=2, log2_table=12, base_res=4, growth=1.5, hidden=32, out_ch=13)
    nets, shells = [], []
    for i, (p, u, t) in enumerate(geo):
        nt = _net(vs, ctx, cfg, synth.ntex_init(cfg.shapes(), np.random.default_rng(10 + i)), tw, tw)
        tex = torch.zeros((tw, tw, pitch), dtype=torch.float16, device="cuda")
        nets.append(nt)
        shells.append(dict(pos=torch.from_numpy(p).cuda(), uv=torch.from_numpy(u).cuda(),
                           tris=torch.from_numpy(t).cuda(), tex=tex, fmt=FMT_SH_F16, degree=deg))
    obj = vs.ShellObject(ctx, shells)
    grads = [torch.zeros((tw, tw, pitch), device="cuda") for _ in shells]
    loss = torch.zeros(len(cams), device="cuda")
    items = [dict(obj=obj, cam=c, out=torch.empty((96, 96, 4), device="cuda"), grad_rgb=targets[j], grads=grads,
                  loss=loss[j:j + 1]) for j, c in enumerate(cams)]
    bi = vs.BatchItems(items)
    ws = vs.make_workspace(ctx, [obj] * len(cams), cams)
    history = []
    for step in range(60):
        for nt, sh in zip(nets, shells):
            nt.forward(sh["tex"])
        for g in grads:
            g.zero_()
        loss.zero_()
        vs.render_batch(ctx, bi, ws, do_backward=True, flags=vs.VS_FLAG_LOSS_L2)
        for nt, g in zip(nets, grads):
            nt.grads.zero_()
            nt.backward(g)
            nt.adam(lr=1e-2)
        history.append(loss.sum().item())
    assert vs.read_stats(ws)["device_status"] == 0
    assert all(np.isfinite(history))
    assert history[-1] < 0.5 * history[0], history[::10]
