"""The C-ABI library on the host: it loads, exports every function
include/vs.h declares, and rejects bad arguments before touching a GPU.
No compute call is made here."""

import ctypes
import os
import subprocess

import pytest

from paper_2409_02482_gb300 import _abi


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_abi.LIB_PATH):
        from paper_2409_02482_gb300 import build
        build.build()
    return _abi.load()


def test_exports_every_declared_function(lib):
    declared = _abi.header_functions()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), name
    nm = subprocess.run(["nm", "-D", "--defined-only", _abi.LIB_PATH], capture_output=True, text=True)
    if nm.returncode == 0:
        exported = {line.split()[-1] for line in nm.stdout.splitlines() if " T " in line}
        assert set(declared) <= exported
    # the binding covers exactly what the header declares
    assert set(_abi.SIGNATURES) == set(declared)


def test_struct_layouts_match_header_sizes():
    # sizes implied by the C declarations on LP64
    assert ctypes.sizeof(_abi.vs_camera) == 76
    assert ctypes.sizeof(_abi.vs_shell_desc) == 88
    assert _abi.vs_shell_desc.grad_pitch.offset == 80   # static_assert in vs_api.cu
    assert ctypes.sizeof(_abi.vs_stats) == 80
    assert ctypes.sizeof(_abi.vs_tuning) == 16


def test_create_without_gpu_reports_cuda_error(lib):
    h = ctypes.c_void_p()
    st = lib.vs_create(ctypes.byref(h), 0)
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        assert st == _abi.VS_OK
        lib.vs_destroy(h)
    else:
        assert st == _abi.VS_ERR_CUDA
        assert lib.vs_last_error()
    assert lib.vs_create(None, 0) == _abi.VS_ERR_INVALID_ARG


def _fake_ctx():
    # the host-only calls check ctx for NULL but never dereference it
    return ctypes.c_void_p(ctypes.addressof(ctypes.c_int(0)))


def _desc(nv=100, nt=150, tw=64, th=32, fmt=_abi.VS_TEX_SH_F16, deg=2, pitch=None):
    d = _abi.vs_shell_desc()
    d.pos, d.uv, d.tris, d.texels = 0x10000, 0x20000, 0x30000, 0x40000   # never dereferenced
    d.num_verts, d.num_tris, d.tex_w, d.tex_h = nv, nt, tw, th
    d.format, d.sh_degree = fmt, deg
    nch = 4 if fmt == _abi.VS_TEX_RGBA_F32 else 1 + 3 * (deg + 1) ** 2
    d.texel_pitch = nch if pitch is None else pitch
    return d


def _load(lib, descs):
    arr = (_abi.vs_shell_desc * len(descs))(*descs)
    out = ctypes.c_void_p()
    st = lib.vs_load_shells(_fake_ctx(), arr, len(descs), ctypes.byref(out))
    return st, out


@pytest.mark.parametrize("bad", [
    dict(nv=2), dict(nt=0), dict(tw=0), dict(fmt=7), dict(deg=4), dict(pitch=27), dict(th=70000),
])
def test_load_shells_rejects_bad_descriptors(lib, bad):
    st, out = _load(lib, [_desc(**bad)])
    assert st == _abi.VS_ERR_INVALID_ARG
    assert not out.value
    assert lib.vs_last_error()


def test_load_shells_rejects_bad_k_and_nulls(lib):
    arr = (_abi.vs_shell_desc * 17)(*[_desc() for _ in range(17)])
    out = ctypes.c_void_p()
    assert lib.vs_load_shells(_fake_ctx(), arr, 0, ctypes.byref(out)) == _abi.VS_ERR_INVALID_ARG
    assert lib.vs_load_shells(_fake_ctx(), arr, 17, ctypes.byref(out)) == _abi.VS_ERR_INVALID_ARG
    assert lib.vs_load_shells(None, arr, 1, ctypes.byref(out)) == _abi.VS_ERR_INVALID_ARG
    d = _desc()
    d.pos = None
    st, _ = _load(lib, [d])
    assert st == _abi.VS_ERR_INVALID_ARG


def _cam(w=800, h=600):
    c = _abi.vs_camera()
    for i, v in enumerate([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 4]):
        c.world_to_cam[i] = v
    c.fx = c.fy = 500.0
    c.cx, c.cy, c.znear = w / 2, h / 2, 0.1
    c.width, c.height = w, h
    return c


def test_workspace_size_covers_the_dominant_terms(lib):
    descs = [_desc(nv=1000 + 10 * i, nt=2000 + 7 * i) for i in range(5)]
    st, obj = _load(lib, descs)
    assert st == 0
    objs = (ctypes.c_void_p * 1)(obj.value)
    cams = (_abi.vs_camera * 1)(_cam())
    size = ctypes.c_size_t()
    assert lib.vs_workspace_size(_fake_ctx(), objs, cams, 1, 0, ctypes.byref(size)) == 0
    # visibility words and snapped vertices
    need = 8 * 5 * 800 * 600 + sum(16 * d.num_verts for d in descs)
    assert need <= size.value <= need + 64 * 1024
    # batch of 3 items ~ three times one item
    objs3 = (ctypes.c_void_p * 3)(obj.value, obj.value, obj.value)
    cams3 = (_abi.vs_camera * 3)(_cam(), _cam(320, 200), _cam(1024, 1024))
    size3 = ctypes.c_size_t()
    assert lib.vs_workspace_size(_fake_ctx(), objs3, cams3, 3, 0, ctypes.byref(size3)) == 0
    assert size3.value > 8 * 5 * (800 * 600 + 320 * 200 + 1024 * 1024)
    lib.vs_free_shells(_fake_ctx(), obj)


def test_loss_flags_are_exclusive(lib):
    st, obj = _load(lib, [_desc()])
    assert st == 0
    objs = (ctypes.c_void_p * 1)(obj.value)
    cams = (_abi.vs_camera * 1)(_cam())
    size = ctypes.c_size_t()
    for fl, want in [(_abi.VS_FLAG_LOSS_L1, 0), (_abi.VS_FLAG_LOSS_L2, 0),
                     (_abi.VS_FLAG_LOSS_L1 | _abi.VS_FLAG_LOSS_L2, _abi.VS_ERR_INVALID_ARG)]:
        assert lib.vs_workspace_size(_fake_ctx(), objs, cams, 1, fl, ctypes.byref(size)) == want
    lib.vs_free_shells(_fake_ctx(), obj)


@pytest.mark.parametrize("w,h,znear", [(0, 10, 0.1), (10, 9000, 0.1), (64, 64, 0.0), (64, 64, -1.0)])
def test_workspace_size_rejects_bad_cameras(lib, w, h, znear):
    st, obj = _load(lib, [_desc()])
    assert st == 0
    c = _cam(w, h)
    c.znear = znear
    objs = (ctypes.c_void_p * 1)(obj.value)
    cams = (_abi.vs_camera * 1)(c)
    size = ctypes.c_size_t()
    assert lib.vs_workspace_size(_fake_ctx(), objs, cams, 1, 0, ctypes.byref(size)) == _abi.VS_ERR_INVALID_ARG
    lib.vs_free_shells(_fake_ctx(), obj)


# ----------------------------------------------------------------------------
# batch tuning: argument checks and the search itself (host logic only)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("fields", [(100, 256, 0), (256, 8192, 0), (16, 256, 0), (256, 256, -1),
                                    (256, 256, 65), (256, 96, 0)])
def test_set_batch_tuning_rejects_bad_values_without_a_context(lib, fields):
    t = _abi.vs_tuning(*fields, 0)
    assert lib.vs_set_batch_tuning(None, 0, 3, ctypes.byref(t)) == _abi.VS_ERR_INVALID_ARG
    msg = lib.vs_last_error().decode()
    assert "ctx" not in msg, msg                # refused for the tuning, not the context
    good = _abi.vs_tuning(512, 128, 2, 0)
    assert lib.vs_set_batch_tuning(None, 0, 3, ctypes.byref(good)) == _abi.VS_ERR_INVALID_ARG
    assert "ctx" in lib.vs_last_error().decode()
    assert lib.vs_set_batch_tuning(None, 0, 17, ctypes.byref(good)) == _abi.VS_ERR_INVALID_ARG
    bad_reserved = _abi.vs_tuning(512, 128, 2, 7)
    assert lib.vs_set_batch_tuning(None, 0, 3, ctypes.byref(bad_reserved)) == _abi.VS_ERR_INVALID_ARG


def _search(lib, cost, start=(256, 256, 0), max_blocks=4):
    from paper_2409_02482_gb300 import tune_search
    calls = []

    def f(t):
        calls.append((t.raster_tris, t.shade_pixels, t.blocks_per_sm))
        return cost(*calls[-1])
    best, n = tune_search(_abi.vs_tuning(*start, 0), max_blocks, f)
    assert n == len(calls)
    assert len(set(calls)) == len(calls)        # no configuration costed twice
    return (best.raster_tris, best.shade_pixels, best.blocks_per_sm), calls


def test_tune_search_finds_separable_minimum(lib):
    import math

    def cost(r, s, b):
        return 10 + (math.log2(r) - 9) ** 2 + 2 * (math.log2(s) - 6) ** 2 + 0.5 * (b - 3) ** 2
    best, calls = _search(lib, cost)
    assert best == (512, 64, 3)
    assert len(calls) <= 3 * (5 + 5 + 4)


def test_tune_search_follows_coupled_valley(lib):
    # the best shade size depends on the block count: a second sweep is needed
    def cost(r, s, b):
        want_s = {1: 1024, 2: 512, 3: 256, 4: 128}[b]
        return 5 + abs(s - want_s) / 256 + 3 * abs(b - 4) + (0 if r == 128 else 1)
    best, calls = _search(lib, cost, start=(256, 1024, 1))
    assert best == (128, 128, 4)


def test_tune_search_ignores_gains_below_one_percent(lib):
    # every move gains 0.5%: noise-level differences keep the start
    def cost(r, s, b):
        return 100.0 * (1 - 0.005 * (r != 256)) * (1 - 0.005 * (s != 256))
    best, _ = _search(lib, cost, start=(256, 256, 2))
    assert best == (256, 256, 2)


def test_tune_search_stops_on_bad_cost(lib):
    from paper_2409_02482_gb300 import tune_search
    with pytest.raises(_abi.VSError) as e:
        tune_search(_abi.vs_tuning(256, 256, 0, 0), 2, lambda t: float("nan"))
    assert e.value.status == _abi.VS_ERR_INVALID_ARG
    with pytest.raises(_abi.VSError):
        tune_search(_abi.vs_tuning(256, 256, 0, 0), 2,
                           lambda t: -1.0 if t.shade_pixels == 64 else 1.0)
    with pytest.raises(_abi.VSError):
        tune_search(_abi.vs_tuning(256, 256, 0, 0), 0, lambda t: 1.0)


# ----------------------------------------------------------------------------
# the baked byte format (VS_TEX_SH_U8): layout agreement and descriptor checks
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("tw,th,deg,shift", [(2048, 2048, 3, 1), (12, 6, 2, 0), (20, 12, 1, 1), (128, 64, 3, 2),
                                            (5, 3, 0, 3)])
def test_baked_layout_matches_the_generators(lib, tw, th, deg, shift):
    import synth
    from paper_2409_02482_gb300 import baked_layout
    assert baked_layout(tw, th, deg, shift) == synth.baked_layout(tw, th, deg, shift)


@pytest.mark.parametrize("tw,th,deg,shift", [(12, 8, 3, 1), (16, 16, 4, 0), (16, 16, 1, 4), (0, 16, 0, 0)])
def test_baked_layout_rejects_bad_sizes(lib, tw, th, deg, shift):
    total = ctypes.c_int64()
    assert lib.vs_baked_layout(tw, th, deg, shift, None, None, None, None, ctypes.byref(total)) == \
        _abi.VS_ERR_INVALID_ARG


def _baked_desc(**kw):
    d = _desc(fmt=_abi.VS_TEX_SH_U8, deg=kw.pop("deg", 3), tw=kw.pop("tw", 64), th=kw.pop("th", 32), pitch=0)
    d.band_shift = kw.pop("shift", 1)
    d.value_min, d.value_max = kw.pop("vmin", -15.0), kw.pop("vmax", 15.0)
    if "texels" in kw:
        d.texels = kw.pop("texels")
    assert not kw
    return d


def test_load_shells_accepts_a_baked_shell(lib):
    st, out = _load(lib, [_baked_desc()])
    assert st == _abi.VS_OK
    lib.vs_free_shells(_fake_ctx(), out)


@pytest.mark.parametrize("bad", [dict(shift=4), dict(tw=60), dict(vmin=1.0, vmax=1.0), dict(vmax=float("inf")),
                                 dict(texels=0x40008), dict(deg=4)])
def test_load_shells_rejects_bad_baked_descriptors(lib, bad):
    st, out = _load(lib, [_baked_desc(**bad)])
    assert st == _abi.VS_ERR_INVALID_ARG
    assert not out.value


# ----------------------------------------------------------------------------
# neural texture: layout agreement with the oracle, config checks (host only)
# ----------------------------------------------------------------------------

def _ntex_cfg(**kw):
    d = dict(levels=8, features=2, log2_table=12, base_res=4, growth=1.5, hidden=64, out_ch=28)
    d.update(kw)
    return _abi.vs_ntex_config(d["levels"], d["features"], d["log2_table"], d["base_res"], d["growth"],
                               d["hidden"], d["out_ch"], d.pop("tensor_cores", 0)), d


@pytest.mark.parametrize("kw", [{}, dict(levels=16, log2_table=19, base_res=16), dict(features=4, hidden=8, out_ch=1)])
def test_ntex_layout_matches_the_oracle(lib, kw):
    from oracle import ntex
    c, d = _ntex_cfg(**kw)
    off = (ctypes.c_int64 * 7)()
    total = ctypes.c_int64()
    assert lib.vs_ntex_layout(ctypes.byref(c), off, ctypes.byref(total)) == 0
    lay, tot = ntex.NtexConfig(**d).layout()
    assert list(off) == [o for _, o, _ in lay] and total.value == tot
    nb = ctypes.c_size_t()
    assert lib.vs_ntex_workspace_size(ctypes.byref(c), 2048, 2048, ctypes.byref(nb)) == 0
    assert nb.value >= (1 << 18) * (2 * c.levels * c.features + 4 * c.hidden + 2 * c.out_ch) * 4


@pytest.mark.parametrize("bad", [dict(levels=0), dict(levels=17), dict(features=9), dict(log2_table=25),
                                 dict(base_res=0), dict(growth=0.5), dict(hidden=0), dict(out_ch=300),
                                 dict(levels=16, base_res=1000, growth=4.0), dict(tensor_cores=2)])
def test_ntex_rejects_bad_configs(lib, bad):
    c, _ = _ntex_cfg(**bad)
    total = ctypes.c_int64()
    assert lib.vs_ntex_layout(ctypes.byref(c), None, ctypes.byref(total)) == _abi.VS_ERR_INVALID_ARG
