"""Host logic of bench.py (no GPU): the clock summary that decides whether a
run counts, the algorithmic byte accounting of the roofline, and the rule
that a stored ncu traffic figure is used only for the sources it was taken
on."""

import json
import os
import shutil

import numpy as np
import pytest

import bench
import synth


def _row(sm, mx, pw, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return ["2026/01/01 00:00:00.000", "0", str(sm), str(mx), str(pw), "0x0", hw, hwt, swt, cap]


def test_clock_summary_median_and_reasons():
    rows = [_row(2070, 2070, 800.5), _row(2055, 2070, 900.25), _row(1980, 2070, 910.0, cap="Active")]
    s = bench.ClockSampler.summarize(rows)
    assert s["sm_mhz"] == 2055 and s["sm_max_mhz"] == 2070 and s["power_w_max"] == 910.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3
    s = bench.ClockSampler.summarize(rows + [_row(1200, 2070, 700, hw="Active", swt="Active")])
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert bench.ClockSampler.summarize([])["reasons"] == ["no samples"]


def test_algorithmic_bytes_count_real_channels_not_padding():
    (scene, cams), = synth.config_scene("c2", scale=0.002, views=2, pitch=32)
    wl = dict(scene=scene, cams=cams, H=cams[0].height, W=cams[0].width)
    frags, d = 1000, 3.25
    total, parts = bench.algorithmic_bytes(wl, frags, d, with_bwd=True)
    D = d * frags * 2
    assert parts["texels"] == pytest.approx(D * 28 * 2)          # 28 FP16 values, not the pitch of 32
    assert parts["grads"] == pytest.approx(D * 28 * 8)           # FP32 read + write of each value
    geo = 2 * sum(20 * s.pos.shape[0] + 12 * s.tris.shape[0] for s in scene.shells)
    assert parts["geometry"] == geo
    assert parts["image"] == 2 * wl["H"] * wl["W"] * (16 + 12)
    assert total == pytest.approx(sum(parts.values()))
    fwd, fparts = bench.algorithmic_bytes(wl, frags, d, with_bwd=False)
    assert fparts["grads"] == 0 and fparts["image"] == 2 * wl["H"] * wl["W"] * 16


def test_step_lower_bound_moves_each_touched_texel_once():
    (scene, cams), = synth.config_scene("c2", scale=0.002, views=3, pitch=32)
    wl = dict(scene=scene, cams=cams, H=cams[0].height, W=cams[0].width)
    touched = 12345
    b = bench.step_lower_bound_bytes(wl, touched)
    geo = sum(20 * s.pos.shape[0] + 12 * s.tris.shape[0] for s in scene.shells)   # once per step
    assert b == pytest.approx(touched * (28 * 2 + 28 * 8) + geo + 3 * wl["H"] * wl["W"] * 28)
    # never above the per-view bytes when every view touches every texel it counts
    per_view, _ = bench.algorithmic_bytes(wl, touched / 3.0, 1.0, with_bwd=True)
    assert b <= per_view


def test_stored_traffic_only_for_the_captured_sources(monkeypatch):
    with open(os.path.join(bench.ROOT, "profiles", "k_persistent_fwdbwd_c2_traffic.json")) as f:
        d = json.load(f)
    per_view = (d["dram_bytes_read"] + d["dram_bytes_write"]) / d["views"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: d["kernel_source_sha256"])
    value, note = bench.stored_traffic(100)
    assert value == pytest.approx(100 * per_view) and "scaled" in note
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 64)
    assert bench.stored_traffic(100)[0] is None


def test_source_hash_covers_the_renderer_only(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_2409_02482_gb300", "csrc")
    dst = tmp_path / "paper_2409_02482_gb300" / "csrc"
    shutil.copytree(src, dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    with open(dst / "vs_ntex.cu", "a") as f:      # the neural texture takes no part in the renderer's launches
        f.write("\n// edit\n")
    assert bench.kernel_source_hash() == h0
    with open(dst / "vs_kernels.cuh", "a") as f:
        f.write("\n// edit\n")
    assert bench.kernel_source_hash() != h0
