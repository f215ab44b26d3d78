"""The seeded input generators: determinism, shapes and the structure the
workloads promise (nested closed shells, outward winding, UV range)."""

import numpy as np
import pytest

import synth


def test_generators_are_deterministic():
    a = synth.config_scene("c2", scale=0.001, views=3)
    b = synth.config_scene("c2", scale=0.001, views=3)
    for (sa, ca), (sb, cb) in zip(a, b):
        for x, y in zip(sa.shells, sb.shells):
            assert np.array_equal(x.pos, y.pos) and np.array_equal(x.tex, y.tex)
        for x, y in zip(ca, cb):
            assert np.array_equal(x.world_to_cam, y.world_to_cam)


@pytest.mark.parametrize("n_lat", [4, 9, 32])
def test_latlong_shell_is_closed_and_outward(n_lat):
    pos, uv, tris = synth.displaced_shells(1, n_lat, seed=3)[0]
    assert tris.shape[0] == 4 * n_lat * n_lat - 4 * n_lat
    p = pos.astype(np.float64)
    a, b, c = p[tris[:, 0]], p[tris[:, 1]], p[tris[:, 2]]
    n = np.cross(b - a, c - a)
    assert np.all(np.einsum("ij,ij->i", n, a + b + c) > 0)
    # closed surface: the signed volume equals the enclosed volume (> 0) and
    # the area-weighted normals cancel
    assert abs(n.sum(0)).max() < 1e-6 * np.abs(n).sum()
    assert np.all((uv >= 0) & (uv <= 1))


def test_shells_are_nested():
    shells = synth.displaced_shells(5, 24, seed=0)
    r = [np.linalg.norm(p, axis=1) for (p, uv, t) in shells]
    for i in range(4):
        assert np.all(r[i] > r[i + 1])


def test_workload_sizes():
    (sc, cams), = synth.config_scene("c1")
    assert sc.k == 3 and sc.num_tris == [1280] * 3
    assert sc.shells[0].tex.shape == (256, 256, 4) and sc.shells[0].tex.dtype == np.float32
    assert cams[0].width == 256 and abs(np.linalg.norm(cams[0].eye()) - 3) < 1e-5
    objs = synth.config_scene("c4", scale=0.001, views=2)
    assert len(objs) == 32
    assert {o[0].k for o in objs} <= {3, 5, 7, 9}
    assert all(o[0].shells[0].tex.shape[2] == synth.sh_channels(1) for o in objs)


def test_sh_texture_statistics():
    rng = np.random.default_rng(0)
    t = synth.sh_texture(64, 64, 2, rng)
    assert t.dtype == np.float16 and t.shape == (64, 64, 28)
    assert abs(t.astype(np.float64).std() - 0.3) < 0.01
