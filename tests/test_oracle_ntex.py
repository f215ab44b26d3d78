"""Pins of the FP64 neural-texture oracle (hash-grid encoding + MLP, Sec. 3
"Texturing Meshes" and the supplement's neural texture architecture)
against independent routes: interpolation identities of the encoding,
central finite differences of the adjoint, and Adam's first-step closed
form.  The spatial hash itself (XOR with the published prime, modulo the
table size) is a definition: these checks pin how it is used -- corner
geometry, weights, dense vs hashed levels -- not its constant."""

import numpy as np
import pytest

import synth
from oracle import ntex


def _params(cfg, seed, scale=0.5):
    rng = np.random.default_rng(seed)
    lay, total = cfg.layout()
    p = np.zeros(total)
    for name, off, shp in lay:
        n = int(np.prod(shp))
        s = scale if name == "table" else (1.0 / np.sqrt(shp[-1]) if name.startswith("W") else 0.1)
        p[off:off + n] = rng.normal(0, s, n)
    return p


def test_layout_is_contiguous_and_complete():
    cfg = ntex.NtexConfig(levels=3, features=2, log2_table=5, hidden=8, out_ch=3)
    lay, total = cfg.layout()
    assert [name for name, _, _ in lay] == ["table", "W0", "b0", "W1", "b1", "W2", "b2"]
    assert total == 3 * 32 * 2 + 8 * 6 + 8 + 64 + 8 + 24 + 3
    ends = [off + int(np.prod(shp)) for _, off, shp in lay]
    assert [off for _, off, _ in lay][1:] == ends[:-1]


def test_encoding_at_grid_vertices_returns_table_entries():
    """A point on a level's grid vertex has weight 1 on that corner."""
    cfg = ntex.NtexConfig(levels=2, features=2, log2_table=6, base_res=4, growth=2.0, hidden=4, out_ch=2)
    P = ntex.unpack(cfg, _params(cfg, 1))
    for l in range(cfg.levels):
        n = cfg.res(l)
        pts = np.array([[i / n, j / n] for i in range(1, n) for j in range(1, n)])
        idx, w = ntex.corners(cfg, l, pts)
        assert np.allclose(w[:, 0], 1.0) and np.allclose(w[:, 1:], 0.0)
        f = ntex.encode(cfg, P, pts)[:, l * 2:(l + 1) * 2]
        assert np.allclose(f, P["table"][l][idx[:, 0]])


def test_dense_levels_reproduce_affine_tables_and_hashed_levels_collide():
    """On a dense level, a table affine in the vertex coordinates gives an
    encoding affine in x (bilinear reproduction, so the lattice is x * N_l);
    a level with more vertices than entries must share entries (hashing)."""
    cfg = ntex.NtexConfig(levels=3, features=1, log2_table=6, base_res=3, growth=2.0, hidden=4, out_ch=2)
    params = np.zeros(cfg.layout()[1])
    P = ntex.unpack(cfg, params)
    n = cfg.res(0)                                   # 3: (3 + 1)^2 = 16 <= 64, dense
    for c1 in range(n + 1):
        for c0 in range(n + 1):
            P["table"][0][c0 + c1 * (n + 1), 0] = 2.0 * c0 - 0.5 * c1 + 1.0
    x = np.random.default_rng(2).uniform(0, 1, (50, 2))
    f = ntex.encode(cfg, P, x)[:, 0]
    assert np.allclose(f, 2.0 * x[:, 0] * n - 0.5 * x[:, 1] * n + 1.0)
    n2 = cfg.res(2)                                  # 12: (12 + 1)^2 = 169 > 64, hashed
    g = np.array([[i / n2 + 1e-9, j / n2 + 1e-9] for i in range(n2 + 1) for j in range(n2 + 1)])
    idx, _ = ntex.corners(cfg, 2, np.clip(g, 0, 1 - 1e-9))
    assert idx.max() < cfg.table_size and len(np.unique(idx[:, 0])) < len(g)


@pytest.mark.parametrize("log2_table", [4, 10])
def test_backward_matches_central_differences(log2_table):
    cfg = ntex.NtexConfig(levels=3, features=2, log2_table=log2_table, base_res=2, growth=1.8, hidden=8, out_ch=3)
    params = _params(cfg, 3)
    W, H = 6, 5
    g = np.random.default_rng(4).normal(size=(H, W, cfg.out_ch))
    grads = ntex.backward(cfg, params, W, H, g)

    def loss(p):
        return float((ntex.forward(cfg, p, W, H)[0] * g).sum())
    h = 1e-6
    rng = np.random.default_rng(5)
    lay, total = cfg.layout()
    checked = 0
    for name, off, shp in lay:
        n = int(np.prod(shp))
        for k in rng.choice(n, min(n, 12), replace=False):
            e = np.zeros(total)
            e[off + k] = h
            fd = (loss(params + e) - loss(params - e)) / (2 * h)
            assert abs(fd - grads[off + k]) < 1e-6 * max(1.0, abs(fd)), (name, k)
            checked += 1
    assert checked > 50 and np.abs(grads).max() > 1e-3


def test_adam_first_step_closed_form():
    """Step 1 with bias correction: m^ = g, v^ = g^2, so the update is
    -lr g / (|g| + eps) -- a unit step against the gradient's sign."""
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    p = np.array([1.0, 2.0, 3.0, 4.0])
    z = np.zeros(4)
    p1, m, v = ntex.adam(p, g, z, z, 1, lr=0.01, eps=1e-15)
    assert np.allclose(p1, p - 0.01 * np.sign(g))
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.01 * g * g)


def test_sampled_texels_equal_the_full_texture():
    """forward_at / backward(texels=...) evaluate the same definition on a
    subset of texels: the subset of the full forward, and the full adjoint
    of a gradient that is zero outside the subset."""
    cfg = ntex.NtexConfig(levels=4, features=2, log2_table=8, base_res=3, growth=1.7, hidden=8, out_ch=5)
    params = synth.ntex_init(cfg.shapes(), np.random.default_rng(3)).astype(np.float64)
    W, H = 13, 11
    idx = np.array([0, 5, 17, 60, 142])
    full, _ = ntex.forward(cfg, params, W, H)
    assert np.array_equal(ntex.forward_at(cfg, params, W, H, idx), full.reshape(-1, cfg.out_ch)[idx])
    g = np.random.default_rng(4).normal(size=(len(idx), cfg.out_ch))
    dense = np.zeros((H * W, cfg.out_ch))
    dense[idx] = g
    a = ntex.backward(cfg, params, W, H, dense.reshape(H, W, cfg.out_ch))
    b = ntex.backward(cfg, params, W, H, g, texels=idx)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-15)
