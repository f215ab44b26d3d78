"""FP64 oracle of the neural texture -- TEST INFRASTRUCTURE (see __init__.py).

Sec. 3 "Texturing Meshes" and the supplement's "Neural Textures
Architecture": a texture is a 2D multiresolution hash encoding (the
trainable positional encoding of Mueller et al. 2022) followed by an MLP of
two hidden layers with ReLU and a linear output, evaluated at the texel
centres of the target resolution ("grounded"), so that the baked texture is
the network's prediction there and bilinear sampling in the renderer matches
training.  Plain numpy, FP64, written from the definitions:

  level l resolution   N_l = floor(N_min * b^l)
  position             p = x * N_l,  x = ((i + 1/2) / W, (j + 1/2) / H)
  corners              c = floor(p) + {0, 1}^2,  weight prod_d (1 - |p_d - c_d|)
  index                dense  c_0 + c_1 (N_l + 1)          if (N_l + 1)^2 <= T
                       hashed (c_0 * 1 XOR c_1 * 2654435761) mod T  otherwise
  feature              f_l = sum_corners weight * table[l, index]      (F values)
  MLP                  h1 = relu(W0 f + b0), h2 = relu(W1 h1 + b1), y = W2 h2 + b2

Parameters live in one flat vector: table [L, T, F], W0 [H, L F], b0 [H],
W1 [H, H], b1 [H], W2 [C, H], b2 [C].
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

PRIME = 2654435761


@dataclasses.dataclass(frozen=True)
class NtexConfig:
    levels: int = 8
    features: int = 2
    log2_table: int = 12
    base_res: int = 4
    growth: float = 1.5
    hidden: int = 64
    out_ch: int = 28

    @property
    def table_size(self) -> int:
        return 1 << self.log2_table

    def res(self, l: int) -> int:
        return int(math.floor(self.base_res * self.growth ** l))

    def shapes(self):
        L, T, F, H, C = self.levels, self.table_size, self.features, self.hidden, self.out_ch
        return [("table", (L, T, F)), ("W0", (H, L * F)), ("b0", (H,)), ("W1", (H, H)), ("b1", (H,)),
                ("W2", (C, H)), ("b2", (C,))]

    def layout(self):
        """(name, offset, shape) of every parameter block in the flat vector."""
        out, off = [], 0
        for name, shp in self.shapes():
            out.append((name, off, shp))
            off += int(np.prod(shp))
        return out, off


def unpack(cfg: NtexConfig, params: np.ndarray):
    lay, total = cfg.layout()
    assert params.size == total
    return {name: params[off:off + int(np.prod(shp))].reshape(shp) for name, off, shp in lay}


def corners(cfg: NtexConfig, l: int, x: np.ndarray):
    """For points x [N, 2]: table indices [N, 4] and weights [N, 4] of level l."""
    n = cfg.res(l)
    p = x * n
    base = np.floor(p).astype(np.int64)
    fr = p - base
    idx, w = [], []
    dense = (n + 1) ** 2 <= cfg.table_size
    for dy in (0, 1):
        for dx in (0, 1):
            c0, c1 = base[:, 0] + dx, base[:, 1] + dy
            wt = (fr[:, 0] if dx else 1 - fr[:, 0]) * (fr[:, 1] if dy else 1 - fr[:, 1])
            if dense:
                ix = c0 + c1 * (n + 1)
            else:
                ix = ((c0 * 1) ^ (c1 * PRIME)) % cfg.table_size
            idx.append(ix)
            w.append(wt)
    return np.stack(idx, 1), np.stack(w, 1)


def texel_centres(tex_w: int, tex_h: int) -> np.ndarray:
    ys, xs = np.mgrid[0:tex_h, 0:tex_w]
    return np.stack([(xs.reshape(-1) + 0.5) / tex_w, (ys.reshape(-1) + 0.5) / tex_h], 1)


def encode(cfg: NtexConfig, P, x: np.ndarray) -> np.ndarray:
    feats = []
    for l in range(cfg.levels):
        idx, w = corners(cfg, l, x)
        feats.append(np.einsum("nk,nkf->nf", w, P["table"][l][idx]))
    return np.concatenate(feats, 1)


def _mlp(cfg: NtexConfig, P, x: np.ndarray):
    f = encode(cfg, P, x)
    z1 = f @ P["W0"].T + P["b0"]
    h1 = np.maximum(z1, 0)
    z2 = h1 @ P["W1"].T + P["b1"]
    h2 = np.maximum(z2, 0)
    y = h2 @ P["W2"].T + P["b2"]
    return y, dict(x=x, f=f, z1=z1, h1=h1, z2=z2, h2=h2)


def forward(cfg: NtexConfig, params: np.ndarray, tex_w: int, tex_h: int):
    """Texel values [tex_h, tex_w, C] and the activations (for the adjoint)."""
    P = unpack(cfg, params.astype(np.float64))
    y, a = _mlp(cfg, P, texel_centres(tex_w, tex_h))
    return y.reshape(tex_h, tex_w, cfg.out_ch), a


def forward_at(cfg: NtexConfig, params: np.ndarray, tex_w: int, tex_h: int, texels: np.ndarray) -> np.ndarray:
    """The values [n, C] of the texels with row-major indices `texels` only
    (the same definition as forward, for spot checks of large textures)."""
    P = unpack(cfg, params.astype(np.float64))
    return _mlp(cfg, P, texel_centres(tex_w, tex_h)[np.asarray(texels)])[0]


def backward(cfg: NtexConfig, params: np.ndarray, tex_w: int, tex_h: int, grad_y: np.ndarray,
             texels: np.ndarray = None) -> np.ndarray:
    """dL/d(params) (flat, FP64) given dL/d(texel values) [tex_h, tex_w, C];
    with `texels` (row-major indices), grad_y is [n, C] for those texels
    and the rest of the texture has a zero gradient."""
    P = unpack(cfg, params.astype(np.float64))
    if texels is None:
        _, a = forward(cfg, params, tex_w, tex_h)
    else:
        _, a = _mlp(cfg, P, texel_centres(tex_w, tex_h)[np.asarray(texels)])
    g = grad_y.reshape(-1, cfg.out_ch).astype(np.float64)
    G = {name: np.zeros(shp) for name, shp in cfg.shapes()}
    G["W2"] = g.T @ a["h2"]
    G["b2"] = g.sum(0)
    dz2 = (g @ P["W2"]) * (a["z2"] > 0)
    G["W1"] = dz2.T @ a["h1"]
    G["b1"] = dz2.sum(0)
    dz1 = (dz2 @ P["W1"]) * (a["z1"] > 0)
    G["W0"] = dz1.T @ a["f"]
    G["b0"] = dz1.sum(0)
    df = dz1 @ P["W0"]
    F = cfg.features
    for l in range(cfg.levels):
        idx, w = corners(cfg, l, a["x"])
        for k in range(4):
            np.add.at(G["table"][l], idx[:, k], w[:, k:k + 1] * df[:, l * F:(l + 1) * F])
    lay, total = cfg.layout()
    out = np.zeros(total)
    for name, off, shp in lay:
        out[off:off + int(np.prod(shp))] = G[name].reshape(-1)
    return out


def adam(params, grads, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.99, eps: float = 1e-15):
    """One Adam step (Kingma & Ba), bias-corrected, in FP64; returns new
    (params, m, v)."""
    m = beta1 * m + (1 - beta1) * grads
    v = beta2 * v + (1 - beta2) * grads * grads
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
