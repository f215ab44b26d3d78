"""Seeded scene generators: shells, UVs, texel arrays, cameras.

Conventions shared by every consumer (they are input formats, not method
arithmetic):

* Shell ``i = 0`` is the outermost; shells are nested (Sec. 3, "Support
  Surfaces as Shells": ordered offsets keep the layers from crossing).
* Triangles are wound counter-clockwise seen from outside (right-hand normal
  points outward).
* ``uv`` lies in [0, 1]^2; texel row 0 sits at v = 0.
* Texel arrays are row-major ``[H, W, pitch]``.  ``RGBA_F32`` holds
  (r, g, b, a).  ``SH_F16`` of degree d holds one alpha logit followed by the
  (d+1)^2 RGB coefficient triples: ``[a, r0, g0, b0, r1, g1, b1, ...]``
  (coefficient-major, channels interleaved, like the paper's baked images in
  which image i stores coefficient i of every channel, Sec. 3 "Baking
  Textures").
* Cameras follow the OpenCV pinhole model: x right, y down, z forward;
  ``world_to_cam`` is the row-major 3x4 matrix [R | t].
"""

from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

FMT_RGBA_F32 = 0
FMT_SH_F16 = 1
FMT_SH_U8 = 2      # baked: RGBA SH bytes, per-band resolutions (see baked_layout)


def sh_channels(degree: int) -> int:
    """Values per texel of an SH_F16 texture: one alpha logit + 3 (d+1)^2."""
    return 1 + 3 * (degree + 1) ** 2


@dataclasses.dataclass
class Shell:
    pos: np.ndarray      # float32 [V, 3]
    uv: np.ndarray       # float32 [V, 2]
    tris: np.ndarray     # int32 [T, 3]
    tex: np.ndarray      # float32/float16 [Ht, Wt, pitch]; FMT_SH_U8: uint8 band buffer
    fmt: int             # FMT_RGBA_F32, FMT_SH_F16 or FMT_SH_U8
    degree: int = 0      # SH degree (SH formats)
    # FMT_SH_U8 only: band-0 size, resolution shift per band, decode range
    tex_w: int = 0
    tex_h: int = 0
    band_shift: int = 0
    vmin: float = -15.0
    vmax: float = 15.0

    @property
    def channels(self) -> int:
        if self.fmt == FMT_SH_U8:
            return 4 * (self.degree + 1) ** 2
        return 4 if self.fmt == FMT_RGBA_F32 else sh_channels(self.degree)

    @property
    def pitch(self) -> int:
        return 0 if self.fmt == FMT_SH_U8 else int(self.tex.shape[2])

    @property
    def width(self) -> int:
        return self.tex_w if self.fmt == FMT_SH_U8 else int(self.tex.shape[1])

    @property
    def height(self) -> int:
        return self.tex_h if self.fmt == FMT_SH_U8 else int(self.tex.shape[0])


@dataclasses.dataclass
class Scene:
    shells: List[Shell]

    @property
    def k(self) -> int:
        return len(self.shells)

    @property
    def num_tris(self) -> List[int]:
        return [int(s.tris.shape[0]) for s in self.shells]


@dataclasses.dataclass
class Camera:
    world_to_cam: np.ndarray  # float32 [3, 4]
    fx: float
    fy: float
    cx: float
    cy: float
    znear: float
    width: int
    height: int

    def eye(self) -> np.ndarray:
        r = self.world_to_cam[:, :3].astype(np.float64)
        t = self.world_to_cam[:, 3].astype(np.float64)
        return -r.T @ t


# ----------------------------------------------------------------------------
# geometry
# ----------------------------------------------------------------------------

def _orient_outward(pos: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """Flip triangles whose right-hand normal points toward the origin."""
    p = pos.astype(np.float64)
    a, b, c = p[tris[:, 0]], p[tris[:, 1]], p[tris[:, 2]]
    n = np.cross(b - a, c - a)
    inward = np.einsum("ij,ij->i", n, (a + b + c) / 3.0) < 0
    out = tris.copy()
    out[inward, 1], out[inward, 2] = tris[inward, 2], tris[inward, 1]
    return out


def _spherical_uv(dirs: np.ndarray) -> np.ndarray:
    """u = azimuth / 2 pi, v = polar angle from +z / pi."""
    x, y, z = dirs[:, 0], dirs[:, 1], dirs[:, 2]
    u = (np.arctan2(y, x) / (2 * math.pi)) % 1.0
    v = np.arccos(np.clip(z, -1.0, 1.0)) / math.pi
    return np.stack([u, v], axis=1)


def icosphere(subdiv: int, radius: float = 1.0):
    """Subdivided icosahedron on a sphere (20 * 4^subdiv faces).

    UVs are the spherical (azimuth, polar) angles of each vertex; triangles
    that straddle the azimuth seam keep the wrapped values, which only makes
    their texture mapping stretched, never invalid.
    Returns (pos float32 [V,3], uv float32 [V,2], tris int32 [T,3]).
    """
    t = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
             (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    v = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in verts]
    f = list(faces)
    for _ in range(subdiv):
        mid = {}

        def midpoint(i, j):
            key = (min(i, j), max(i, j))
            if key not in mid:
                m = v[i] + v[j]
                v.append(m / np.linalg.norm(m))
                mid[key] = len(v) - 1
            return mid[key]

        nf = []
        for (a, b, c) in f:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = nf
    dirs = np.array(v)
    tris = _orient_outward(dirs, np.array(f, dtype=np.int32))
    pos = (dirs * radius).astype(np.float32)
    uv = _spherical_uv(dirs).astype(np.float32)
    return pos, uv, tris.astype(np.int32)


def _latlong_topology(n_lat: int):
    """Vertex directions, UVs and CCW-outward triangles of a lat-long sphere.

    Rows 1..n_lat-1 carry 2*n_lat+1 vertices (the last duplicates the first
    with u = 1, the UV seam).  Each pole fan triangle has its own pole vertex
    so its UV can sit at the middle of its column.  T = 4 n_lat^2 - 4 n_lat.
    """
    n_lon = 2 * n_lat
    theta = np.pi * np.arange(1, n_lat) / n_lat                 # polar angle
    phi = 2 * np.pi * np.arange(n_lon + 1) / n_lon              # azimuth
    th, ph = np.meshgrid(theta, phi, indexing="ij")
    ring_dirs = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph),
                          np.cos(th)], axis=-1).reshape(-1, 3)
    ring_uv = np.stack([ph / (2 * np.pi), th / np.pi], axis=-1).reshape(-1, 2)
    n_ring = ring_dirs.shape[0]
    cols = np.arange(n_lon)
    pole_u = (cols + 0.5) / n_lon
    north = np.tile([0.0, 0.0, 1.0], (n_lon, 1))
    south = np.tile([0.0, 0.0, -1.0], (n_lon, 1))
    north_uv = np.stack([pole_u, np.zeros(n_lon)], axis=1)
    south_uv = np.stack([pole_u, np.ones(n_lon)], axis=1)
    dirs = np.concatenate([ring_dirs, north, south])
    uv = np.concatenate([ring_uv, north_uv, south_uv])

    def rid(i, j):  # ring i (0-based over theta rows), column j
        return i * (n_lon + 1) + j

    tris = []
    n_rows = n_lat - 1
    i = np.arange(n_rows - 1)[:, None]
    j = cols[None, :]
    a, b = rid(i, j), rid(i, j + 1)
    c, d = rid(i + 1, j), rid(i + 1, j + 1)
    # (a, c, b) and (b, c, d): south x east = outward
    quads = np.stack([np.stack([a, c, b], -1), np.stack([b, c, d], -1)], axis=2)
    tris.append(quads.reshape(-1, 3))
    nid = n_ring + cols
    sid = n_ring + n_lon + cols
    tris.append(np.stack([nid, rid(0, cols), rid(0, cols + 1)], -1))
    last = n_rows - 1
    tris.append(np.stack([rid(last, cols), sid, rid(last, cols + 1)], -1))
    tris = np.concatenate(tris).astype(np.int32)
    return dirs, uv, tris


def latlong_shell(n_lat: int, radius_fn) -> tuple:
    """Star-shaped closed shell r(dir) on a lat-long grid."""
    dirs, uv, tris = _latlong_topology(n_lat)
    r = radius_fn(dirs)
    pos = (dirs * r[:, None]).astype(np.float32)
    return pos, uv.astype(np.float32), tris


class SmoothNoise:
    """Seeded smooth function on the unit sphere with max |n| = 1.

    A sum of randomly oriented low-frequency plane waves restricted to the
    sphere: n(d) = sum_j a_j cos(w_j <u_j, d> + p_j), normalised on a dense
    Fibonacci sample.  It gives the base shape folds and bumps like the
    paper's captured objects without any trained asset.
    """

    def __init__(self, seed: int, terms: int = 24, max_freq: float = 4.0):
        rng = np.random.default_rng(seed)
        u = rng.normal(size=(terms, 3))
        self.u = u / np.linalg.norm(u, axis=1, keepdims=True)
        self.w = rng.uniform(1.0, max_freq, size=terms)
        self.p = rng.uniform(0, 2 * np.pi, size=terms)
        self.a = rng.normal(size=terms) / np.sqrt(self.w)
        self.scale = 1.0
        probe = _fibonacci_dirs(20000)
        self.scale = 1.0 / np.abs(self(probe)).max()

    def __call__(self, dirs: np.ndarray) -> np.ndarray:
        ph = dirs @ self.u.T * self.w[None, :] + self.p[None, :]
        return (np.cos(ph) @ self.a) * self.scale


def _fibonacci_dirs(n: int) -> np.ndarray:
    i = np.arange(n) + 0.5
    z = 1 - 2 * i / n
    r = np.sqrt(1 - z * z)
    ga = np.pi * (3 - np.sqrt(5))
    return np.stack([r * np.cos(ga * i), r * np.sin(ga * i), z], axis=1)


def displaced_shells(k: int, n_lat, seed: int = 0, amp: float = 0.1,
                     spacing: float = 0.02):
    """k nested shells R(dir) - spacing * i of one noise-displaced sphere.

    ``n_lat`` is an int or a per-shell sequence (lat-long rows).  The radial
    offsets mirror the paper's cumulative, ordered offsets that keep layers
    from crossing.  Returns a list of (pos, uv, tris).
    """
    noise = SmoothNoise(seed)
    if isinstance(n_lat, (int, np.integer)):
        n_lat = [int(n_lat)] * k
    out = []
    for i in range(k):
        out.append(latlong_shell(n_lat[i],
                                 lambda d, i=i: 1.0 + amp * noise(d) - spacing * i))
    return out


def concentric_icospheres(radii: Sequence[float], subdiv: int = 3):
    return [icosphere(subdiv, r) for r in radii]


# ----------------------------------------------------------------------------
# textures
# ----------------------------------------------------------------------------

def rgba_texture(h: int, w: int, rng: np.random.Generator,
                 alpha_range=(0.2, 0.8)) -> np.ndarray:
    """RGBA_F32 texels: RGB ~ U[0,1], alpha ~ U[alpha_range]."""
    tex = np.empty((h, w, 4), dtype=np.float32)
    tex[..., :3] = rng.random((h, w, 3), dtype=np.float32)
    lo, hi = alpha_range
    tex[..., 3] = lo + (hi - lo) * rng.random((h, w), dtype=np.float32)
    return tex


def sh_texture(h: int, w: int, degree: int, rng: np.random.Generator,
               sigma: float = 0.3, pitch: Optional[int] = None) -> np.ndarray:
    """SH_F16 texels, every value ~ N(0, sigma) stored as float16.

    Padding channels (pitch > channels) are zero.
    """
    c = sh_channels(degree)
    pitch = c if pitch is None else pitch
    tex = np.zeros((h, w, pitch), dtype=np.float16)
    # blocks of rows, each from its own generator seeded by `rng`, filled by
    # a thread pool (numpy releases the GIL): large textures (4096^2 x 49)
    # generate in seconds, deterministically for a given rng state
    rows = 128
    seeds = rng.integers(0, 2 ** 63 - 1, size=(h + rows - 1) // rows)

    def fill(b):
        r0, r1 = b * rows, min(h, (b + 1) * rows)
        vals = np.random.default_rng(int(seeds[b])).standard_normal((r1 - r0, w, c), dtype=np.float32)
        vals *= np.float32(sigma)
        tex[r0:r1, :, :c] = vals

    if len(seeds) == 1:
        fill(0)
    else:
        from concurrent.futures import ThreadPoolExecutor
        import os
        with ThreadPoolExecutor(min(len(seeds), os.cpu_count() or 1)) as ex:
            list(ex.map(fill, range(len(seeds))))
    return tex


BAKED_STRIDES = (4, 16, 32, 32)   # bytes per texel of band l: 4 (2l + 1), padded


def baked_layout(tex_w: int, tex_h: int, degree: int, band_shift: int):
    """Byte layout of a FMT_SH_U8 buffer: per band l, (offset, w, h, stride)
    with (w, h) = (tex_w, tex_h) >> l * band_shift and each band starting on
    a 256-byte boundary; returns (bands, total bytes)."""
    bands, off = [], 0
    for band in range(degree + 1):
        w, h = tex_w >> (band * band_shift), tex_h >> (band * band_shift)
        bands.append((off, w, h, BAKED_STRIDES[band]))
        off += -(-w * h * BAKED_STRIDES[band] // 256) * 256
    return bands, off


def baked_values_to_bytes(values: np.ndarray, vmin: float, vmax: float) -> np.ndarray:
    """Quantise decoded SH values to the stored bytes: q = round(255 (x -
    vmin) / (vmax - vmin)), clipped to [0, 255] (the inverse of the decode)."""
    q = np.rint((values.astype(np.float64) - vmin) * (255.0 / (vmax - vmin)))
    return np.clip(q, 0, 255).astype(np.uint8)


def baked_sh_texture(tex_w: int, tex_h: int, degree: int, band_shift: int, rng: np.random.Generator,
                     vmin: float = -15.0, vmax: float = 15.0, base_sigma: float = 3.5) -> np.ndarray:
    """FMT_SH_U8 buffer of random baked texels.  Decoded values before
    quantisation: band 0 ~ N(0, base_sigma) for all of RGBA (so that
    sigmoid(value * Y_0) spans (0, 1)), band l >= 1 ~ N(0, base_sigma / (2 l))
    (weaker view dependence in higher bands).  Padding bytes are zero."""
    bands, total = baked_layout(tex_w, tex_h, degree, band_shift)
    buf = np.zeros(total, np.uint8)
    for band, (off, w, h, stride) in enumerate(bands):
        n = 4 * (2 * band + 1)
        sigma = base_sigma if band == 0 else base_sigma / (2 * band)
        # the quantisation of baked_values_to_bytes, in place in FP32 (random
        # values: the rounding of the scale does not matter)
        vals = rng.standard_normal((h, w, n), dtype=np.float32)
        k = np.float32(255.0 / (vmax - vmin))
        vals *= np.float32(sigma) * k
        vals += np.float32(-vmin) * k
        np.rint(vals, out=vals)
        np.clip(vals, 0, 255, out=vals)
        img = np.zeros((h, w, stride), np.uint8)
        img[..., :n] = vals
        buf[off:off + w * h * stride] = img.reshape(-1)
    return buf


def ntex_init(shapes, rng: np.random.Generator) -> np.ndarray:
    """Initial neural-texture parameters (float32, flat in the order of
    `shapes` = [(name, shape), ...]): hash tables U(-1e-4, 1e-4) (the hash
    encoding's usual start), weights N(0, 2 / fan_in) (for ReLU layers),
    biases 0."""
    out = []
    for name, shp in shapes:
        n = int(np.prod(shp))
        if name == "table":
            out.append(rng.uniform(-1e-4, 1e-4, n))
        elif name.startswith("W"):
            out.append(rng.normal(0.0, math.sqrt(2.0 / shp[-1]), n))
        else:
            out.append(np.zeros(n))
    return np.concatenate(out).astype(np.float32)


# ----------------------------------------------------------------------------
# cameras
# ----------------------------------------------------------------------------

def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0), width=256,
            height=256, fov_y_deg=40.0, znear=0.1) -> Camera:
    """OpenCV pinhole camera at ``eye`` looking at ``target``."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    right = np.cross(f, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    r = np.stack([right, down, f])
    t = -r @ eye
    m = np.concatenate([r, t[:, None]], axis=1).astype(np.float32)
    focal = (height / 2.0) / math.tan(math.radians(fov_y_deg) / 2.0)
    return Camera(world_to_cam=m, fx=float(np.float32(focal)),
                  fy=float(np.float32(focal)), cx=width / 2.0, cy=height / 2.0,
                  znear=float(np.float32(znear)), width=int(width),
                  height=int(height))


def fibonacci_cameras(n: int, dist: float, width: int, height: int,
                      elev_range=(5.0, 80.0), seed: int = 0,
                      fov_y_deg: float = 40.0) -> List[Camera]:
    """n views on a Fibonacci lattice of the band elev_range (degrees),
    looking at the origin, world up +z; the lattice is rotated by a seeded
    azimuth."""
    rng = np.random.default_rng(seed)
    rot = rng.uniform(0, 2 * np.pi)
    lo, hi = np.radians(elev_range[0]), np.radians(elev_range[1])
    z = np.sin(lo) + (np.sin(hi) - np.sin(lo)) * (np.arange(n) + 0.5) / n
    ga = np.pi * (3 - np.sqrt(5))
    az = rot + ga * np.arange(n)
    rxy = np.sqrt(1 - z * z)
    eyes = dist * np.stack([rxy * np.cos(az), rxy * np.sin(az), z], axis=1)
    return [look_at(e, width=width, height=height, fov_y_deg=fov_y_deg)
            for e in eyes]


# ----------------------------------------------------------------------------
# the five workloads (and scaled-down variants of them for tests)
# ----------------------------------------------------------------------------

def _n_lat_for_tris(t: float) -> int:
    return max(4, int(round(math.sqrt(t / 4.0))))


CONFIGS = {
    # name: description of the full-size workload
    "c1": "k=3 icospheres (subdiv 3) r=1.0/0.9/0.8, 256^2 RGBA_F32, 1 view 256^2 at d=3",
    "c2": "k=7 displaced shells ~200k tris, 2048^2 SH2 FP16, 100 views 800^2, hemisphere d=4",
    "c3": "k=9 displaced shells ~500k tris, 2048^2 SH2 FP16, 64 views 1024^2, hemisphere d=4, L2 fit",
    "c4": "32 objects, k in {3,5,7,9}, tris/shell log-uniform 10k-1M, 8 views each at "
          "512^2/800^2/1024^2/1920x1080, 1024^2 SH1 FP16, fwd+bwd",
    "c5": "k=9 shells ~2M tris, 4096^2 SH3 FP16, 256 views 3840x2160 on a sphere at d=3.5",
}


def _sh_scene(k, n_lat, tex_res, degree, seed, tex_seed, pitch=None, sigma=0.3, textures=True):
    geo = displaced_shells(k, n_lat, seed=seed)
    ss = np.random.SeedSequence(tex_seed).spawn(k)
    shells = []
    for i, (pos, uv, tris) in enumerate(geo):
        if textures:
            rng = np.random.default_rng(ss[i])
            tex = sh_texture(tex_res, tex_res, degree, rng, sigma=sigma, pitch=pitch)
        else:   # shape only (zero-strided): the caller makes the values
            c = sh_channels(degree)
            tex = np.broadcast_to(np.float16(0), (tex_res, tex_res, c if pitch is None else pitch))
        shells.append(Shell(pos, uv, tris, tex, FMT_SH_F16, degree))
    return Scene(shells)


def _baked_scene(k, n_lat, tex_res, degree, band_shift, seed, tex_seed):
    geo = displaced_shells(k, n_lat, seed=seed)
    ss = np.random.SeedSequence(tex_seed).spawn(k)
    shells = []
    for i, (pos, uv, tris) in enumerate(geo):
        buf = baked_sh_texture(tex_res, tex_res, degree, band_shift, np.random.default_rng(ss[i]))
        shells.append(Shell(pos, uv, tris, buf, FMT_SH_U8, degree, tex_w=tex_res, tex_h=tex_res,
                            band_shift=band_shift))
    return Scene(shells)


def config_scene(name: str, scale: float = 1.0, views: Optional[int] = None,
                 tex_seed: int = 0, pitch: Optional[int] = None, textures: bool = True):
    """Build workload ``name`` ('c1'..'c5', or 'c2b': the C2 geometry and
    views with the paper's deployed textures -- RGBA SH degree 3 in bytes,
    2048^2 base halving per band down to 256^2).

    ``scale`` < 1 shrinks triangle counts (by scale), texture side and image
    side (by sqrt(scale)) for fast tests while keeping the structure.
    Returns (list of (Scene, [Camera])) -- one entry per object.
    """
    s = math.sqrt(scale)

    def res(x):
        return max(16, int(round(x * s / 8)) * 8)

    def texres(x):
        return max(8, 1 << int(round(math.log2(max(8, x * s)))))

    if name == "c1":
        rng = np.random.default_rng(tex_seed)
        shells = []
        for r in (1.0, 0.9, 0.8):
            pos, uv, tris = icosphere(3, r)
            shells.append(Shell(pos, uv, tris, rgba_texture(texres(256), texres(256), rng),
                                FMT_RGBA_F32))
        w = res(256)
        cam = look_at(_eye(3.0, 20.0, 30.0), width=w, height=w)
        return [(Scene(shells), [cam])]
    if name == "c2":
        n = 100 if views is None else views
        sc = _sh_scene(7, _n_lat_for_tris(200e3 * scale), texres(2048), 2, 0, tex_seed, pitch, textures=textures)
        w = res(800)
        return [(sc, fibonacci_cameras(n, 4.0, w, w))]
    if name == "c2b":
        n = 100 if views is None else views
        sc = _baked_scene(7, _n_lat_for_tris(200e3 * scale), texres(2048), 3, 1, 0, tex_seed)
        w = res(800)
        return [(sc, fibonacci_cameras(n, 4.0, w, w))]
    if name == "c3":
        n = 64 if views is None else views
        sc = _sh_scene(9, _n_lat_for_tris(500e3 * scale), texres(2048), 2, 0, tex_seed, pitch, textures=textures)
        w = res(1024)
        return [(sc, fibonacci_cameras(n, 4.0, w, w))]
    if name == "c4":
        n_obj = 32
        n_views = 8 if views is None else views
        rng = np.random.default_rng(4)
        resolutions = [(512, 512), (800, 800), (1024, 1024), (1920, 1080)]
        out = []
        for o in range(n_obj):
            k = int(rng.choice([3, 5, 7, 9]))
            tris = np.exp(rng.uniform(np.log(10e3), np.log(1e6), size=k)) * scale
            n_lat = [_n_lat_for_tris(t) for t in tris]
            sc = _sh_scene(k, n_lat, texres(1024), 1, 100 + o, 1000 * (tex_seed + 1) + o, pitch,
                           textures=textures)
            cams = []
            for vi in range(n_views):
                wv, hv = resolutions[int(rng.integers(len(resolutions)))]
                cams += fibonacci_cameras(1, 4.0, res(wv), res(hv), seed=1000 * o + vi)
            out.append((sc, cams))
        return out
    if name == "c5":
        n = 256 if views is None else views
        sc = _sh_scene(9, _n_lat_for_tris(2e6 * scale), texres(4096), 3, 0, tex_seed, pitch, textures=textures)
        return [(sc, fibonacci_cameras(n, 3.5, res(3840), res(2160),
                                       elev_range=(-80.0, 80.0)))]
    raise KeyError(name)


def _eye(dist, elev_deg, azim_deg):
    e, a = math.radians(elev_deg), math.radians(azim_deg)
    return (dist * math.cos(e) * math.cos(a), dist * math.cos(e) * math.sin(a),
            dist * math.sin(e))
