"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these recompute the oracle's own formulas: each compares it with an
independent route (ray casting, a library routine, a closed form, brute
force, finite differences) chosen so that a plausible slip -- a dropped term,
a wrong sign or index, a transposed operand -- fails at least one of them.
The paper prints no worked numeric example, so there is no table to copy.
"""

import math

import numpy as np
import pytest

import oracle
import synth
from synth import FMT_RGBA_F32, FMT_SH_F16, FMT_SH_U8, Camera, Scene, Shell


# ----------------------------------------------------------------------------
# independent helpers (FP64, numpy) -- no oracle code
# ----------------------------------------------------------------------------

def pixel_rays(cam):
    """Camera centre and unit world ray directions through pixel centres."""
    R = cam.world_to_cam[:, :3].astype(np.float64)
    t = cam.world_to_cam[:, 3].astype(np.float64)
    eye = -R.T @ t
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    dc = np.stack([(xs + 0.5 - cam.cx) / cam.fx, (ys + 0.5 - cam.cy) / cam.fy,
                   np.ones(xs.shape)], axis=-1)
    dw = dc @ R
    dw /= np.linalg.norm(dw, axis=-1, keepdims=True)
    return eye, dw


def raycast_front(eye, dirs, pos, tris):
    """Nearest front-facing hit per ray (Moller-Trumbore, FP64).

    Returns (tri id or -1, t, second-nearest t) per ray."""
    p = pos.astype(np.float64)
    a, b, c = p[tris[:, 0]], p[tris[:, 1]], p[tris[:, 2]]
    e1, e2 = b - a, c - a
    n = np.cross(e1, e2)
    tvec = eye[None, :] - a
    qvec = np.cross(tvec, e1)
    tt_num = np.einsum("ij,ij->i", e2, qvec)
    d = dirs.reshape(-1, 3)
    ids = np.full(d.shape[0], -1)
    t_best = np.full(d.shape[0], np.inf)
    t_second = np.full(d.shape[0], np.inf)
    for s in range(0, d.shape[0], 256):
        dd = d[s:s + 256]
        pvec = np.cross(dd[:, None, :], e2[None, :, :])
        det = np.einsum("tj,dtj->dt", e1, pvec)
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / det
            u = np.einsum("tj,dtj->dt", tvec, pvec) * inv
            v = (dd @ qvec.T) * inv
            tt = tt_num[None, :] * inv
        front = (dd @ n.T) < 0
        ok = front & (u >= 0) & (v >= 0) & (u + v <= 1) & (tt > 0)
        tm = np.where(ok, tt, np.inf)
        order = np.argsort(tm, axis=1)[:, :2]
        best = tm[np.arange(len(dd)), order[:, 0]]
        ids[s:s + 256] = np.where(np.isfinite(best), order[:, 0], -1)
        t_best[s:s + 256] = best
        t_second[s:s + 256] = tm[np.arange(len(dd)), order[:, 1]]
    return ids, t_best, t_second


def project64(pos, cam):
    R = cam.world_to_cam[:, :3].astype(np.float64)
    t = cam.world_to_cam[:, 3].astype(np.float64)
    pc = pos.astype(np.float64) @ R.T + t
    return np.stack([cam.fx * pc[:, 0] / pc[:, 2] + cam.cx,
                     cam.fy * pc[:, 1] / pc[:, 2] + cam.cy], axis=1), pc[:, 2]


def edge_distance_px(scr, tri, px, py):
    """Distance (pixels) from point to the three edge lines of a projected tri."""
    d = []
    for j in range(3):
        a, b = scr[tri[j]], scr[tri[(j + 1) % 3]]
        ab = b - a
        d.append(abs(ab[0] * (py - a[1]) - ab[1] * (px - a[0])) / max(np.hypot(*ab), 1e-30))
    return min(d)


def real_sh_scipy(degree, v):
    """Real orthonormal SH from scipy's complex Y_l^m: sqrt(2)(-1)^m Re / Im,
    index l^2 + l + m."""
    from scipy.special import sph_harm_y
    v = np.asarray(v, np.float64)
    theta = math.acos(max(-1.0, min(1.0, v[2])))
    phi = math.atan2(v[1], v[0])
    out = []
    for l in range(degree + 1):
        for m in range(-l, l + 1):
            y = sph_harm_y(l, abs(m), theta, phi)
            if m > 0:
                out.append(math.sqrt(2) * (-1) ** m * y.real)
            elif m < 0:
                out.append(math.sqrt(2) * (-1) ** m * y.imag)
            else:
                out.append(y.real)
    return np.array(out)


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def constant_shell(pos, uv, tris, values, fmt=FMT_RGBA_F32, degree=0, size=4, dtype=np.float32):
    tex = np.broadcast_to(np.asarray(values, dtype), (size, size, len(values))).copy()
    return Shell(pos, uv, tris, tex, fmt, degree)


def inradius(pos, tris):
    p = pos.astype(np.float64)
    a, b, c = p[tris[:, 0]], p[tris[:, 1]], p[tris[:, 2]]
    n = np.cross(b - a, c - a)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    return float(np.abs(np.einsum("ij,ij->i", n, a)).min())


def ray_center_distance(cam):
    eye, d = pixel_rays(cam)
    return np.linalg.norm(np.cross(np.broadcast_to(eye, d.shape), d), axis=-1)


# ----------------------------------------------------------------------------
# coverage and depth (Fig. 3c; rasterization of Sec. 3 "Baking Textures")
# ----------------------------------------------------------------------------

def test_raster_brute_force_equals_bbox():
    rng = np.random.default_rng(3)
    # random small mesh with vertices on the half-pixel lattice: edges through
    # pixel centres, shared edges and vertices, mixed orientations
    cam = synth.look_at((0.0, -3.0, 0.4), width=24, height=20)
    pos = rng.normal(size=(30, 3)).astype(np.float32) * 0.5
    tris = rng.integers(0, 30, size=(60, 3)).astype(np.int32)
    k_b, c_b, s_b = oracle.raster(pos, tris, cam, brute=True, coverage=True, threads=1)
    k_x, c_x, s_x = oracle.raster(pos, tris, cam, brute=False, coverage=True, threads=3)
    assert np.array_equal(k_b, k_x)
    assert np.array_equal(c_b, c_x)
    assert (k_x != 0).sum() > 50
    pos2, uv2, tris2 = synth.displaced_shells(1, 8, seed=5, amp=0.3)[0]
    cam2 = synth.look_at((2.5, 1.0, 0.5), width=40, height=32)
    k_b = oracle.raster(pos2, tris2, cam2, brute=True, threads=1)[0]
    k_x = oracle.raster(pos2, tris2, cam2, brute=False, threads=4)[0]
    assert np.array_equal(k_b, k_x)


@pytest.mark.parametrize("eye", [(0.0, -3.0, 0.0), (2.1, 1.3, 1.7), (0.3, 0.2, 3.2)])
def test_watertight_convex_icosphere(eye):
    """Convex closed mesh: each pixel inside the insphere's silhouette is
    covered by exactly one front triangle; none outside the circumsphere's;
    never more than one anywhere (no double cover, no holes)."""
    pos, uv, tris = synth.icosphere(2, 1.0)
    cam = synth.look_at(eye, width=96, height=80)
    _, cover, stats = oracle.raster(pos, tris, cam, coverage=True)
    dist = ray_center_distance(cam)
    margin = 0.05 * np.linalg.norm(eye) / cam.fx
    rin = inradius(pos, tris)
    assert cover.max() <= 1
    assert np.all(cover[dist < rin - margin] == 1)
    assert np.all(cover[dist > 1.0 + margin] == 0)
    assert stats[2] == 0 and stats[3] == 0
    assert stats[0] + stats[1] == tris.shape[0]


def _grid_camera(w, h):
    # identity pose, focal 256 and z = 1: world x = (s - cx)/256 lands
    # exactly on screen coordinate s
    return Camera(world_to_cam=np.concatenate([np.eye(3), np.zeros((3, 1))], 1).astype(np.float32),
                  fx=256.0, fy=256.0, cx=w / 2.0, cy=h / 2.0, znear=0.1, width=w, height=h)


def test_watertight_lattice_triangulation():
    """Delaunay triangulation of points on pixel centres, pixel corners and
    edge midpoints: many edges and vertices pass exactly through pixel
    centres, so only the top-left rule decides; every pixel centre strictly
    inside the hull is covered exactly once."""
    from scipy.spatial import ConvexHull, Delaunay
    w, h = 40, 36
    cam = _grid_camera(w, h)
    rng = np.random.default_rng(7)
    pts = np.unique(rng.integers(4, 2 * min(w, h) - 8, size=(120, 2)) * 0.5, axis=0)
    tri = Delaunay(pts).simplices.astype(np.int32)
    pos = np.stack([(pts[:, 0] - cam.cx) / 256.0, (pts[:, 1] - cam.cy) / 256.0,
                    np.ones(len(pts))], axis=1).astype(np.float32)
    xy, _, _, _ = oracle.setup_vertices(pos, cam)
    assert np.array_equal(xy, np.round(pts * 256).astype(np.int64))   # exact placement
    # make every triangle front-facing (negative signed area in y-down screen space)
    p = pts[tri]
    a2 = (p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - \
         (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1])
    tri[a2 > 0] = tri[a2 > 0][:, [0, 2, 1]]
    _, cover, stats = oracle.raster(pos, tri, cam, coverage=True)
    assert stats[0] == len(tri)
    eq = ConvexHull(pts).equations
    ys, xs = np.mgrid[0:h, 0:w]
    c = np.stack([xs + 0.5, ys + 0.5, np.ones_like(xs, dtype=float)], -1)
    inside = np.all(c @ eq.T < -1e-9, axis=-1)
    assert cover.max() <= 1
    assert np.all(cover[inside] == 1)
    on_vertex = np.isin((xs + 0.5) * 1000 + (ys + 0.5), pts[:, 0] * 1000 + pts[:, 1])
    assert on_vertex[inside].sum() > 5            # the case is exercised


def test_top_left_rule_shared_edges():
    """Two triangles sharing a vertical and a horizontal edge through pixel
    centres: the shared pixels go to the triangle to the right of the
    vertical edge / below the horizontal edge (top-left rule)."""
    w, h = 16, 16
    cam = _grid_camera(w, h)
    # square [4.5, 10.5]^2 split along the vertical x = 7.5 into two rects of
    # two triangles each
    P = {"a": (4.5, 4.5), "b": (7.5, 4.5), "c": (10.5, 4.5),
         "d": (4.5, 10.5), "e": (7.5, 10.5), "f": (10.5, 10.5)}
    names = list(P)
    pts = np.array([P[n] for n in names])
    ix = {n: i for i, n in enumerate(names)}
    tris = np.array([[ix["a"], ix["d"], ix["b"]], [ix["b"], ix["d"], ix["e"]],
                     [ix["b"], ix["e"], ix["c"]], [ix["c"], ix["e"], ix["f"]]], np.int32)
    pos = np.stack([(pts[:, 0] - cam.cx) / 256.0, (pts[:, 1] - cam.cy) / 256.0,
                    np.ones(len(pts))], axis=1).astype(np.float32)
    keys, cover, stats = oracle.raster(pos, tris, cam, coverage=True)
    hits = oracle.hits_from_keys(keys)
    assert stats[0] == 4
    # column x = 7 has centre 7.5 on the shared vertical edge: belongs to the
    # right half (triangles 2, 3); the top row y = 4 (centre 4.5) is a top
    # edge -> covered; the bottom row (centre 10.5) is a bottom edge -> not;
    # left column x = 4 (left edge) covered, right column x = 10 not.
    assert np.all(cover[4:10, 4:10] == 1)
    assert np.all(cover[10, :] == 0) and np.all(cover[:, 10] == 0)
    assert set(np.unique(hits[4:10, 7])) <= {2, 3}
    assert set(np.unique(hits[4:10, 4:7])) <= {0, 1}


def test_projection_matches_fp64_pinhole():
    """Snapped vertices sit within 1/512 px (+ FP32 rounding) of the exact
    FP64 pinhole projection; depth keys follow 2^30 znear / z."""
    pos, _, _ = synth.displaced_shells(1, 12, seed=2)[0]
    for cam in synth.fibonacci_cameras(3, 4.0, 300, 200):
        xy, invw, q, flags = oracle.setup_vertices(pos, cam)
        scr, z = project64(pos, cam)
        assert np.all(flags == 0)
        err = np.abs(xy / 256.0 - scr).max()
        assert err <= 1.0 / 512 + 1e-3
        assert np.allclose(invw, 1.0 / z, rtol=1e-6)
        assert np.allclose(q.astype(np.float64), 2.0 ** 30 * cam.znear / z, rtol=1e-6)


def test_raycast_agrees_except_near_edges():
    """Non-convex, self-occluding shell: the nearest front hit of an FP64 ray
    cast equals the oracle's triangle except where the pixel centre is within
    a hair of a triangle edge (snapping) or two hits tie in depth."""
    # one mesh made of a bumpy shell and a second blob in front of it: front
    # faces overlap on screen, so the nearest-hit rule decides
    p1, _, t1 = synth.displaced_shells(1, 14, seed=11, amp=0.3)[0]
    p2, _, t2 = synth.icosphere(2, 0.35)
    p2 = p2 + np.array([1.2, 0.3, 0.2], np.float32)
    pos = np.concatenate([p1, p2]).astype(np.float32)
    tris = np.concatenate([t1, t2 + len(p1)]).astype(np.int32)
    cam = synth.look_at((3.2, 0.8, 0.35), width=72, height=64)
    keys, cover, _ = oracle.raster(pos, tris, cam, coverage=True)
    hits = oracle.hits_from_keys(keys).reshape(-1)
    assert (cover >= 2).sum() > 10             # overlapping front faces exist
    eye, dirs = pixel_rays(cam)
    ids, t1, t2 = raycast_front(eye, dirs, pos, tris)
    scr, _ = project64(pos, cam)
    bad = 0
    for p in np.nonzero(ids != hits)[0]:
        y, x = divmod(p, cam.width)
        px, py = x + 0.5, y + 0.5
        near_edge = any(edge_distance_px(scr, tris[t], px, py) < 0.01
                        for t in (ids[p], hits[p]) if t >= 0)
        tie = np.isfinite(t2[p]) and abs(t2[p] - t1[p]) < 1e-6 * t1[p]
        if not (near_edge or tie):
            bad += 1
    assert bad == 0
    assert (ids == hits).mean() > 0.99


def test_nested_shells_keep_depth_order():
    """Sec. 3 "Support Surfaces as Shells": nested shells are met in order,
    so per pixel the depth key (larger = nearer) never increases inward."""
    shells = synth.displaced_shells(4, 20, seed=1, amp=0.15)
    cam = synth.look_at((2.0, -2.8, 1.1), width=80, height=80)
    keys = np.stack([oracle.raster(p, t, cam)[0] for (p, uv, t) in shells])
    K = keys >> np.uint64(32)
    both = (keys[:-1] != 0) & (keys[1:] != 0)
    assert both.sum() > 1000
    assert np.all(K[:-1][both] >= K[1:][both])
    # inner shells are covered only where outer ones are
    assert np.all((keys[1:] != 0) <= (keys[:-1] != 0))


# ----------------------------------------------------------------------------
# texture sampling (Fig. 5) and SH decode (Sec. 3 "Texturing Meshes")
# ----------------------------------------------------------------------------

def test_bilinear_at_texel_centres_returns_texel():
    rng = np.random.default_rng(0)
    tex = rng.normal(size=(5, 7, 3))
    for y in range(5):
        for x in range(7):
            out = oracle.sample(tex, (x + 0.5) / 7, (y + 0.5) / 5)
            assert np.array_equal(out, tex[y, x])


def test_bilinear_reproduces_affine_texture():
    H, W = 6, 9
    ys, xs = np.mgrid[0:H, 0:W]
    tex = np.stack([0.3 + 0.7 * xs - 0.2 * ys, -1.0 + 0.05 * xs + 0.9 * ys], -1).astype(np.float64)
    rng = np.random.default_rng(1)
    for _ in range(200):
        X, Y = rng.uniform(0, W - 1), rng.uniform(0, H - 1)
        out = oracle.sample(tex, (X + 0.5) / W, (Y + 0.5) / H)
        assert np.allclose(out, [0.3 + 0.7 * X - 0.2 * Y, -1.0 + 0.05 * X + 0.9 * Y], atol=1e-12)


def test_bilinear_clamps_to_edge():
    rng = np.random.default_rng(2)
    tex = rng.normal(size=(4, 6, 2))
    for v in rng.uniform(0, 1, 20):
        assert np.allclose(oracle.sample(tex, 0.0, v), oracle.sample(tex, 0.5 / 6, v), atol=1e-15)
        assert np.allclose(oracle.sample(tex, 1.0, v), oracle.sample(tex, 5.5 / 6, v), atol=1e-15)
    assert np.allclose(oracle.sample(tex, 0.0, 0.0), tex[0, 0])
    assert np.allclose(oracle.sample(tex, 1.0, 1.0), tex[3, 5])


def test_bilinear_tent_of_single_texel():
    """A single non-zero texel gives the separable tent (1-|dx|)(1-|dy|)."""
    tex = np.zeros((8, 8, 1))
    tex[3, 5, 0] = 1.0
    rng = np.random.default_rng(4)
    for _ in range(100):
        X, Y = rng.uniform(3.2, 6.8), rng.uniform(1.2, 4.8)
        out = oracle.sample(tex, (X + 0.5) / 8, (Y + 0.5) / 8)[0]
        assert abs(out - max(0, 1 - abs(X - 5)) * max(0, 1 - abs(Y - 3))) < 1e-12


def test_half_precision_values_decode_exactly():
    vals = np.array([0.0, -0.0, 1.0, -2.5, 0.1, 65504.0, 2.0 ** -24, 3 * 2.0 ** -24,
                     2.0 ** -14, -0.3333], np.float16)
    tex = vals.reshape(1, 1, -1)
    out = oracle.sample(tex, 0.5, 0.5)
    assert np.array_equal(out, vals.astype(np.float64))


def test_sh_basis_orthonormal_by_quadrature():
    mu, wmu = np.polynomial.legendre.leggauss(16)
    nphi = 16
    phis = 2 * np.pi * np.arange(nphi) / nphi
    G = np.zeros((16, 16))
    for m_, w_ in zip(mu, wmu):
        s = math.sqrt(1 - m_ * m_)
        for ph in phis:
            Y = oracle.sh_basis(3, [s * math.cos(ph), s * math.sin(ph), m_])
            G += w_ * (2 * np.pi / nphi) * np.outer(Y, Y)
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_sh_basis_matches_scipy_real_harmonics():
    rng = np.random.default_rng(5)
    for _ in range(50):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        assert np.allclose(oracle.sh_basis(3, v), real_sh_scipy(3, v), atol=1e-13)
    # l = 1 band is (y, z, x) * sqrt(3 / 4 pi); l = 0 is constant
    v = np.array([0.48, -0.6, 0.64])
    Y = oracle.sh_basis(1, v)
    assert np.allclose(Y[1:4], math.sqrt(3 / (4 * math.pi)) * v[[1, 2, 0]], atol=1e-15)
    assert abs(Y[0] - 0.5 / math.sqrt(math.pi)) < 1e-16


def test_perspective_correct_uv_is_ray_plane_intersection():
    """Barycentrics from snapped screen positions and 1/w reproduce the UV of
    the true ray-plane intersection (Sec. 3 "Texturing Meshes": the sample
    point is the surface point seen through the pixel)."""
    rng = np.random.default_rng(6)
    f, cx, cy = 300.0, 64.0, 48.0
    for _ in range(100):
        while True:
            X = rng.integers(0, 128 * 256, 3)
            Y = rng.integers(0, 96 * 256, 3)
            a2 = (X[1] - X[0]) * (Y[2] - Y[0]) - (X[2] - X[0]) * (Y[1] - Y[0])
            if a2 < -1e6:
                break
        z = rng.uniform(1.0, 9.0, 3)
        uv = rng.uniform(0, 1, (3, 2)).astype(np.float32)
        P = np.stack([z * (X / 256.0 - cx) / f, z * (Y / 256.0 - cy) / f, z], 1)
        # a point inside the triangle in screen space
        bc = rng.dirichlet([1, 1, 1])
        px = int(round(bc @ X))
        py = int(round(bc @ Y))
        d = np.array([(px / 256.0 - cx) / f, (py / 256.0 - cy) / f, 1.0])
        n = np.cross(P[1] - P[0], P[2] - P[0])
        hit = d * (n @ P[0]) / (n @ d)
        # 3D barycentrics of the hit point
        A = np.stack([P[0] - P[2], P[1] - P[2]], 1)
        b01 = np.linalg.lstsq(A, hit - P[2], rcond=None)[0]
        beta = np.array([b01[0], b01[1], 1 - b01.sum()])
        want = beta @ uv.astype(np.float64)
        got = oracle.interp_uv(X, Y, 1.0 / z, uv, px, py)
        assert np.allclose(got, want, atol=1e-11)


def test_ray_direction_matches_pixel_rays():
    cam = synth.fibonacci_cameras(1, 4.0, 50, 30)[0]
    _, d = pixel_rays(cam)
    for (x, y) in [(0, 0), (49, 29), (17, 3), (25, 15)]:
        assert np.allclose(oracle.ray_dir(cam, x, y), d[y, x], atol=1e-14)


# ----------------------------------------------------------------------------
# compositing (Eq. 6 with Eq. 1's transmittance over earlier layers)
# ----------------------------------------------------------------------------

def _sure_hits(cam, shells_geo, margin_px=0.5):
    """Per pixel and shell: +1 surely hit, -1 surely missed, 0 ambiguous."""
    dist = ray_center_distance(cam)
    eye = np.linalg.norm(pixel_rays(cam)[0])
    m = margin_px * eye / cam.fx
    out = []
    for (pos, uv, tris) in shells_geo:
        r_in, r_out = inradius(pos, tris), float(np.linalg.norm(pos, axis=1).max())
        s = np.zeros(dist.shape, np.int8)
        s[dist < r_in - m] = 1
        s[dist > r_out + m] = -1
        out.append(s)
    return np.stack(out)


def _closed_form_composite(colors, alphas, bg, sure):
    """C = sum_{i<m} c_i a_i prod_{j<i}(1-a_j) + bg prod_{j<m}(1-a_j) where the
    m covered shells form a prefix (nested shells)."""
    k = len(alphas)
    H, W = sure.shape[1:]
    out = np.zeros((H, W, 4))
    valid = np.all(sure != 0, axis=0)
    for y, x in zip(*np.nonzero(valid)):
        C = np.zeros(3)
        T = 1.0
        for i in range(k):
            if sure[i, y, x] > 0:
                C += T * alphas[i] * np.asarray(colors[i])
                T *= 1 - alphas[i]
        out[y, x, :3] = C + T * np.asarray(bg)
        out[y, x, 3] = 1 - T
    return out, valid


def test_composite_closed_form_concentric_shells():
    geo = synth.concentric_icospheres([1.0, 0.9, 0.8], subdiv=3)
    colors = [(0.9, 0.2, 0.1), (0.1, 0.8, 0.3), (0.2, 0.3, 0.95)]
    alphas = [0.35, 0.6, 0.8]
    shells = [constant_shell(p, u, t, list(c) + [a], dtype=np.float64)
              for (p, u, t), c, a in zip(geo, colors, alphas)]
    cam = synth.look_at((1.5, -2.4, 0.9), width=96, height=96)
    bg = (0.25, 0.5, 0.75)
    rgba, hits, _ = oracle.render(Scene(shells), cam, bg=bg)
    sure = _sure_hits(cam, geo)
    want, valid = _closed_form_composite(colors, alphas, bg, sure)
    assert valid.sum() > 0.8 * valid.size
    for i in range(3):                        # every sure hit / miss agrees
        assert np.all(hits[i][sure[i] > 0] >= 0)
        assert np.all(hits[i][sure[i] < 0] == -1)
    assert np.abs(rgba[valid] - want[valid]).max() < 1e-12
    assert (sure.sum(0) == 3).sum() > 100     # all three layers seen somewhere


def test_single_opaque_shell_is_surface_render():
    """k = 1, alpha = 1: the blend reduces to an opaque surface render
    (Sec. 2, surface-based representations): output = texture colour."""
    pos, uv, tris = synth.icosphere(2, 1.0)
    rng = np.random.default_rng(8)
    tex = rng.random((16, 16, 4)).astype(np.float32)
    tex[..., 3] = 1.0
    sc = Scene([Shell(pos, uv, tris, tex, FMT_RGBA_F32)])
    cam = synth.look_at((0.4, -2.9, 0.6), width=64, height=64)
    rgba, hits, _ = oracle.render(sc, cam, bg=(0.3, 0.3, 0.3))
    h = hits[0] >= 0
    assert h.sum() > 1000
    assert np.abs(rgba[h][:, 3] - 1.0).max() < 1e-14
    assert np.all(rgba[~h] == [0.3, 0.3, 0.3, 0.0])
    # the background no longer shows through anywhere the shell is hit
    rgba0, _, _ = oracle.render(sc, cam, bg=(0, 0, 0))
    assert np.abs(rgba0[h] - rgba[h]).max() < 1e-14
    # and the colour is the texture seen along the FP64 ray (away from edges,
    # where snapping can move the sample point by a fraction of a pixel)
    eye, dirs = pixel_rays(cam)
    scr, _ = project64(pos, cam)
    p64 = pos.astype(np.float64)
    checked = 0
    for y, x in zip(*np.nonzero(h)):
        t = tris[hits[0, y, x]]
        if edge_distance_px(scr, t, x + 0.5, y + 0.5) < 0.05:
            continue
        if np.ptp(uv[t], axis=0).max() > 0.5:     # UV-seam faces: huge UV gradient
            continue
        a, b, c = p64[t]
        n = np.cross(b - a, c - a)
        d = dirs[y, x]
        pt = eye + d * (n @ (a - eye)) / (n @ d)
        A = np.stack([a - c, b - c], 1)
        b01 = np.linalg.lstsq(A, pt - c, rcond=None)[0]
        beta = np.array([b01[0], b01[1], 1 - b01.sum()])
        u, v = beta @ uv[t].astype(np.float64)
        want = oracle.sample(tex, u, v)[:3]
        assert np.abs(rgba[y, x, :3] - want).max() < 2e-3
        checked += 1
    assert checked > 1000


def test_transparent_shell_is_invisible():
    geo = synth.concentric_icospheres([1.0, 0.9, 0.8], subdiv=2)
    rng = np.random.default_rng(9)

    def tex(alpha=None):
        t = rng.random((8, 8, 4)).astype(np.float32)
        if alpha is not None:
            t[..., 3] = alpha
        return t
    t0, t1, t2 = tex(), tex(0.0), tex()
    full = Scene([Shell(*geo[0], t0, FMT_RGBA_F32), Shell(*geo[1], t1, FMT_RGBA_F32),
                  Shell(*geo[2], t2, FMT_RGBA_F32)])
    dropped = Scene([Shell(*geo[0], t0, FMT_RGBA_F32), Shell(*geo[2], t2, FMT_RGBA_F32)])
    cam = synth.look_at((0.0, -3.0, 0.5), width=48, height=48)
    a, _, _ = oracle.render(full, cam, bg=(0.1, 0.2, 0.3))
    b, _, _ = oracle.render(dropped, cam, bg=(0.1, 0.2, 0.3))
    assert np.abs(a - b).max() < 1e-15


def test_constant_sh_textures_closed_form():
    """Constant SH textures: colour = sigmoid(sum_m sh_m Y_m(v)) with v the
    pixel's ray direction, alpha = sigmoid(a); layout [a, rgb_0, rgb_1, ...]."""
    geo = synth.concentric_icospheres([1.0, 0.85], subdiv=3)
    rng = np.random.default_rng(10)
    deg = 3
    coeffs = [np.float16(rng.normal(0, 0.8, synth.sh_channels(deg))) for _ in geo]
    shells = [constant_shell(p, u, t, c, FMT_SH_F16, deg, dtype=np.float16)
              for (p, u, t), c in zip(geo, coeffs)]
    cam = synth.look_at((-1.2, 2.5, 1.3), width=64, height=64)
    bg = (0.05, 0.1, 0.9)
    rgba, hits, _ = oracle.render(Scene(shells), cam, bg=bg)
    sure = _sure_hits(cam, geo)
    _, dirs = pixel_rays(cam)
    valid = np.all(sure != 0, axis=0)
    checked = 0
    for y, x in zip(*np.nonzero(valid)):
        Y = real_sh_scipy(deg, dirs[y, x])
        C, T = np.zeros(3), 1.0
        for i, c in enumerate(coeffs):
            if sure[i, y, x] < 0:
                continue
            c = c.astype(np.float64)
            a = sigmoid(c[0])
            rgb = sigmoid(np.array([c[1 + ch::3][:16] @ Y for ch in range(3)]))
            C += T * a * rgb
            T *= 1 - a
        assert np.allclose(rgba[y, x, :3], C + T * np.asarray(bg), atol=1e-12)
        assert abs(rgba[y, x, 3] - (1 - T)) < 1e-12
        checked += 1
    assert checked > 1000


# ----------------------------------------------------------------------------
# near-plane clipping (close-up views): triangles crossing z = znear are cut
# there in camera space, the rest is rasterized under the same rules
# ----------------------------------------------------------------------------

def _tilted_lattice(n=14, seed=0):
    """A planar lattice in camera space (identity pose) from z = 0.02 (bottom
    rows, behind a near plane at 0.5) to z = 2.2 (top), jittered vertices;
    world = camera space, so rays and depths are known exactly."""
    rng = np.random.default_rng(seed)
    g = np.linspace(-1.0, 1.0, n)
    gx, gy = np.meshgrid(g, g)
    gx = gx + rng.uniform(-0.02, 0.02, gx.shape) * (np.abs(gx) < 1)
    gy = gy + rng.uniform(-0.02, 0.02, gy.shape) * (np.abs(gy) < 1)
    z = 1.11 - 1.09 * gy                         # y = +1 (bottom of the image) nearest
    pos = np.stack([0.9 * gx * z, 0.9 * gy * z * 0.7, z], -1).reshape(-1, 3).astype(np.float32)
    uv = np.stack([(gx + 1) / 2, (gy + 1) / 2], -1).reshape(-1, 2).astype(np.float32)
    tris = []
    for r in range(n - 1):
        for c in range(n - 1):
            a, b, d, e = r * n + c, r * n + c + 1, (r + 1) * n + c, (r + 1) * n + c + 1
            tris += [[a, b, e], [a, e, d]]
    tris = np.array(tris, np.int32)
    return pos, uv, tris


def _identity_camera(w, h, f, znear):
    return Camera(world_to_cam=np.concatenate([np.eye(3), np.zeros((3, 1))], 1).astype(np.float32),
                  fx=f, fy=f, cx=w / 2.0, cy=h / 2.0, znear=znear, width=w, height=h)


def _front_facing(pos, tris, cam):
    """Orient every triangle front-facing in the camera (normals towards it)."""
    p = pos.astype(np.float64)[tris]
    n = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    # front = counter-clockwise seen from the camera at the origin looking +z
    # with y down: the normal points towards the camera, n . centroid < 0
    flip = np.einsum("ij,ij->i", n, p.mean(1)) > 0
    t = tris.copy()
    t[flip] = t[flip][:, [0, 2, 1]]
    return t


def test_clipping_covers_the_visible_part_of_a_cut_lattice_exactly_once():
    """A lattice cut by the near plane: every pixel whose ray meets it in
    front of znear (by a margin) is covered exactly once -- clipped and
    unclipped parts tile without cracks, also along mesh edges cut by the
    plane, where both triangles must compute the same point -- and pixels
    whose hit lies behind znear are not covered."""
    w, h, f, znear = 96, 80, 70.0, 0.5
    cam = _identity_camera(w, h, f, znear)
    pos, uv, tris = _tilted_lattice()
    tris = _front_facing(pos, tris, cam)
    _, cover, stats = oracle.raster(pos, tris, cam, coverage=True)
    assert stats[4] > 10 and stats[2] > 10              # clipped and fully behind
    assert cover.max() <= 1
    # FP64 ray against the lattice plane pieces: ray cast on the mesh
    ys, xs = np.mgrid[0:h, 0:w]
    d = np.stack([(xs + 0.5 - cam.cx) / f, (ys + 0.5 - cam.cy) / f, np.ones(xs.shape)], -1)
    ids, tt, _ = raycast_front(np.zeros(3), d / np.linalg.norm(d, axis=-1, keepdims=True), pos, tris)
    z_hit = tt.reshape(h, w) / np.linalg.norm(d, axis=-1)         # camera z of the hit
    hit = ids.reshape(h, w) >= 0
    # away from the mesh border, where the hit is near an edge the fill rule decides
    scr_ok = np.ones((h, w), bool)
    front = hit & (z_hit > znear * 1.02)
    behind = hit & (z_hit < znear * 0.98)
    inner = front & np.roll(front, 1, 0) & np.roll(front, -1, 0) & np.roll(front, 1, 1) & np.roll(front, -1, 1)
    assert inner.sum() > 2000 and behind.sum() > 200
    assert np.all(cover[inner & scr_ok] == 1)
    assert np.all(cover[behind] == 0)


def test_clipped_parts_interpolate_the_ray_plane_uv():
    """UVs at the cut are interpolated along the 3D edge, and the clipped
    parts interpolate perspective-correctly from them: the UV seen through a
    pixel equals the UV of the FP64 ray-plane hit, on either side of a
    lattice edge cut by the near plane."""
    w, h, f, znear = 192, 160, 140.0, 0.5
    cam = _identity_camera(w, h, f, znear)
    pos, uv, tris = _tilted_lattice(seed=3)
    tris = _front_facing(pos, tris, cam)
    N = 16
    tex = np.zeros((N, N, 4), np.float64)
    tex[..., 0] = np.arange(N)[None, :]              # r = u N - 1/2 after bilinear, inside
    tex[..., 1] = np.arange(N)[:, None]              # g = v N - 1/2
    tex[..., 3] = 1.0
    sc = Scene([Shell(pos, uv, tris, tex, FMT_RGBA_F32)])
    rgba, hits, _ = oracle.render(sc, cam)
    ys, xs = np.mgrid[0:h, 0:w]
    d = np.stack([(xs + 0.5 - cam.cx) / f, (ys + 0.5 - cam.cy) / f, np.ones(xs.shape)], -1)
    p64 = pos.astype(np.float64)
    ps, _ = project64(pos, cam)
    checked = 0
    stats = oracle.raster(pos, tris, cam)[2]
    assert stats[4] > 10
    for y, x in zip(*np.nonzero(hits[0] >= 0)):
        t = tris[hits[0, y, x]]
        a, b, c = p64[t]
        n = np.cross(b - a, c - a)
        dd = d[y, x]
        pt = dd * (n @ a) / (n @ dd)
        A = np.stack([a - c, b - c], 1)
        b01 = np.linalg.lstsq(A, pt - c, rcond=None)[0]
        beta = np.array([b01[0], b01[1], 1 - b01.sum()])
        want = beta @ uv[t].astype(np.float64)
        if np.any((want < 0.5 / N + 1e-3) | (want > 1 - 0.5 / N - 1e-3)):
            continue                                  # clamp-to-edge zone
        got = (rgba[y, x, :2] + 0.5) / N
        # vertices snap to 1/256 px: on ~14 px triangles spanning 1/13 in UV
        # that moves the UV by up to ~2e-5
        assert np.abs(got - want).max() < 1e-4
        if min(p64[t][:, 2]) < znear:                # a clipped triangle
            checked += 1
    assert checked > 150


def test_close_up_nested_shells_match_a_ray_cast_that_skips_the_near_zone():
    """Camera close to nested shells with the near plane through the outer
    one: each shell's nearest front hit is the FP64 ray cast's nearest front
    hit with camera depth >= znear (away from edges and from the cut)."""
    geo = synth.concentric_icospheres([1.0, 0.8], subdiv=4)
    cam = synth.look_at((0.0, -1.45, 0.25), width=72, height=72, fov_y_deg=60.0, znear=0.6)
    eye, dirs = pixel_rays(cam)
    R = cam.world_to_cam[:, :3].astype(np.float64)
    checked = 0
    clipped_seen = 0
    for i, (pos, uv, tris) in enumerate(geo):
        _, cover, stats = oracle.raster(pos, tris, cam, coverage=True)
        clipped_seen += stats[4]
        hits = oracle.hits_from_keys(oracle.raster(pos, tris, cam)[0])
        p = pos.astype(np.float64)
        a, b, c = p[tris[:, 0]], p[tris[:, 1]], p[tris[:, 2]]
        n = np.cross(b - a, c - a)
        for y in range(0, 72, 2):
            for x in range(0, 72, 2):
                dd = dirs[y, x]
                denom = n @ dd
                with np.errstate(divide="ignore", invalid="ignore"):
                    tt = np.einsum("ij,ij->i", n, a - eye) / denom
                P = eye + tt[:, None] * dd
                zc = (P - eye) @ R[2]
                # inside-triangle test via barycentrics
                v0, v1, v2 = b - a, c - a, P - a
                d00 = np.einsum("ij,ij->i", v0, v0); d01 = np.einsum("ij,ij->i", v0, v1)
                d11 = np.einsum("ij,ij->i", v1, v1); d20 = np.einsum("ij,ij->i", v2, v0)
                d21 = np.einsum("ij,ij->i", v2, v1)
                den = d00 * d11 - d01 * d01
                bv = (d11 * d20 - d01 * d21) / den
                bw = (d00 * d21 - d01 * d20) / den
                bu = 1 - bv - bw
                mb = np.minimum(np.minimum(bu, bv), bw)
                front = (denom < 0) & (tt > 0)
                ok = front & (mb > 2e-3) & (zc >= cam.znear * 1.01)
                # undecidable here: a front face within 2e-3 (barycentric) of
                # its edge, or hit within 1 % of the near plane
                edge = front & (np.abs(mb) <= 2e-3) & (zc >= cam.znear * 0.99)
                cut = front & (mb > -2e-3) & (np.abs(zc - cam.znear) < cam.znear * 0.01)
                if edge.any() or cut.any():
                    continue
                want = int(np.argmin(np.where(ok, tt, np.inf))) if ok.any() else -1
                assert hits[y, x] == want, (i, y, x)
                checked += 1
    assert clipped_seen > 50 and checked > 800


# ----------------------------------------------------------------------------
# per-layer buffers (Figs. S1/S3): each shell before blending
# ----------------------------------------------------------------------------

def test_layer_buffers_recompose_the_image():
    """The per-shell weights T_i alpha_i sum to the composite's alpha and
    sum_i weight_i rgb_i + (1 - alpha) bg is its colour; opacity is within
    [0, 1], normals are unit vectors facing the camera and missed shells are
    all zero; flag on or off."""
    (sc, cams), = synth.config_scene("c2", scale=0.003, views=2)
    for flags in (0, oracle.ALPHA_ATTEN):
        cam = cams[1]
        hits, _, _ = oracle.raster_scene(sc, cam)
        bg = np.array([0.3, 0.1, 0.6])
        lay, rgba = oracle.layers(sc, cam, hits, bg=tuple(bg), flags=flags)
        w = lay[..., 6]
        assert np.abs(w.sum(0) - rgba[..., 3]).max() < 1e-12
        col = (w[..., None] * lay[..., 7:10]).sum(0) + (1 - rgba[..., 3:4]) * bg
        assert np.abs(col - rgba[..., :3]).max() < 1e-12
        hit = hits >= 0
        assert np.all(lay[~hit] == 0)
        n = lay[..., 0:3][hit]
        assert np.abs(np.linalg.norm(n, axis=-1) - 1).max() < 1e-12
        eye, dirs = pixel_rays(cam)
        facing = np.einsum("khwc,hwc->khw", lay[..., 0:3], dirs)[hit]
        assert np.all(facing < 0)                  # front faces turn towards the viewer
        assert lay[..., 5][hit].min() >= 0 and lay[..., 5][hit].max() <= 1
        # T_i alpha_i from the per-layer opacities, front to back
        T = np.ones(hits.shape[1:])
        for i in range(sc.k):
            a = lay[i, ..., 5]
            assert np.abs(lay[i, ..., 6] - T * a).max() < 1e-12
            T = T * (1 - a)


def test_layer_uv_and_normal_of_a_planar_quad():
    """A slanted textured quad: every covered pixel's layer UV is the FP64
    ray-plane intersection's UV and its normal the plane's."""
    th = math.radians(55.0)
    ax, az = np.array([1.0, 0.0, 0.0]), np.array([0.0, math.sin(th), math.cos(th)])
    corners = np.array([-ax - az, ax - az, ax + az, -ax + az])
    pos = corners.astype(np.float32)
    uv = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float32)
    tris = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    n = np.cross(ax, az)
    view = 0.8 * n + 0.4 * az + 0.2 * ax
    cam = synth.look_at(tuple(3.0 * view / np.linalg.norm(view)), width=64, height=64)
    if oracle.raster_scene(Scene([constant_shell(pos, uv, tris, [0, 0, 0, 1])]), cam)[0][0].max() < 0:
        tris = tris[:, ::-1].copy()
    sc = Scene([constant_shell(pos, uv, tris, [0.2, 0.4, 0.6, 0.5])])
    hits, _, _ = oracle.raster_scene(sc, cam)
    lay, _ = oracle.layers(sc, cam, hits)
    eye, dirs = pixel_rays(cam)
    p64 = pos.astype(np.float64)
    nn = np.cross(p64[tris[0, 1]] - p64[tris[0, 0]], p64[tris[0, 2]] - p64[tris[0, 0]])
    nn /= np.linalg.norm(nn)
    h = hits[0] >= 0
    assert h.sum() > 500
    assert np.abs(lay[0][h][:, 0:3] - nn).max() < 1e-12
    checked = 0
    for y, x in zip(*np.nonzero(h)):
        d = dirs[y, x]
        pt = eye + d * (nn @ (p64[0] - eye)) / (nn @ d)
        a, b = p64[1] - p64[0], p64[3] - p64[0]
        uu = (pt - p64[0]) @ a / (a @ a)
        vv = (pt - p64[0]) @ b / (b @ b)
        # vertices snap to 1/256 px: a ~30 px quad side moves UV by ~1e-4
        assert abs(lay[0, y, x, 3] - uu) < 3e-4 and abs(lay[0, y, x, 4] - vv) < 3e-4
        checked += 1
    assert checked > 500


# ----------------------------------------------------------------------------
# transparency attenuation (Sec. 3): alpha_w = 2 sigmoid(10 |v . n|) - 1
# ----------------------------------------------------------------------------

def test_attenuation_tilted_plane_closed_form():
    """One planar quad with constant colour and alpha, seen at a slant: every
    covered pixel composites alpha * (2 sigmoid(10 |v . n|) - 1) over the
    background, v the pixel ray and n the plane normal; head-on rays keep
    nearly all of alpha, grazing ones lose most of it."""
    th = math.radians(70.0)
    ax, az = np.array([1.0, 0.0, 0.0]), np.array([0.0, math.sin(th), math.cos(th)])
    n = np.cross(ax, az)                     # unit plane normal
    corners = [-ax - az, ax - az, ax + az, -ax + az]
    pos = np.array(corners, np.float32)
    uv = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float32)
    tris = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    view = 0.35 * n + az + 0.2 * ax                # about 18 degrees above the plane
    eye = 3.0 * view / np.linalg.norm(view)
    cam = synth.look_at(tuple(eye), target=(0.0, 0.0, 0.0), width=64, height=64)
    if oracle.raster_scene(Scene([constant_shell(pos, uv, tris, [0, 0, 0, 1])]), cam)[0][0].max() < 0:
        tris = tris[:, ::-1].copy()          # make the quad face the camera
    color, a, bg = np.array([0.8, 0.3, 0.1]), 0.7, np.array([0.1, 0.2, 0.9])
    sc = Scene([constant_shell(pos, uv, tris, list(color) + [a], dtype=np.float64)])
    rgba, hits, _ = oracle.render(sc, cam, bg=tuple(bg), flags=oracle.ALPHA_ATTEN)
    plain, _, _ = oracle.render(sc, cam, bg=tuple(bg))
    _, dirs = pixel_rays(cam)
    h = hits[0] >= 0
    assert h.sum() > 500
    p64 = pos.astype(np.float64)            # the normal of the stored (FP32) plane
    n = np.cross(p64[1] - p64[0], p64[3] - p64[0])
    n /= np.linalg.norm(n)
    aw = 2.0 / (1.0 + np.exp(-10.0 * np.abs(dirs @ n))) - 1.0
    ae = a * aw
    want = ae[..., None] * color + (1 - ae[..., None]) * bg
    assert np.abs(rgba[h][:, :3] - want[h]).max() < 1e-12
    assert np.abs(rgba[h][:, 3] - ae[h]).max() < 1e-12
    assert np.all(rgba[~h] == plain[~h])
    assert np.abs(plain[h][:, 3] - a).max() < 1e-15       # flag off: unchanged
    assert 0.0 < aw[h].min() < aw[h].max() < 1.0


def test_attenuation_grazing_and_head_on_limits():
    """|v . n| = 1 gives alpha_w = 2 sigmoid(10) - 1 (the sphere's centre
    pixel, seen head on) and v . n -> 0 gives alpha_w -> 0 (its silhouette)."""
    pos, uv, tris = synth.icosphere(4, 1.0)
    sc = Scene([constant_shell(pos, uv, tris, [0.5, 0.5, 0.5, 1.0], dtype=np.float64)])
    cam = synth.look_at((0.0, -4.0, 0.0), width=96, height=96)
    rgba, hits, _ = oracle.render(sc, cam, flags=oracle.ALPHA_ATTEN)
    h = hits[0] >= 0
    a = rgba[..., 3]
    # the pixel nearest the sphere's centre sees it almost head on
    assert abs(a[48, 48] - (2 / (1 + math.exp(-10)) - 1)) < 2e-3
    # silhouette pixels (hit, with a missed 4-neighbour) are strongly attenuated
    edge = h & ~(np.roll(h, 1, 0) & np.roll(h, -1, 0) & np.roll(h, 1, 1) & np.roll(h, -1, 1))
    assert edge.sum() > 50 and a[edge].min() >= 0.0
    assert a[edge].mean() < 0.7 * a[h].max() and a[edge].max() < a[48, 48]
    assert np.all(a[h] <= 2 / (1 + math.exp(-10)) - 1 + 1e-15)


def test_attenuation_nested_shells_use_each_hit_face_normal():
    """Nested icospheres, flag on: each layer's alpha is scaled by the weight
    of its own hit triangle's face normal (the flat normal of the baked mesh,
    not the radial direction), then the usual front-to-back blend."""
    geo = synth.concentric_icospheres([1.0, 0.9, 0.8], subdiv=1)
    colors = [np.array([0.9, 0.2, 0.1]), np.array([0.1, 0.8, 0.3]), np.array([0.2, 0.3, 0.95])]
    alphas = [0.35, 0.6, 0.8]
    shells = [constant_shell(p, u, t, list(c) + [a], dtype=np.float64)
              for (p, u, t), c, a in zip(geo, colors, alphas)]
    cam = synth.look_at((1.5, -2.4, 0.9), width=64, height=64)
    bg = np.array([0.25, 0.5, 0.75])
    rgba, hits, _ = oracle.render(Scene(shells), cam, bg=tuple(bg), flags=oracle.ALPHA_ATTEN)
    _, dirs = pixel_rays(cam)
    normals = []
    for (p, _, t) in geo:
        p = p.astype(np.float64)
        nn = np.cross(p[t[:, 1]] - p[t[:, 0]], p[t[:, 2]] - p[t[:, 0]])
        normals.append(nn / np.linalg.norm(nn, axis=1, keepdims=True))
    radial_differs = 0
    for y in range(64):
        for x in range(64):
            C, T = np.zeros(3), 1.0
            for i in range(3):
                t = hits[i, y, x]
                if t < 0:
                    continue
                vn = abs(dirs[y, x] @ normals[i][t])
                ae = alphas[i] * (2 / (1 + math.exp(-10 * vn)) - 1)
                C += T * ae * colors[i]
                T *= 1 - ae
            assert np.abs(rgba[y, x, :3] - (C + T * bg)).max() < 1e-12
            assert abs(rgba[y, x, 3] - (1 - T)) < 1e-12
            if hits[0, y, x] >= 0:
                pt = geo[0][0][geo[0][2][hits[0, y, x]]].astype(np.float64).mean(0)
                vr = abs(dirs[y, x] @ (pt / np.linalg.norm(pt)))
                radial_differs += abs(vr - abs(dirs[y, x] @ normals[0][hits[0, y, x]])) > 1e-3
    assert radial_differs > 100


# ----------------------------------------------------------------------------
# the baked format (Sec. 3 "Mixed Resolutions", "Squeezing and Quantization",
# "Baking Textures"): RGBA SH bytes, band l at (W, H) >> l s
# ----------------------------------------------------------------------------

def _band_table(tw, th, degree, shift):
    """The documented layout, written out independently of synth."""
    strides = {0: 4, 1: 16, 2: 32, 3: 32}
    out, off = [], 0
    for band in range(degree + 1):
        w, h = tw >> (band * shift), th >> (band * shift)
        out.append((off, w, h, strides[band]))
        off += ((w * h * strides[band] + 255) // 256) * 256
    return out, off


def _baked_shell(buf, tw, th, degree, shift, vmin=-15.0, vmax=15.0, geo=None):
    pos, uv, tris = geo if geo is not None else synth.icosphere(1, 1.0)
    return Shell(pos, uv, tris, buf, FMT_SH_U8, degree, tex_w=tw, tex_h=th, band_shift=shift,
                 vmin=vmin, vmax=vmax)


@pytest.mark.parametrize("tw,th,degree,shift", [(16, 8, 3, 1), (8, 8, 2, 0), (32, 16, 1, 2), (4, 4, 0, 1),
                                                (12, 6, 2, 0), (20, 12, 1, 1)])
def test_baked_texel_centres_decode_their_bytes(tw, th, degree, shift):
    """At the centre of band-l texel (x, y) every coefficient of the band
    decodes to vmin + (vmax - vmin) q / 255 of its own byte in the
    documented layout (256-byte aligned bands, RGBA quadruples per
    coefficient)."""
    table, total = _band_table(tw, th, degree, shift)
    assert synth.baked_layout(tw, th, degree, shift) == (table, total)
    rng = np.random.default_rng(tw * 7 + degree)
    buf = rng.integers(0, 256, total, dtype=np.uint8)
    vmin, vmax = -3.0, 12.0
    sh = _baked_shell(buf, tw, th, degree, shift, vmin, vmax)
    for band, (off, w, h, stride) in enumerate(table):
        for _ in range(6):
            x, y = int(rng.integers(0, w)), int(rng.integers(0, h))
            for j in range(2 * band + 1):
                got = oracle.sample_baked(sh, band * band + j, (x + 0.5) / w, (y + 0.5) / h)
                q = buf[off + (y * w + x) * stride + 4 * j: off + (y * w + x) * stride + 4 * j + 4]
                assert np.abs(got - (vmin + (vmax - vmin) * q.astype(np.float64) / 255.0)).max() < 1e-12


def test_baked_bands_interpolate_at_their_own_resolution():
    """Bytes affine in each band's texel index are reproduced exactly by the
    bilinear fetch at any interior UV, with the band's own resolution:
    q(u, v) = b0 + gx (u w_l - 1/2) + gy (v h_l - 1/2)."""
    tw, th, degree, shift = 32, 32, 3, 1
    table, total = _band_table(tw, th, degree, shift)
    buf = np.zeros(total, np.uint8)
    coef = {}
    for band, (off, w, h, stride) in enumerate(table):
        for j in range(2 * band + 1):
            for c in range(4):
                b0, gx, gy = 10 + 3 * j + c, 1 + (j + c) % 3, 2 - (c % 2)
                coef[(band * band + j, c)] = (b0, gx, gy, w, h)
                ys, xs = np.mgrid[0:h, 0:w]
                img = b0 + gx * xs + gy * ys
                assert img.max() <= 255
                view = buf[off: off + w * h * stride].reshape(h, w, stride)
                view[..., 4 * j + c] = img
    vmin, vmax = -15.0, 15.0
    sh = _baked_shell(buf, tw, th, degree, shift, vmin, vmax)
    rng = np.random.default_rng(3)
    for _ in range(40):
        u, v = rng.uniform(0.25, 0.75, 2)       # interior for every band (4x4 smallest)
        for m in range(16):
            got = oracle.sample_baked(sh, m, u, v)
            for c in range(4):
                b0, gx, gy, w, h = coef[(m, c)]
                q = b0 + gx * (u * w - 0.5) + gy * (v * h - 0.5)
                assert abs(got[c] - (vmin + (vmax - vmin) * q / 255.0)) < 1e-12


def test_baked_constant_textures_closed_form_view_dependent_alpha():
    """Constant baked bytes on concentric shells: every channel, alpha
    included, is sigmoid(sum_m value_{m,c} Y_m(v)) with scipy's real SH and
    the FP64 pixel ray, composited front to back."""
    geo = synth.concentric_icospheres([1.0, 0.85], subdiv=3)
    deg, tw = 3, 16
    table, total = _band_table(tw, tw, deg, 1)
    rng = np.random.default_rng(21)
    shells, values = [], []
    for g in geo:
        qv = rng.integers(60, 200, (16, 4))           # per (coefficient, channel)
        buf = np.zeros(total, np.uint8)
        for band, (off, w, h, stride) in enumerate(table):
            view = buf[off: off + w * h * stride].reshape(h, w, stride)
            for j in range(2 * band + 1):
                view[..., 4 * j: 4 * j + 4] = qv[band * band + j]
        shells.append(_baked_shell(buf, tw, tw, deg, 1, geo=g))
        values.append(-15.0 + 30.0 * qv.astype(np.float64) / 255.0)
    cam = synth.look_at((-1.2, 2.5, 1.3), width=64, height=64)
    bg = (0.05, 0.1, 0.9)
    rgba, hits, _ = oracle.render(Scene(shells), cam, bg=bg)
    sure = _sure_hits(cam, geo)
    _, dirs = pixel_rays(cam)
    valid = np.all(sure != 0, axis=0)
    checked = 0
    for y, x in zip(*np.nonzero(valid)):
        Y = real_sh_scipy(deg, dirs[y, x])
        C, T = np.zeros(3), 1.0
        for i, val in enumerate(values):
            if sure[i, y, x] < 0:
                continue
            z = Y @ val                                  # [4] = sum_m Y_m value_{m,c}
            a = sigmoid(z[3])
            C += T * a * sigmoid(z[:3])
            T *= 1 - a
        assert np.allclose(rgba[y, x, :3], C + T * np.asarray(bg), atol=1e-12)
        assert abs(rgba[y, x, 3] - (1 - T)) < 1e-12
        checked += 1
    assert checked > 1000


def test_baked_format_has_no_gradient():
    (sc, cams), = synth.config_scene("c2b", scale=0.002, views=1)
    hits, _, _ = oracle.raster_scene(sc, cams[0])
    with pytest.raises(ValueError):
        oracle.backward(sc, cams[0], hits, np.zeros((cams[0].height, cams[0].width, 3)))


# ----------------------------------------------------------------------------
# backward (Sec. 3 "Texturing Meshes": fitting texels through the renderer)
# ----------------------------------------------------------------------------

def _tiny_scene(fmt, degree, seed, size=4):
    geo = synth.concentric_icospheres([1.0, 0.85], subdiv=1)
    rng = np.random.default_rng(seed)
    shells = []
    for (p, u, t) in geo:
        if fmt == FMT_RGBA_F32:
            tex = rng.uniform(0.1, 0.9, (size, size, 4))
        else:
            tex = rng.normal(0, 0.5, (size, size, synth.sh_channels(degree)))
        shells.append(Shell(p, u, t, tex.astype(np.float64), fmt, degree))
    return Scene(shells)


@pytest.mark.parametrize("fmt,degree,flags", [(FMT_RGBA_F32, 0, 0), (FMT_SH_F16, 1, 0), (FMT_SH_F16, 2, 0),
                                               (FMT_RGBA_F32, 0, oracle.ALPHA_ATTEN),
                                               (FMT_SH_F16, 2, oracle.ALPHA_ATTEN)])
def test_backward_matches_central_differences(fmt, degree, flags):
    sc = _tiny_scene(fmt, degree, seed=20 + degree)
    cam = synth.look_at((0.7, -2.8, 0.9), width=20, height=18)
    bg = (0.2, 0.4, 0.6)
    hits, _, _ = oracle.raster_scene(sc, cam)
    rng = np.random.default_rng(30)
    g = rng.normal(size=(cam.height, cam.width, 3))
    grads = oracle.backward(sc, cam, hits, g, bg=bg, flags=flags)

    def loss():
        return float((oracle.shade(sc, cam, hits, bg=bg, threads=1, flags=flags)[0][..., :3] * g).sum())

    h = 1e-6
    worst = 0.0
    for i, s in enumerate(sc.shells):
        flat = s.tex.reshape(-1)
        for j in range(flat.size):
            v0 = flat[j]
            flat[j] = v0 + h
            lp = loss()
            flat[j] = v0 - h
            lm = loss()
            flat[j] = v0
            fd = (lp - lm) / (2 * h)
            worst = max(worst, abs(fd - grads[i].reshape(-1)[j]))
    assert worst < 1e-7
    assert max(np.abs(gr).max() for gr in grads) > 1e-2


def test_backward_constant_texture_closed_form():
    """Constant RGBA textures: bilinear weights sum to one, so the gradient
    summed over a shell's texels is sum_pixels T_i a_i g for rgb and
    sum_pixels T_i (c_i - A_{i+1}) . g for alpha (A = colour behind)."""
    geo = synth.concentric_icospheres([1.0, 0.9, 0.8], subdiv=2)
    colors = [np.array([0.9, 0.2, 0.1]), np.array([0.1, 0.8, 0.3]), np.array([0.2, 0.3, 0.95])]
    alphas = [0.35, 0.6, 0.8]
    shells = [constant_shell(p, u, t, list(c) + [a], dtype=np.float64)
              for (p, u, t), c, a in zip(geo, colors, alphas)]
    sc = Scene(shells)
    cam = synth.look_at((1.1, -2.6, 0.7), width=40, height=40)
    bg = np.array([0.3, 0.1, 0.5])
    hits, _, _ = oracle.raster_scene(sc, cam)
    g = np.random.default_rng(12).normal(size=(40, 40, 3))
    grads = oracle.backward(sc, cam, hits, g, bg=bg)
    want_rgb = np.zeros((3, 3))
    want_a = np.zeros(3)
    for y in range(40):
        for x in range(40):
            on = [i for i in range(3) if hits[i, y, x] >= 0]
            T, Ts = 1.0, {}
            for i in on:
                Ts[i] = T
                T *= 1 - alphas[i]
            A = bg.copy()
            for i in reversed(on):
                want_rgb[i] += Ts[i] * alphas[i] * g[y, x]
                want_a[i] += Ts[i] * (colors[i] - A) @ g[y, x]
                A = alphas[i] * colors[i] + (1 - alphas[i]) * A
    for i in range(3):
        assert np.allclose(grads[i][..., :3].sum((0, 1)), want_rgb[i], atol=1e-10)
        assert abs(grads[i][..., 3].sum() - want_a[i]) < 1e-10


# ----------------------------------------------------------------------------
# the workloads themselves
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["c1", "c2", "c3", "c4", "c5"])
def test_workloads_cull_nothing_at_near_plane_or_guard_band(name):
    """Cameras stay outside the shells: no triangle crosses the near plane or
    leaves the guard band, so culling is back faces only."""
    objs = synth.config_scene(name, scale=0.002, views=2)
    for sc, cams in objs[:4]:
        for cam in cams[:2]:
            for s in sc.shells:
                xy, invw, q, flags = oracle.setup_vertices(s.pos, cam)
                assert np.all(flags == 0)


# ----------------------------------------------------------------------------
# image losses (the L1 colour loss of Sec. 3 "Texturing Meshes"; the L2 one of
# the fitting benchmark)
# ----------------------------------------------------------------------------

def _loss_case():
    rgba = np.zeros((1, 2, 4))
    rgba[0, 0, :3] = (0.5, 0.25, 1.0)
    rgba[0, 1, :3] = (0.0, 0.75, 0.5)
    target = np.array([[[0.25, 0.25, 0.0], [0.5, 0.5, 0.5]]])
    return rgba, target


def test_l1_loss_closed_form():
    rgba, target = _loss_case()
    L, g = oracle.l1_loss_grad(rgba, target)
    # |d| = 0.25, 0, 1, 0.5, 0.25, 0 over 6 values
    assert L == pytest.approx(2.0 / 6.0, abs=1e-15)
    assert np.array_equal(g * 6.0, np.array([[[1.0, 0.0, 1.0], [-1.0, 1.0, 0.0]]]))


def test_l2_loss_closed_form():
    rgba, target = _loss_case()
    L, g = oracle.l2_loss_grad(rgba, target)
    assert L == pytest.approx((0.0625 + 1.0 + 0.25 + 0.0625) / 6.0, abs=1e-15)
    assert np.allclose(g * 6.0, 2.0 * np.array([[[0.25, 0.0, 1.0], [-0.5, 0.25, 0.0]]]), atol=1e-15)


@pytest.mark.parametrize("which", ["l1", "l2"])
def test_loss_gradients_match_finite_differences(which):
    rng = np.random.default_rng(11)
    rgba = rng.random((5, 7, 4))
    target = rng.random((5, 7, 3))
    fn = oracle.l1_loss_grad if which == "l1" else oracle.l2_loss_grad
    _, g = fn(rgba, target)
    h = 1e-7
    for idx in [(0, 0, 0), (2, 3, 1), (4, 6, 2), (1, 5, 0)]:
        assert abs(rgba[idx] - target[idx]) > 10 * h   # away from the L1 kink
        p, m = rgba.copy(), rgba.copy()
        p[idx] += h
        m[idx] -= h
        fd = (fn(p, target)[0] - fn(m, target)[0]) / (2 * h)
        assert fd == pytest.approx(g[idx], rel=1e-6, abs=1e-9)


def test_l1_at_most_root_l2():
    """mean |d| <= sqrt(mean d^2), equality for constant |d|."""
    rng = np.random.default_rng(12)
    rgba, target = rng.random((6, 5, 4)), rng.random((6, 5, 3))
    assert oracle.l1_loss_grad(rgba, target)[0] <= math.sqrt(oracle.l2_loss_grad(rgba, target)[0])
    flat = np.zeros((2, 2, 4))
    tgt = np.full((2, 2, 3), 0.5)
    flat[..., :3] = tgt + np.where(rng.random((2, 2, 3)) < 0.5, -0.25, 0.25)
    assert oracle.l1_loss_grad(flat, tgt)[0] == pytest.approx(math.sqrt(oracle.l2_loss_grad(flat, tgt)[0]))


def test_backward_error_scales():
    """The per-texel error scales of the adjoint (the yardstick of the GPU
    gradient bars; no part of the method): they leave the gradient unchanged,
    bound it (|grad| <= S_w <= S_1, zero exactly where nothing reaches), equal
    |grad| where no term can cancel (colour values of RGBA textures and the
    Y_0 coefficients of SH textures under a nonnegative output gradient), sum
    over a constant texture to the per-fragment magnitudes -- the alpha one
    T_i (|c_i| + |A_{i+1}|) . |g| -- and count four taps per fragment."""
    bg = np.array([0.3, 0.1, 0.5])
    # (1) random textures, signed gradient
    for fmt, degree in ((FMT_RGBA_F32, 0), (FMT_SH_F16, 2)):
        sc = _tiny_scene(fmt, degree, seed=40 + degree)
        cam = synth.look_at((0.7, -2.8, 0.9), width=24, height=20)
        hits, _, _ = oracle.raster_scene(sc, cam)
        g = np.random.default_rng(41).normal(size=(cam.height, cam.width, 3))
        plain = oracle.backward(sc, cam, hits, g, bg=bg)
        grads, (sw, s1, sy) = oracle.backward(sc, cam, hits, g, bg=bg, with_scale=True)
        same, _ = oracle.backward(sc, cam, hits, g, bg=bg, with_scale=True, gmag=np.abs(g))
        for a, b, c, w, r in zip(plain, grads, same, sw, s1):
            assert np.array_equal(a, b) and np.array_equal(a, c)
            assert np.all(np.abs(a) <= w * (1 + 1e-12)) and np.all(w <= r * (1 + 1e-12))
            assert np.array_equal(w == 0, r == 0) and np.all(a[w == 0] == 0)
        assert max(float(w.max()) for w in sw) > 0
        # a tap-weight allowance widens S_1 beside footprints near texel
        # lines and changes neither the gradient nor S_w
        g2, (sw2, s12, _) = oracle.backward(sc, cam, hits, g, bg=bg, with_scale=True, weight_err=0.25)
        for a, b, w, w2, r, r2 in zip(grads, g2, sw, sw2, s1, s12):
            assert np.array_equal(a, b) and np.array_equal(w, w2) and np.all(r2 >= r)
        assert any(np.any((r2 > 0) & (r == 0)) for r, r2 in zip(s1, s12))
        # (2) nonnegative output gradient: no cancellation in the colour terms
        gp = np.abs(g)
        grads, (sw, _, sy) = oracle.backward(sc, cam, hits, gp, bg=bg, with_scale=True)
        cols = slice(0, 3) if fmt == FMT_RGBA_F32 else slice(1, 4)
        for a, w in zip(grads, sw):
            assert np.allclose(np.abs(a[..., cols]), w[..., cols], rtol=1e-12, atol=0)
        # S_y: the coefficient terms without their basis value -- none for
        # RGBA and the alpha logit; for Y_0 (a constant) S_w = Y_0 S_y
        for w, y in zip(sw, sy):
            if fmt == FMT_RGBA_F32:
                assert not y.any()
            else:
                assert not y[..., 0].any()
                assert np.allclose(w[..., 1:4], oracle.sh_basis(0, [0.0, 0.0, 1.0])[0] * y[..., 1:4], rtol=1e-12)
        # the alpha terms do cancel somewhere: strictly larger scale there
        assert any(np.any(w[..., 3 if fmt == FMT_RGBA_F32 else 0] > np.abs(a[..., 3 if fmt == FMT_RGBA_F32 else 0]) * 1.01)
                   for a, w in zip(grads, sw))
    # (3) constant RGBA textures: closed forms of the sums
    geo = synth.concentric_icospheres([1.0, 0.9, 0.8], subdiv=2)
    colors = [np.array([0.9, 0.2, 0.1]), np.array([0.1, 0.8, 0.3]), np.array([0.2, 0.3, 0.95])]
    alphas = [0.35, 0.6, 0.8]
    sc = Scene([constant_shell(p, u, t, list(c) + [a], dtype=np.float64)
                for (p, u, t), c, a in zip(geo, colors, alphas)])
    cam = synth.look_at((1.1, -2.6, 0.7), width=32, height=32)
    hits, _, _ = oracle.raster_scene(sc, cam)
    g = np.random.default_rng(13).normal(size=(32, 32, 3))
    _, (sw, s1, sy) = oracle.backward(sc, cam, hits, g, bg=bg, with_scale=True)
    want_rgb, want_a = np.zeros((3, 3)), np.zeros(3)
    for y in range(32):
        for x in range(32):
            on = [i for i in range(3) if hits[i, y, x] >= 0]
            T, Ts = 1.0, {}
            for i in on:
                Ts[i] = T
                T *= 1 - alphas[i]
            A = bg.copy()
            for i in reversed(on):
                want_rgb[i] += Ts[i] * alphas[i] * np.abs(g[y, x])
                want_a[i] += Ts[i] * (np.abs(colors[i]) + np.abs(A)) @ np.abs(g[y, x])
                A = alphas[i] * colors[i] + (1 - alphas[i]) * A
    for i in range(3):
        assert np.allclose(sw[i][..., :3].sum((0, 1)), want_rgb[i], rtol=1e-10)
        assert abs(sw[i][..., 3].sum() - want_a[i]) < 1e-10 * want_a[i]
        assert np.allclose(s1[i].sum((0, 1)), 4 * sw[i].sum((0, 1)), rtol=1e-10)
