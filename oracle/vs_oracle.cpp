// FP64 CPU oracle of the k-shell ("Volumetric Surfaces") renderer.
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
// baseline leg of the benchmark load this library; the product path never
// does.  It shares no code, header, table or constant with the CUDA path.
//
// What it computes, step by step, in the paper's order:
//   * Sec. 3 "Baking Textures" / Sec. 4 real-time renderer: every shell is a
//     triangle mesh, rasterized in a fixed outer-to-inner order, each with
//     its own nearest-hit test ("only sampling the first intersection with
//     each surface", Fig. 3c).
//   * Sec. 3 "Texturing Meshes", Fig. 5: the texture value at a UV point is
//     the bilinear mix of the four surrounding texel centers, like an OpenGL
//     fragment shader; SH coefficients are decoded with the view direction v
//     (the ray direction of Sec. 2, r(t) = o + v t) into RGBA.
//   * Eq. 6 with the transmittance of Eq. 1 (products over *earlier* layers
//     only): C = sum_i c_i a_i prod_{j<i} (1 - a_j), front to back.
//   * Sec. 3 "Texturing Meshes": texture fitting differentiates the renderer
//     with respect to texel values; the adjoint below is that derivative.
//
// Discrete rules the paper leaves open (readings of the silent parts):
//   * vertices go through an FP32 world->camera->screen transform in a fixed
//     operation order (each op rounded to float, no fused multiply-add; this
//     file must be compiled with -ffp-contract=off), are snapped to 1/256 px
//     with round-half-even, and carry a depth key q = rint(2^30 znear / w);
//   * pixel centers (x + 1/2, y + 1/2), one sample per pixel;
//   * integer edge functions, top-left fill rule, front faces only
//     (counter-clockwise seen from outside), zero-area faces culled,
//     faces with a vertex nearer than znear or beyond +-32768 px culled;
//   * depth key at a pixel K = floor(sum_j e_j q_j / sum_j e_j) in exact
//     integer arithmetic; the nearest (largest K) wins, ties go to the lower
//     triangle index;
//   * perspective-correct barycentrics, texel (x, y) centred at
//     ((x+1/2)/W, (y+1/2)/H), clamp-to-edge, no mipmaps;
//   * SH_F16: alpha = sigmoid(a), rgb = sigmoid(sum_m sh_m Y_m(v));
//     RGBA_F32: values used as they are;
//   * output (C + T bg, 1 - T).
// Everything after the snapped integers and the FP32 1/w is FP64.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

struct OShell {
  const float* pos;        // [nv, 3]
  const float* uv;         // [nv, 2]
  const int32_t* tris;     // [nt, 3]
  int32_t nv, nt;
  const void* tex;         // [th, tw, pitch] texel values
  int32_t tw, th, fmt, degree, pitch;
  int32_t dtype;           // storage of tex: 0 float32, 1 float16, 2 float64
  // FMT_SH_U8 only: tex is the byte buffer of all SH bands, band l at
  // resolution (tw >> l*band_shift, th >> l*band_shift); decoded value =
  // vmin + (vmax - vmin) q / 255
  int32_t band_shift;
  double vmin, vmax;
};

struct OCam {
  float w2c[12];           // row-major 3x4 [R | t], world -> camera
  float fx, fy, cx, cy, znear;
  int32_t width, height;
};

// value meaning; storage is OShell::dtype except for the baked bytes of FMT_SH_U8
enum { FMT_RGBA_F32 = 0, FMT_SH_F16 = 1, FMT_SH_U8 = 2 };
enum { VF_NEAR = 1, VF_GUARD = 2 };

struct SVert {
  int64_t X = 0, Y = 0;    // snapped screen position, 1/256 px
  float invw = 0.f;        // FP32 1/w
  uint32_t q = 0;          // depth key
  int flags = 0;
};

// --- vertex transform (pinned FP32 sequence) --------------------------------
// World -> camera space.
void cam_xyz(const float* p, const OCam& c, float* out) {
  const float* m = c.w2c;
  float x = p[0], y = p[1], z = p[2];
  float xc = m[0] * x;
  xc = xc + m[1] * y;
  xc = xc + m[2] * z;
  xc = xc + m[3];
  float yc = m[4] * x;
  yc = yc + m[5] * y;
  yc = yc + m[6] * z;
  yc = yc + m[7];
  float zc = m[8] * x;
  zc = zc + m[9] * y;
  zc = zc + m[10] * z;
  zc = zc + m[11];
  out[0] = xc; out[1] = yc; out[2] = zc;
}

// Camera space (zc >= znear) -> snapped screen position, 1/w, depth key.
SVert project(float xc, float yc, float zc, const OCam& c) {
  SVert v;
  float iw = 1.0f / zc;
  float sx = c.fx * xc;
  sx = sx * iw;
  sx = sx + c.cx;
  float sy = c.fy * yc;
  sy = sy * iw;
  sy = sy + c.cy;
  float X = sx * 256.0f, Y = sy * 256.0f;
  if (!(std::fabs(X) < 8388608.0f && std::fabs(Y) < 8388608.0f)) {
    v.flags = VF_GUARD;
    return v;
  }
  v.X = (int64_t)std::nearbyint(X);
  v.Y = (int64_t)std::nearbyint(Y);
  v.invw = iw;
  float kq = c.znear * 1073741824.0f;
  float qf = iw * kq;
  v.q = (uint32_t)std::nearbyint(qf);
  return v;
}

SVert setup_vertex(const float* p, const OCam& c) {
  float pc[3];
  cam_xyz(p, c, pc);
  if (!(pc[2] >= c.znear)) {
    SVert v;
    v.flags = VF_NEAR;
    return v;
  }
  return project(pc[0], pc[1], pc[2], c);
}

std::vector<SVert> setup_all(const OShell& s, const OCam& c) {
  std::vector<SVert> v(s.nv);
  for (int i = 0; i < s.nv; ++i) v[i] = setup_vertex(s.pos + 3 * i, c);
  return v;
}

int64_t floor_div(int64_t a, int64_t b) {  // b > 0
  int64_t q = a / b;
  if ((a % b) != 0 && a < 0) --q;
  return q;
}

// Triangle prepared for rasterization: front-facing, all vertices valid.
struct Tri {
  int64_t X[3], Y[3];
  uint32_t q[3];
  bool tl[3];              // edge j (opposite vertex j) is a top or left edge
  int64_t xlo, xhi, ylo, yhi;
  double iw[3];            // 1/w per vertex
  float uv[3][2];          // texture coordinates per vertex (if the shell has UVs)
};

// orient(a, b, p) = (bx - ax)(py - ay) - (by - ay)(px - ax); for a
// front-facing triangle (orient(v0, v1, v2) < 0 in y-down screen space) the
// weights e_j = orient(v_{j+2}, v_{j+1}, p) are >= 0 inside and e_j is the
// barycentric weight of vertex j.
inline void edge_values(const Tri& t, int64_t px, int64_t py, int64_t e[3]) {
  for (int j = 0; j < 3; ++j) {
    int a = (j + 2) % 3, b = (j + 1) % 3;
    e[j] = (t.X[b] - t.X[a]) * (py - t.Y[a]) - (t.Y[b] - t.Y[a]) * (px - t.X[a]);
  }
}

inline bool covered(const Tri& t, const int64_t e[3]) {
  for (int j = 0; j < 3; ++j) {
    if (e[j] < 0) return false;
    if (e[j] == 0 && !t.tl[j]) return false;
  }
  return true;
}

// A vertex of a (possibly clipped) triangle: screen data and UV.
struct PVert {
  SVert sv;
  float uv[2];
};

// Orientation, fill rule and pixel box of three screen vertices; false if
// a vertex is off the guard band (*why = 3) or the triangle is back-facing
// or degenerate (*why = 1).
bool finish_tri(const PVert* p0, const PVert* p1, const PVert* p2, const OCam& c, Tri* t, int* why) {
  const PVert* v[3] = {p0, p1, p2};
  if ((v[0]->sv.flags | v[1]->sv.flags | v[2]->sv.flags) & VF_GUARD) { *why = 3; return false; }
  for (int j = 0; j < 3; ++j) {
    t->X[j] = v[j]->sv.X; t->Y[j] = v[j]->sv.Y; t->q[j] = v[j]->sv.q;
    t->iw[j] = v[j]->sv.invw;
    t->uv[j][0] = v[j]->uv[0]; t->uv[j][1] = v[j]->uv[1];
  }
  int64_t a2 = (t->X[1] - t->X[0]) * (t->Y[2] - t->Y[0]) -
               (t->X[2] - t->X[0]) * (t->Y[1] - t->Y[0]);
  if (a2 >= 0) { *why = 1; return false; }
  for (int j = 0; j < 3; ++j) {
    int a = (j + 2) % 3, b = (j + 1) % 3;
    // gradient of e_j: d/dpx = -(Yb - Ya), d/dpy = (Xb - Xa); interior on
    // the positive side.  Left edge: interior to the right (d/dpx > 0).
    // Top edge: horizontal with the interior below (+y is down).
    int64_t ax = -(t->Y[b] - t->Y[a]);
    int64_t by = t->X[b] - t->X[a];
    t->tl[j] = (ax > 0) || (ax == 0 && by > 0);
  }
  int64_t mnx = std::min({t->X[0], t->X[1], t->X[2]});
  int64_t mxx = std::max({t->X[0], t->X[1], t->X[2]});
  int64_t mny = std::min({t->Y[0], t->Y[1], t->Y[2]});
  int64_t mxy = std::max({t->Y[0], t->Y[1], t->Y[2]});
  // pixel centres 256 x + 128 inside [mn, mx]
  t->xlo = std::max<int64_t>(0, -floor_div(-(mnx - 128), 256));
  t->xhi = std::min<int64_t>(c.width - 1, floor_div(mxx - 128, 256));
  t->ylo = std::max<int64_t>(0, -floor_div(-(mny - 128), 256));
  t->yhi = std::min<int64_t>(c.height - 1, floor_div(mxy - 128, 256));
  *why = 0;
  return true;
}

// Rasterizable parts of mesh triangle `tri` (0, 1 or 2).  *why: 0 whole, 1
// back-facing or degenerate, 2 entirely nearer than znear, 3 off the guard
// band, 4 clipped at the near plane.
//
// Near-plane clipping (the paper's close-up views need it; it only says
// the meshes are rasterized): a triangle with one or two vertices nearer
// than znear is clipped against the plane z = znear in camera space
// (Sutherland-Hodgman, vertices in order).  The point on a crossing edge is
// computed from its (inside, outside) ends, t = (znear - z_out) / (z_in -
// z_out), x = x_out + t (x_in - x_out) (same for y and the UVs), z = znear,
// all in FP32 in this order, so two triangles sharing the edge get the same
// point; it is projected and snapped like a vertex.  The 3- or 4-gon is
// split into (P0, P1, P2) and (P0, P2, P3); each part is culled or
// rasterized under the rules above and keeps the mesh triangle's id.
int prepare_tris(const OShell& s, const std::vector<SVert>& sv, int32_t tri, const OCam& c, Tri out[2],
                 int* why) {
  const int32_t* idx = s.tris + 3 * tri;
  PVert v[3];
  int nnear = 0;
  for (int j = 0; j < 3; ++j) {
    v[j].sv = sv[idx[j]];
    v[j].uv[0] = s.uv ? s.uv[2 * idx[j]] : 0.0f;
    v[j].uv[1] = s.uv ? s.uv[2 * idx[j] + 1] : 0.0f;
    nnear += (v[j].sv.flags & VF_NEAR) ? 1 : 0;
  }
  if (nnear == 3) { *why = 2; return 0; }
  if (nnear == 0) return finish_tri(&v[0], &v[1], &v[2], c, &out[0], why) ? 1 : 0;
  float pc[3][3];
  for (int j = 0; j < 3; ++j) cam_xyz(s.pos + 3 * idx[j], c, pc[j]);
  PVert poly[4];
  int n = 0;
  for (int a = 0; a < 3; ++a) {
    const int b = (a + 1) % 3;
    const bool ina = pc[a][2] >= c.znear, inb = pc[b][2] >= c.znear;
    if (ina) poly[n++] = v[a];
    if (ina != inb) {
      const int i = ina ? a : b, o = ina ? b : a;
      float t = (c.znear - pc[o][2]) / (pc[i][2] - pc[o][2]);
      float x = pc[o][0] + t * (pc[i][0] - pc[o][0]);
      float y = pc[o][1] + t * (pc[i][1] - pc[o][1]);
      float u = v[o].uv[0] + t * (v[i].uv[0] - v[o].uv[0]);
      float w = v[o].uv[1] + t * (v[i].uv[1] - v[o].uv[1]);
      poly[n].sv = project(x, y, c.znear, c);
      poly[n].uv[0] = u;
      poly[n].uv[1] = w;
      ++n;
    }
  }
  int m = 0, w;
  if (finish_tri(&poly[0], &poly[1], &poly[2], c, &out[m], &w)) ++m;
  if (n == 4 && finish_tri(&poly[0], &poly[2], &poly[3], c, &out[m], &w)) ++m;
  *why = 4;
  return m;
}

// The part of mesh triangle `tri` used to shade fixed-point pixel centre
// (px, py): its only part, or, for a triangle clipped into two, the part
// that covers the pixel under the fill rule (the parts do not overlap), the
// first one if neither does.  False if nothing of the triangle is
// rasterizable.
bool tri_at(const OShell& s, const std::vector<SVert>& sv, int32_t tri, const OCam& c, int64_t px, int64_t py,
            Tri* t) {
  Tri parts[2];
  int why;
  const int n = prepare_tris(s, sv, tri, c, parts, &why);
  if (n == 0) return false;
  *t = parts[0];
  if (n == 2) {
    int64_t e[3];
    edge_values(parts[1], px, py, e);
    if (covered(parts[1], e)) *t = parts[1];
  }
  return true;
}

inline uint32_t depth_key(const Tri& t, const int64_t e[3]) {
  __int128 n = (__int128)e[0] * t.q[0] + (__int128)e[1] * t.q[1] + (__int128)e[2] * t.q[2];
  __int128 s = (__int128)e[0] + e[1] + e[2];
  return (uint32_t)(n / s);
}

void raster_rows(const OShell& s, const OCam& c, const std::vector<SVert>& sv, int brute,
                 int64_t y0, int64_t y1, uint64_t* keys, int32_t* cover, int64_t* stats) {
  const int64_t W = c.width;
  for (int32_t ti = 0; ti < s.nt; ++ti) {
    Tri parts[2];
    int why;
    const int np = prepare_tris(s, sv, ti, c, parts, &why);
    if (stats) stats[why] += 1;
    for (int pi = 0; pi < np; ++pi) {
    const Tri& t = parts[pi];
    int64_t xa = t.xlo, xb = t.xhi, ya = std::max(t.ylo, y0), yb = std::min(t.yhi, y1 - 1);
    if (brute) { xa = 0; xb = W - 1; ya = y0; yb = y1 - 1; }
    for (int64_t y = ya; y <= yb; ++y) {
      int64_t py = 256 * y + 128;
      for (int64_t x = xa; x <= xb; ++x) {
        int64_t px = 256 * x + 128;
        int64_t e[3];
        edge_values(t, px, py, e);
        if (!covered(t, e)) continue;
        if (cover) cover[y * W + x] += 1;
        uint64_t key = ((uint64_t)depth_key(t, e) << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)ti);
        uint64_t& slot = keys[y * W + x];
        if (key > slot) slot = key;
      }
    }
    }
  }
}

template <class F>
void parallel_rows(int64_t h, int nthreads, F f) {
  if (nthreads <= 1 || h < 2) { f(0, h, 0); return; }
  nthreads = (int)std::min<int64_t>(nthreads, h);
  std::vector<std::thread> th;
  for (int i = 0; i < nthreads; ++i) {
    int64_t a = h * i / nthreads, b = h * (i + 1) / nthreads;
    th.emplace_back([=] { f(a, b, i); });
  }
  for (auto& t : th) t.join();
}

// --- texture sampling ---------------------------------------------------------
double half_to_double(uint16_t h) {
  int s = h >> 15, e = (h >> 10) & 31, m = h & 1023;
  double v;
  if (e == 0) v = std::ldexp((double)m, -24);
  else if (e == 31) v = m ? NAN : INFINITY;
  else v = std::ldexp((double)(m | 1024), e - 25);
  return s ? -v : v;
}

inline double texel_value(const OShell& s, int64_t x, int64_t y, int ch) {
  size_t off = ((size_t)y * s.tw + (size_t)x) * s.pitch + ch;
  if (s.dtype == 0) return (double)((const float*)s.tex)[off];
  if (s.dtype == 2) return ((const double*)s.tex)[off];
  return half_to_double(((const uint16_t*)s.tex)[off]);
}

struct Footprint {
  int64_t x[2], y[2];      // clamped tap columns / rows
  double fx, fy;           // weight of column x[1] / row y[1]
};

// Bilinear footprint of UV point (u, v): texel centres at ((x+1/2)/W, (y+1/2)/H).
Footprint footprint(const OShell& s, double u, double v) {
  double X = u * s.tw - 0.5, Y = v * s.th - 0.5;
  double fx0 = std::floor(X), fy0 = std::floor(Y);
  Footprint f;
  f.fx = X - fx0;
  f.fy = Y - fy0;
  int64_t ix = (int64_t)fx0, iy = (int64_t)fy0;
  f.x[0] = std::clamp<int64_t>(ix, 0, s.tw - 1);
  f.x[1] = std::clamp<int64_t>(ix + 1, 0, s.tw - 1);
  f.y[0] = std::clamp<int64_t>(iy, 0, s.th - 1);
  f.y[1] = std::clamp<int64_t>(iy + 1, 0, s.th - 1);
  return f;
}

inline double tap_weight(const Footprint& f, int a, int b) {  // a: column tap, b: row tap
  return (a ? f.fx : 1.0 - f.fx) * (b ? f.fy : 1.0 - f.fy);
}

void sample(const OShell& s, const Footprint& f, int nch, double* out) {
  for (int ch = 0; ch < nch; ++ch) {
    double acc = 0.0;
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) acc += tap_weight(f, a, b) * texel_value(s, f.x[a], f.y[b], ch);
    out[ch] = acc;
  }
}

// --- the baked texel format (Sec. 3 "Mixed Resolutions", "Squeezing and
// Quantization", "Baking Textures") ---------------------------------------------
// SH coefficient m (band l = floor(sqrt(m))) of all four channels RGBA, one
// byte each.  Band l is its own image of (tw >> l s) x (th >> l s) texels, s =
// band_shift (s = 1 halves the resolution per band: the paper's 2048^2 base
// colour down to 256^2 for band 3).  A texel of band l holds the band's 2l+1
// coefficients as RGBA byte quadruples, padded to 4, 16, 32, 32 bytes for
// l = 0..3; bands follow each other, each starting on a 256-byte boundary.
// The decoded value is vmin + (vmax - vmin) q / 255 (the paper's rescale of
// the stored q(x) = round(255 x) / 255 to [vmin, vmax]).
struct Band {
  int64_t w, h, stride, offset;
};

Band band_layout(const OShell& s, int l) {
  static const int64_t kStride[4] = {4, 16, 32, 32};
  Band b{0, 0, 0, 0};
  for (int j = 0; j <= l; ++j) {
    if (j > 0) b.offset += (b.w * b.h * b.stride + 255) / 256 * 256;
    b.w = (int64_t)s.tw >> (j * s.band_shift);
    b.h = (int64_t)s.th >> (j * s.band_shift);
    b.stride = kStride[j];
  }
  return b;
}

Footprint footprint_wh(int64_t w, int64_t h, double u, double v) {
  OShell t{};
  t.tw = (int32_t)w;
  t.th = (int32_t)h;
  return footprint(t, u, v);
}

// Bilinear sample at UV (u, v) of coefficient m of every channel, decoded.
void sample_baked(const OShell& s, int m, double u, double v, double out[4]) {
  const int l = (int)std::floor(std::sqrt((double)m) + 1e-9);
  const int j = m - l * l;
  const Band b = band_layout(s, l);
  const Footprint f = footprint_wh(b.w, b.h, u, v);
  const uint8_t* base = (const uint8_t*)s.tex + b.offset;
  for (int ch = 0; ch < 4; ++ch) {
    double acc = 0.0;
    for (int yb = 0; yb < 2; ++yb)
      for (int xa = 0; xa < 2; ++xa) {
        const uint8_t q = base[(f.y[yb] * b.w + f.x[xa]) * b.stride + 4 * j + ch];
        acc += tap_weight(f, xa, yb) * (s.vmin + (s.vmax - s.vmin) * (double)q / 255.0);
      }
    out[ch] = acc;
  }
}

// --- real spherical harmonics, l <= 3, orthonormal on the unit sphere ---------
// Real forms of the complex Y_l^m without the Condon-Shortley sign; the l = 1
// band is proportional to (y, z, x).  Index l^2 + l + m.
void sh_basis(int deg, const double v[3], double* Y) {
  const double pi = 3.14159265358979323846;
  const double x = v[0], y = v[1], z = v[2];
  Y[0] = 0.5 * std::sqrt(1.0 / pi);
  if (deg < 1) return;
  const double c1 = std::sqrt(3.0 / (4.0 * pi));
  Y[1] = c1 * y;
  Y[2] = c1 * z;
  Y[3] = c1 * x;
  if (deg < 2) return;
  const double c2a = 0.5 * std::sqrt(15.0 / pi);
  const double c2b = 0.25 * std::sqrt(5.0 / pi);
  const double c2c = 0.25 * std::sqrt(15.0 / pi);
  Y[4] = c2a * x * y;
  Y[5] = c2a * y * z;
  Y[6] = c2b * (3.0 * z * z - 1.0);
  Y[7] = c2a * x * z;
  Y[8] = c2c * (x * x - y * y);
  if (deg < 3) return;
  const double c3a = 0.25 * std::sqrt(35.0 / (2.0 * pi));
  const double c3b = 0.5 * std::sqrt(105.0 / pi);
  const double c3c = 0.25 * std::sqrt(21.0 / (2.0 * pi));
  const double c3d = 0.25 * std::sqrt(7.0 / pi);
  const double c3e = 0.25 * std::sqrt(105.0 / pi);
  Y[9] = c3a * y * (3.0 * x * x - y * y);
  Y[10] = c3b * x * y * z;
  Y[11] = c3c * y * (5.0 * z * z - 1.0);
  Y[12] = c3d * z * (5.0 * z * z - 3.0);
  Y[13] = c3c * x * (5.0 * z * z - 1.0);
  Y[14] = c3e * z * (x * x - y * y);
  Y[15] = c3a * x * (x * x - 3.0 * y * y);
}

inline double sigmoid(double x) { return 1.0 / (1.0 + std::exp(-x)); }

// Unit world-space direction of the ray through the centre of pixel (x, y).
void ray_dir(const OCam& c, int64_t x, int64_t y, double v[3]) {
  double dc[3] = {((double)x + 0.5 - c.cx) / c.fx, ((double)y + 0.5 - c.cy) / c.fy, 1.0};
  double n = 0.0;
  for (int i = 0; i < 3; ++i) {
    v[i] = c.w2c[0 + i] * dc[0] + c.w2c[4 + i] * dc[1] + c.w2c[8 + i] * dc[2];
    n += v[i] * v[i];
  }
  n = std::sqrt(n);
  for (int i = 0; i < 3; ++i) v[i] /= n;
}

// Perspective-correct UV at pixel centre (px, py) (1/256 px fixed point).
void interp_uv(const Tri& t, int64_t px, int64_t py, double out[2]) {
  int64_t e[3];
  edge_values(t, px, py, e);
  double w[3], sw = 0.0;
  for (int j = 0; j < 3; ++j) { w[j] = (double)e[j] * t.iw[j]; sw += w[j]; }
  out[0] = out[1] = 0.0;
  for (int j = 0; j < 3; ++j) {
    out[0] += w[j] / sw * t.uv[j][0];
    out[1] += w[j] / sw * t.uv[j][1];
  }
}

int num_values(const OShell& s) {
  return s.fmt == FMT_RGBA_F32 ? 4 : 1 + 3 * (s.degree + 1) * (s.degree + 1);
}

// One fragment: (pixel, shell, triangle) -> rgb, alpha, plus what the adjoint needs.
struct Frag {
  double rgb[3], alpha;    // alpha = alpha_raw * atten
  double alpha_raw;        // opacity from the texels
  double atten;            // transparency attenuation (1 unless enabled)
  Footprint fp;
  double val[64];          // interpolated texel values
  double uv[2];            // perspective-correct texture coordinates at the pixel
  double normal[3];        // unit geometric normal of the face, (p1 - p0) x (p2 - p0)
};

// Sec. 3 "Transparency Attenuation": alpha_w = 2 sigmoid(10 |v . n|) - 1,
// with v the unit ray direction and n the unit normal of the hit face (the
// flat geometric normal of the baked triangle).
double attenuation(const OShell& s, const int32_t* idx, const double v[3]) {
  double p[3][3];
  for (int j = 0; j < 3; ++j)
    for (int d = 0; d < 3; ++d) p[j][d] = s.pos[3 * idx[j] + d];
  const double a[3] = {p[1][0] - p[0][0], p[1][1] - p[0][1], p[1][2] - p[0][2]};
  const double b[3] = {p[2][0] - p[0][0], p[2][1] - p[0][1], p[2][2] - p[0][2]};
  const double n[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
  const double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  const double vn = std::fabs(n[0] * v[0] + n[1] * v[1] + n[2] * v[2]) / len;
  return 2.0 / (1.0 + std::exp(-10.0 * vn)) - 1.0;
}

enum { OFLAG_ALPHA_ATTEN = 2 };

bool shade_fragment(const OShell& s, const OCam& c, const std::vector<SVert>& sv, int32_t tri,
                    int64_t x, int64_t y, const double* Y, const double* v, int flags, Frag* f) {
  const int32_t* idx = s.tris + 3 * tri;
  Tri t;
  if (!tri_at(s, sv, tri, c, 256 * x + 128, 256 * y + 128, &t)) return false;
  double uv[2];
  interp_uv(t, 256 * x + 128, 256 * y + 128, uv);
  f->uv[0] = uv[0];
  f->uv[1] = uv[1];
  {
    double p[3][3];
    for (int j = 0; j < 3; ++j)
      for (int d = 0; d < 3; ++d) p[j][d] = s.pos[3 * idx[j] + d];
    const double a[3] = {p[1][0] - p[0][0], p[1][1] - p[0][1], p[1][2] - p[0][2]};
    const double b[3] = {p[2][0] - p[0][0], p[2][1] - p[0][1], p[2][2] - p[0][2]};
    const double n[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    const double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (int d = 0; d < 3; ++d) f->normal[d] = n[d] / len;
  }
  if (s.fmt == FMT_SH_U8) {
    // RGBA all view-dependent: channel c = sigmoid(sum_m sh_{m,c} Y_m(v))
    const int nb = (s.degree + 1) * (s.degree + 1);
    double z[4] = {0, 0, 0, 0};
    for (int m = 0; m < nb; ++m) {
      double val[4];
      sample_baked(s, m, uv[0], uv[1], val);
      for (int ch = 0; ch < 4; ++ch) z[ch] += val[ch] * Y[m];
    }
    for (int ch = 0; ch < 3; ++ch) f->rgb[ch] = sigmoid(z[ch]);
    f->alpha_raw = sigmoid(z[3]);
    f->atten = (flags & OFLAG_ALPHA_ATTEN) ? attenuation(s, idx, v) : 1.0;
    f->alpha = f->alpha_raw * f->atten;
    return true;
  }
  f->fp = footprint(s, uv[0], uv[1]);
  int nv = num_values(s);
  sample(s, f->fp, nv, f->val);
  if (s.fmt == FMT_RGBA_F32) {
    for (int ch = 0; ch < 3; ++ch) f->rgb[ch] = f->val[ch];
    f->alpha = f->val[3];
  } else {
    int nb = (s.degree + 1) * (s.degree + 1);
    f->alpha = sigmoid(f->val[0]);
    for (int ch = 0; ch < 3; ++ch) {
      double z = 0.0;
      for (int m = 0; m < nb; ++m) z += f->val[1 + 3 * m + ch] * Y[m];
      f->rgb[ch] = sigmoid(z);
    }
  }
  f->alpha_raw = f->alpha;
  f->atten = (flags & OFLAG_ALPHA_ATTEN) ? attenuation(s, idx, v) : 1.0;
  f->alpha = f->alpha_raw * f->atten;
  return true;
}

}  // namespace

extern "C" {

int oracle_setup_vertices(const float* pos, int32_t nv, const OCam* cam, int64_t* xy, float* invw,
                          uint32_t* q, int32_t* flags) {
  for (int i = 0; i < nv; ++i) {
    SVert v = setup_vertex(pos + 3 * i, *cam);
    xy[2 * i] = v.X;
    xy[2 * i + 1] = v.Y;
    invw[i] = v.invw;
    q[i] = v.q;
    flags[i] = v.flags;
  }
  return 0;
}

// keys: [H*W] zero-initialised by the caller; max of (K << 32 | ~tri).
// cover (optional): [H*W] zero-initialised, += 1 per covering front triangle.
// stats (optional): [5] = {front, back or zero-area, behind the near plane,
// guard band, clipped at the near plane}.
int oracle_raster(const float* pos, int32_t nv, const int32_t* tris, int32_t nt, const OCam* cam,
                  int32_t brute, int32_t nthreads, uint64_t* keys, int32_t* cover, int64_t* stats) {
  OShell s{};
  s.pos = pos; s.nv = nv; s.tris = tris; s.nt = nt;
  std::vector<SVert> sv = setup_all(s, *cam);
  if (stats) std::memset(stats, 0, 5 * sizeof(int64_t));
  int nth = std::max(1, nthreads);
  std::vector<int64_t> st(5 * nth, 0);
  parallel_rows(cam->height, nth, [&](int64_t y0, int64_t y1, int i) {
    raster_rows(s, *cam, sv, brute, y0, y1, keys, cover, st.data() + 5 * i);
  });
  if (stats) {
    // every band sees every triangle once: report the counts of band 0
    for (int j = 0; j < 5; ++j) stats[j] = st[j];
  }
  return 0;
}

// Shade + composite every pixel from per-shell hits [k, H, W] (-1 = miss).
// out: [H, W, 4] = (C + T bg, 1 - T).  stats (optional): [k] fragments per shell.
// layers (optional): [k, H, W, 12] per-shell buffers (Figs. S1/S3): unit
// face normal (3), uv (2), opacity, blending weight T_i alpha_i, rgb (3), 0,
// 0; all zero where the shell has no fragment.
int oracle_shade(const OShell* shells, int32_t k, const OCam* cam, const double* bg,
                 const int32_t* hits, double* out, int32_t nthreads, int64_t* frags, int32_t flags,
                 double* layers) {
  const int64_t W = cam->width, H = cam->height;
  std::vector<std::vector<SVert>> sv(k);
  int maxdeg = 0;
  for (int i = 0; i < k; ++i) {
    sv[i] = setup_all(shells[i], *cam);
    if (shells[i].fmt != FMT_RGBA_F32) maxdeg = std::max(maxdeg, (int)shells[i].degree);
  }
  int nth = std::max(1, nthreads);
  std::vector<int64_t> cnt((size_t)nth * k, 0);
  parallel_rows(H, nth, [&](int64_t y0, int64_t y1, int ti) {
    for (int64_t y = y0; y < y1; ++y)
      for (int64_t x = 0; x < W; ++x) {
        double v[3], Y[16];
        ray_dir(*cam, x, y, v);
        sh_basis(maxdeg, v, Y);
        double C[3] = {0, 0, 0}, T = 1.0;
        for (int i = 0; i < k; ++i) {
          int32_t h = hits[(size_t)i * H * W + y * W + x];
          if (h < 0) continue;
          Frag f;
          if (!shade_fragment(shells[i], *cam, sv[i], h, x, y, Y, v, flags, &f)) continue;
          cnt[(size_t)ti * k + i] += 1;
          if (layers) {
            double* L = layers + 12 * ((size_t)i * H * W + y * W + x);
            for (int d = 0; d < 3; ++d) L[d] = f.normal[d];
            L[3] = f.uv[0];
            L[4] = f.uv[1];
            L[5] = f.alpha;
            L[6] = T * f.alpha;
            for (int ch = 0; ch < 3; ++ch) L[7 + ch] = f.rgb[ch];
          }
          for (int ch = 0; ch < 3; ++ch) C[ch] += T * f.alpha * f.rgb[ch];
          T *= (1.0 - f.alpha);
        }
        double* o = out + 4 * (y * W + x);
        for (int ch = 0; ch < 3; ++ch) o[ch] = C[ch] + T * bg[ch];
        o[3] = 1.0 - T;
      }
  });
  if (frags)
    for (int i = 0; i < k; ++i) {
      frags[i] = 0;
      for (int t = 0; t < nth; ++t) frags[i] += cnt[(size_t)t * k + i];
    }
  return 0;
}

// Adjoint of oracle_shade w.r.t. the texel values.  grad_rgb: [H, W, 3] =
// dL/d(output rgb).  grad_tex[i]: [th, tw, pitch] FP64, accumulated into
// (NULL: shell i's gradient is not wanted; its scales are then not
// written either).
//
// Optional error scales (abs_tex, reach_tex non-NULL, same layout as
// grad_tex), a yardstick for comparing gradients, not part of the method.
// For every texel value and every (fragment, tap) that reaches it, let M be
// the SAME product as the gradient term with every factor replaced by its
// absolute value and every difference by the sum of the absolute values of
// its terms (c_i . g - A_{i+1} . g -> |c_i| . |g| + |A_{i+1}| . |g|, the
// colour seen behind counted with |bg|), without the tap weight.
// abs_tex accumulates |w| M and reach_tex accumulates M.  A floating-point
// evaluation of the adjoint in any order errs per texel value by a small
// multiple of machine epsilon times the first sum, also where terms cancel,
// plus the error of its tap weights times the second.  gmag [H, W, 3]
// (NULL = |grad_rgb|) gives the size of each pixel's output gradient before
// cancellation (e.g. (|C| + |target|) 2 / n for the L2 loss).  With the
// transparency attenuation on, aw_err is an absolute error of each alpha_w
// that the scales allow for: every term of a fragment's adjoint scales with
// its alpha_w, and the transmittances with the (1 - alpha_j) of the pixel's
// other fragments, so the fragment's M is multiplied by
// 1 + aw_err (1 / alpha_w + sum_j 1 / (1 - alpha_j)).  weight_err: where
// a fragment's texel coordinate lies within weight_err of a texel centre
// line, an evaluation in lower precision may place its footprint one texel
// over, giving the texel beyond a tap weight of at most weight_err: M is
// then also added to reach_tex at those texels.  ysc_tex (optional, like
// abs_tex): for the SH coefficient values, the sum of |w| M with the SH
// basis value left out of M -- the scale of an absolute error in the basis
// values (a basis value near zero is a difference of terms of the ray
// direction, so its error does not shrink with it).
int oracle_backward(const OShell* shells, int32_t k, const OCam* cam, const double* bg,
                    const int32_t* hits, const double* grad_rgb, double* const* grad_tex, int32_t flags,
                    const double* gmag, double* const* abs_tex, double* const* reach_tex, double aw_err,
                    double weight_err, double* const* ysc_tex) {
  // the baked bytes are a deployment format: no gradient (the paper fits
  // continuous textures and quantises when baking)
  for (int i = 0; i < k; ++i)
    if (shells[i].fmt == FMT_SH_U8) return -3;
  const int64_t W = cam->width, H = cam->height;
  std::vector<std::vector<SVert>> sv(k);
  int maxdeg = 0;
  for (int i = 0; i < k; ++i) {
    sv[i] = setup_all(shells[i], *cam);
    if (shells[i].fmt != FMT_RGBA_F32) maxdeg = std::max(maxdeg, (int)shells[i].degree);
  }
  std::vector<Frag> fr(k);
  std::vector<char> hit(k);
  std::vector<double> Tin(k);
  for (int64_t y = 0; y < H; ++y)
    for (int64_t x = 0; x < W; ++x) {
      const double* g = grad_rgb + 3 * (y * W + x);
      // a pixel with a zero output gradient (and error scale) adds nothing
      if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0 &&
          (!gmag || (gmag[3 * (y * W + x)] == 0.0 && gmag[3 * (y * W + x) + 1] == 0.0 &&
                     gmag[3 * (y * W + x) + 2] == 0.0)))
        continue;
      double v[3], Y[16];
      ray_dir(*cam, x, y, v);
      sh_basis(maxdeg, v, Y);
      double T = 1.0, sens = 0.0;   // sens: error scale only
      for (int i = 0; i < k; ++i) {
        int32_t h = hits[(size_t)i * H * W + y * W + x];
        hit[i] = h >= 0 && shade_fragment(shells[i], *cam, sv[i], h, x, y, Y, v, flags, &fr[i]);
        Tin[i] = T;
        if (hit[i]) {
          T *= (1.0 - fr[i].alpha);
          sens += 1.0 / std::max(1.0 - fr[i].alpha, 1e-300);
        }
      }
      // back to front: A = colour seen behind shell i (bg behind the last)
      double A[3] = {bg[0], bg[1], bg[2]};
      double gm[3], Am[3];   // error scale only
      for (int ch = 0; ch < 3; ++ch) {
        gm[ch] = gmag ? gmag[3 * (y * W + x) + ch] : std::fabs(g[ch]);
        Am[ch] = std::fabs(bg[ch]);
      }
      for (int i = k - 1; i >= 0; --i) {
        if (!hit[i]) continue;
        const Frag& f = fr[i];
        const OShell& s = shells[i];
        double gc[3], ga = 0.0, gcm[3], gam = 0.0;
        for (int ch = 0; ch < 3; ++ch) {
          gc[ch] = Tin[i] * f.alpha * g[ch];                 // dL/dc_i
          ga += Tin[i] * (f.rgb[ch] - A[ch]) * g[ch];         // dL/dalpha_i
          gcm[ch] = Tin[i] * f.alpha * gm[ch];
          gam += Tin[i] * (std::fabs(f.rgb[ch]) + Am[ch]) * gm[ch];
        }
        for (int ch = 0; ch < 3; ++ch) {
          A[ch] = f.alpha * f.rgb[ch] + (1.0 - f.alpha) * A[ch];
          Am[ch] = f.alpha * std::fabs(f.rgb[ch]) + (1.0 - f.alpha) * Am[ch];
        }
        int nv = num_values(s);
        double dval[64], dmag[64], ymag[64];
        // alpha = alpha_raw * atten, atten independent of the texels
        if (s.fmt == FMT_RGBA_F32) {
          dval[0] = gc[0]; dval[1] = gc[1]; dval[2] = gc[2]; dval[3] = ga * f.atten;
          dmag[0] = gcm[0]; dmag[1] = gcm[1]; dmag[2] = gcm[2]; dmag[3] = gam * f.atten;
          for (int ch = 0; ch < 4; ++ch) ymag[ch] = 0.0;
        } else {
          int nb = (s.degree + 1) * (s.degree + 1);
          const double sa = f.alpha_raw * (1.0 - f.alpha_raw);
          dval[0] = ga * f.atten * sa;
          dmag[0] = gam * f.atten * sa;
          ymag[0] = 0.0;
          for (int ch = 0; ch < 3; ++ch) {
            const double sc = f.rgb[ch] * (1.0 - f.rgb[ch]);
            double dz = gc[ch] * sc;
            for (int m = 0; m < nb; ++m) {
              dval[1 + 3 * m + ch] = dz * Y[m];
              dmag[1 + 3 * m + ch] = gcm[ch] * sc * std::fabs(Y[m]);
              ymag[1 + 3 * m + ch] = gcm[ch] * sc;
            }
          }
        }
        if ((flags & OFLAG_ALPHA_ATTEN) && aw_err > 0.0) {
          const double grow = 1.0 + aw_err * (1.0 / std::max(f.atten, 1e-300) + sens);
          for (int ch = 0; ch < nv; ++ch) {
            dmag[ch] *= grow;
            ymag[ch] *= grow;
          }
        }
        for (int b = 0; b < 2; ++b)
          for (int a = 0; a < 2; ++a) {
            double w = tap_weight(f.fp, a, b);
            const size_t off = ((size_t)f.fp.y[b] * s.tw + (size_t)f.fp.x[a]) * s.pitch;
            if (!grad_tex[i]) continue;   // shell not asked for
            double* gt = grad_tex[i] + off;
            for (int ch = 0; ch < nv; ++ch) gt[ch] += w * dval[ch];
            if (abs_tex) {
              double* at = abs_tex[i] + off;
              for (int ch = 0; ch < nv; ++ch) at[ch] += std::fabs(w) * dmag[ch];
            }
            if (reach_tex) {
              double* rt = reach_tex[i] + off;
              for (int ch = 0; ch < nv; ++ch) rt[ch] += dmag[ch];
            }
            if (ysc_tex) {
              double* yt = ysc_tex[i] + off;
              for (int ch = 0; ch < nv; ++ch) yt[ch] += std::fabs(w) * ymag[ch];
            }
          }
        if (reach_tex && grad_tex[i] && weight_err > 0.0) {
          const double X = f.uv[0] * s.tw - 0.5, Yc = f.uv[1] * s.th - 0.5;
          const int64_t ix = (int64_t)std::floor(X), iy = (int64_t)std::floor(Yc);
          const double ex = X - (double)ix, ey = Yc - (double)iy;
          int64_t xs[3], ys[3];
          int nx = 0, ny = 0;
          xs[nx++] = ix;
          xs[nx++] = ix + 1;
          if (ex < weight_err) xs[nx++] = ix - 1;
          else if (ex > 1.0 - weight_err) xs[nx++] = ix + 2;
          ys[ny++] = iy;
          ys[ny++] = iy + 1;
          if (ey < weight_err) ys[ny++] = iy - 1;
          else if (ey > 1.0 - weight_err) ys[ny++] = iy + 2;
          for (int b = 0; b < ny; ++b)
            for (int a = 0; a < nx; ++a) {
              if (a < 2 && b < 2) continue;   // the footprint's own taps, added above
              const int64_t cx = std::clamp<int64_t>(xs[a], 0, s.tw - 1), cy = std::clamp<int64_t>(ys[b], 0, s.th - 1);
              double* rt = reach_tex[i] + ((size_t)cy * s.tw + (size_t)cx) * s.pitch;
              for (int ch = 0; ch < nv; ++ch) rt[ch] += dmag[ch];
            }
        }
      }
    }
  return 0;
}

// Number of distinct texels touched by the bilinear footprints of all
// fragments of each shell (the D of the algorithmic-bytes count).
int oracle_footprint_texels(const OShell* shells, int32_t k, const OCam* cam, const int32_t* hits,
                            int64_t* distinct) {
  const int64_t W = cam->width, H = cam->height;
  for (int i = 0; i < k; ++i) {
    const OShell& s = shells[i];
    std::vector<SVert> sv = setup_all(s, *cam);
    std::vector<uint8_t> mark((size_t)s.tw * s.th, 0);
    for (int64_t y = 0; y < H; ++y)
      for (int64_t x = 0; x < W; ++x) {
        int32_t h = hits[(size_t)i * H * W + y * W + x];
        if (h < 0) continue;
        Tri t;
        if (!tri_at(s, sv, h, *cam, 256 * x + 128, 256 * y + 128, &t)) continue;
        double uv[2];
        interp_uv(t, 256 * x + 128, 256 * y + 128, uv);
        Footprint f = footprint(s, uv[0], uv[1]);
        for (int b = 0; b < 2; ++b)
          for (int a = 0; a < 2; ++a) mark[(size_t)f.y[b] * s.tw + f.x[a]] = 1;
      }
    int64_t n = 0;
    for (uint8_t m : mark) n += m;
    distinct[i] = n;
  }
  return 0;
}

// Baked shells: distinct texels per band (distinct[4 i + l]) touched by the
// bilinear footprints of every fragment, each band at its own resolution.
int oracle_footprint_texels_baked(const OShell* shells, int32_t k, const OCam* cam, const int32_t* hits,
                                  int64_t* distinct) {
  const int64_t W = cam->width, H = cam->height;
  for (int i = 0; i < k; ++i) {
    const OShell& s = shells[i];
    for (int l = 0; l < 4; ++l) distinct[4 * i + l] = 0;
    if (s.fmt != FMT_SH_U8) continue;
    std::vector<SVert> sv = setup_all(s, *cam);
    for (int l = 0; l <= s.degree; ++l) {
      const Band b = band_layout(s, l);
      std::vector<uint8_t> mark((size_t)(b.w * b.h), 0);
      for (int64_t y = 0; y < H; ++y)
        for (int64_t x = 0; x < W; ++x) {
          int32_t h = hits[(size_t)i * H * W + y * W + x];
          if (h < 0) continue;
          Tri t;
          if (!tri_at(s, sv, h, *cam, 256 * x + 128, 256 * y + 128, &t)) continue;
          double uv[2];
          interp_uv(t, 256 * x + 128, 256 * y + 128, uv);
          const Footprint f = footprint_wh(b.w, b.h, uv[0], uv[1]);
          for (int yb = 0; yb < 2; ++yb)
            for (int xa = 0; xa < 2; ++xa) mark[(size_t)(f.y[yb] * b.w + f.x[xa])] = 1;
        }
      int64_t n = 0;
      for (uint8_t m : mark) n += m;
      distinct[4 * i + l] = n;
    }
  }
  return 0;
}

// --- single-step entry points for the pins --------------------------------------
int oracle_sh_basis(int32_t deg, const double* v, double* Y) {
  sh_basis(deg, v, Y);
  return 0;
}

// Bilinear sample of all `nch` raw values of a texture at UV (u, v).
int oracle_sample(const void* tex, int32_t dtype, int32_t tw, int32_t th, int32_t pitch, int32_t nch,
                  double u, double v, double* out) {
  OShell s{};
  s.tex = tex; s.dtype = dtype; s.tw = tw; s.th = th; s.pitch = pitch;
  Footprint f = footprint(s, u, v);
  sample(s, f, nch, out);
  return 0;
}

// Baked format: bilinear sample of coefficient m (all four channels, decoded)
// at UV (u, v).
int oracle_sample_baked(const uint8_t* tex, int32_t tw, int32_t th, int32_t degree, int32_t band_shift,
                        double vmin, double vmax, int32_t m, double u, double v, double* out) {
  if (m < 0 || m >= (degree + 1) * (degree + 1)) return -1;
  OShell s{};
  s.tex = tex; s.tw = tw; s.th = th; s.degree = degree; s.fmt = FMT_SH_U8;
  s.band_shift = band_shift; s.vmin = vmin; s.vmax = vmax;
  sample_baked(s, m, u, v, out);
  return 0;
}

// Perspective-correct UV of a (front-facing) triangle with snapped vertices
// X, Y (1/256 px), per-vertex 1/w and UVs, at fixed-point point (px, py).
int oracle_interp_uv(const int64_t* X, const int64_t* Y, const double* invw, const float* uv,
                     int64_t px, int64_t py, double* out) {
  Tri t{};
  for (int j = 0; j < 3; ++j) {
    t.X[j] = X[j]; t.Y[j] = Y[j]; t.iw[j] = invw[j];
    t.uv[j][0] = uv[2 * j]; t.uv[j][1] = uv[2 * j + 1];
  }
  interp_uv(t, px, py, out);
  return 0;
}

// Unit ray direction through pixel (x, y).
int oracle_ray_dir(const OCam* cam, int32_t x, int32_t y, double* v) {
  ray_dir(*cam, x, y, v);
  return 0;
}

}  // extern "C"
