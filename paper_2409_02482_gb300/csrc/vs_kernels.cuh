// Device code of the k-shell renderer (sm_103a): the phases as device
// functions and the kernel templates built from them -- per-phase kernels
// for the plain per-view path and the persistent multi-item kernel.  The
// shading kernels are instantiated once per texel class, each in its own
// translation unit (vs_tc_*.cu); vs_kernels.cu holds the rest.
//
// Phases of one (object, view) item -- the hot path of the paper's baked
// real-time renderer (Sec. 3 "Baking Textures": rasterize every mesh in a
// fixed order and blend in the frame buffer) and of its texture fitting
// (Sec. 3 "Texturing Meshes"):
//   SETUP  clear the per-shell visibility words; transform + snap vertices
//   RASTER per triangle: cull, integer edge functions, exact depth key,
//          64-bit max-reduction (key << 32 | ~triangle) per (shell, pixel) --
//          the nearest hit of each shell, ties to the lower triangle
//          (Fig. 3c); each warp walks the pixels of its triangles' boxes
//          together, larger boxes one triangle at a time
//   SHADE  per warp of 32 pixels: compact the hits into a fragment list,
//          shade it 32 fragments at a time (perspective-correct UV, bilinear
//          fetch at texel centres (Fig. 5), SH decode with the ray
//          direction), composite each pixel front to back (Eq. 6 with
//          Eq. 1's transmittance) and, for the adjoint, scatter the texel
//          gradients 32 fragments at a time.

#pragma once

#include <cuda_runtime.h>

#include "vs_device.cuh"
#include "vs_kernels.h"

#ifndef VS_BWD_BLOCKS
#define VS_BWD_BLOCKS 3   // resident 256-thread blocks per SM for kernels with the adjoint
#endif
#ifndef VS_FWD_BLOCKS
#define VS_FWD_BLOCKS 3   // ... and for forward-only kernels
#endif
#ifndef VS_PERS_BWD_BLOCKS
#define VS_PERS_BWD_BLOCKS 4   // resident blocks per SM of the persistent kernel with the adjoint (pers_threads(true) each)
#endif
#ifndef VS_PERS_FWD_BLOCKS
#define VS_PERS_FWD_BLOCKS 3   // ... and of the forward-only persistent kernel
#endif

namespace vsd {

// ----------------------------------------------------------------------------
// SETUP
// ----------------------------------------------------------------------------
// One warp per unit.
static __device__ void unit_setup(const DItem& it, const DShell* sh, int u) {
  if (u < it.clear_units) {
    const size_t total = (size_t)it.k * it.cam.W * it.cam.H;
    const size_t beg = (size_t)u * kClearPerUnit;
    const size_t end = min(total, beg + (size_t)kClearPerUnit);
    uint4* p = reinterpret_cast<uint4*>(it.vis + beg);
    const size_t n2 = (end - beg) >> 1;
    for (size_t i = threadIdx.x & 31; i < n2; i += 32) clear_vis2(p + i);
    if (((end - beg) & 1) && (threadIdx.x & 31) == 0) it.vis[end - 1] = 0ull;
    return;
  }
  u -= it.clear_units;
  int i = 0;
  while (i + 1 < it.k && u >= it.setup_pre[i + 1]) ++i;
  const DShell& s = sh[i];
  const int v0 = (u - it.setup_pre[i]) * kSetupPerUnit;
  const int v1 = min(v0 + kSetupPerUnit, s.nv);
  for (int v = v0 + (threadIdx.x & 31); v < v1; v += 32) s.vsetup[v] = setup_vertex(s.pos + 3 * (size_t)v, it.cam);
}

// ----------------------------------------------------------------------------
// RASTER
// ----------------------------------------------------------------------------
// Loads triangle t of shell s; 0 = front-facing and rasterizable, 1..3 =
// culled (back/zero-area, behind the near plane, guard band), 4 = index out
// of range, 5 = to be clipped at the near plane.
__device__ __forceinline__ int load_tri(const DShell& s, const DCam& c, int t, Tri& T, int idx[3]) {
  const int* ip = s.tris + 3 * (size_t)t;
  idx[0] = __ldg(ip);
  idx[1] = __ldg(ip + 1);
  idx[2] = __ldg(ip + 2);
  if ((unsigned)idx[0] >= (unsigned)s.nv || (unsigned)idx[1] >= (unsigned)s.nv || (unsigned)idx[2] >= (unsigned)s.nv)
    return 4;
  return make_tri(__ldcg(s.vsetup + idx[0]), __ldcg(s.vsetup + idx[1]), __ldcg(s.vsetup + idx[2]), c.W, c.H, T);
}

__device__ __forceinline__ void raster_pixel(const Tri& T, int t, int x, int y, int W, unsigned long long* vis) {
  long long e[3];
  edge_values(T, 256 * x + 128, 256 * y + 128, e);
  if (covered(T, e)) red_max_vis(vis + (size_t)y * W + x, vis_key(depth_key(T, e), t));
}

// The parts of triangle t clipped at the near plane, rasterized by the whole
// warp (each lane strides over the parts' screen boxes).  Rare: out of line.
static __device__ __forceinline__ void raster_clipped(const DShell& s, const DCam& c, int t, unsigned long long* vis) {
  const int* ip = s.tris + 3 * (size_t)t;
  const int idx[3] = {__ldg(ip), __ldg(ip + 1), __ldg(ip + 2)};   // checked in range by load_tri
  Tri part[2];
  float2 puv[2][3];
  const int np = clip_tri(s.pos, nullptr, c, idx, part, puv);
  const int lane = threadIdx.x & 31;
  for (int k = 0; k < np; ++k) {
    const int bw = part[k].xhi - part[k].xlo + 1, bh = part[k].yhi - part[k].ylo + 1;
    const int npq = bw > 0 && bh > 0 ? bw * bh : 0;
    for (int p = lane; p < npq; p += 32) {
      const int yy = p / bw;
      raster_pixel(part[k], t, part[k].xlo + (p - yy * bw), part[k].ylo + yy, c.W, vis);
    }
  }
}

// Triangle record shared by the lanes of a warp during the raster walk.
// Small boxes (<= kSmallMaxPixels pixel centres) keep every edge function
// value within +-2^30, so the walk runs in 32-bit integers: e_j(dx, dy) =
// c_j + gx_j dx + gy_j dy for pixel (xlo + dx, ylo + dy).
struct TriS {
  int c[3], gx[3], gy[3];
  unsigned q[3];
  int tl_bw;           // bits 0-2: top-left edges; bits 8+: box width
  float rbw;           // 1 / box width
  float rS;            // 1 / S, S = sum of the edge values = twice the area
  int t;
};
struct TriPos {        // box origin of a record
  int xlo, ylo;
};

// floor(sum_j e_j q_j / S) for the 32-bit edge values of a small box; same
// estimate-and-correct scheme as depth_key_r.
__device__ __forceinline__ unsigned depth_key32(const unsigned q[3], const int e[3], int S, float rS) {
  const unsigned long long N = (unsigned long long)(unsigned)e[0] * q[0] +
                               (unsigned long long)(unsigned)e[1] * q[1] +
                               (unsigned long long)(unsigned)e[2] * q[2];
  const float est = fmaf((float)e[0], (float)q[0], fmaf((float)e[1], (float)q[1], (float)e[2] * (float)q[2])) * rS;
  const unsigned qmin = min(q[0], min(q[1], q[2])), qmax = max(q[0], max(q[1], q[2]));
  unsigned Q = (unsigned)fminf(fmaxf(est, (float)qmin), (float)qmax);
  Q = min(max(Q, qmin), qmax);
  long long R = (long long)(N - (unsigned long long)Q * (unsigned)S);
  Q = (unsigned)((long long)Q + (long long)floorf((float)R * rS));
  R = (long long)(N - (unsigned long long)Q * (unsigned)S);
#pragma unroll 1
  for (int i = 0; i < 4 && R < 0; ++i) { --Q; R += S; }
#pragma unroll 1
  for (int i = 0; i < 4 && R >= S; ++i) { ++Q; R -= S; }
  return Q;
}

// Per-lane triangle counts of a raster unit, two 16-bit fields per word (a
// lane sees one triangle per round and a unit has at most 2048 / 32 = 64
// rounds, so no field overflows): fb = front | back << 16, ng = near plane |
// guard band << 16, lc = large box | clipped << 16, plus an error bit.
struct RasterCounts {
  unsigned fb, ng, lc, bad;
};

// One round of a raster unit: 32 triangles t0 + lane of one shell.  Each
// lane sets up one triangle; then the warp walks all (triangle, box pixel)
// pairs of the 32 triangles together: window by window, a warp-wide OR of
// the triangles' start bits tells every lane which triangle owns its pair,
// so lanes do not idle on small or culled boxes.  Larger boxes are
// rasterized by the whole warp, one triangle at a time.
template <bool FULL>
__device__ __forceinline__ void raster_round(const DItem& it, const DShell& s, int t0, unsigned long long* vis,
                                             char* smem, RasterCounts& rc) {
  TriS* s_tri = reinterpret_cast<TriS*>(smem);
  TriPos* s_pos = reinterpret_cast<TriPos*>(smem + sizeof(TriS) * 32);
  int* s_start = reinterpret_cast<int*>(smem + (sizeof(TriS) + sizeof(TriPos)) * 32);
  const unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31, wbase = 0;
  const int t = t0 + lane;
  const int W = it.cam.W;
  unsigned front = 0, back = 0, nearc = 0, guard = 0, large = 0, bad = 0, clip = 0;
  int npx = 0;
  TriS r;
  TriPos pos;
  if (t < s.nt) {
    Tri T;
    int idx[3];
    const int why = load_tri(s, it.cam, t, T, idx);
    if (why == 0) {
      front = 1;
      const int bw = T.xhi - T.xlo + 1, bh = T.yhi - T.ylo + 1;
      if (bw > 0 && bh > 0) {
        if (bw * bh <= kSmallMaxPixels) {
          npx = bw * bh;
          const int ox = 256 * T.xlo + 128, oy = 256 * T.ylo + 128;
          int S = 0;
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const int a = (j + 2) % 3, b = (j + 1) % 3;
            const int ax = T.X[a] - ox, ay = T.Y[a] - oy;
            const int ex = T.X[b] - T.X[a], ey = T.Y[b] - T.Y[a];
            r.c[j] = ex * (0 - ay) - ey * (0 - ax);
            r.gx[j] = -ey * 256;
            r.gy[j] = ex * 256;
            r.q[j] = T.q[j];
            S += r.c[j];
          }
          // S = e_0 + e_1 + e_2 is the same at every point
          r.tl_bw = T.tl[0] | (T.tl[1] << 1) | (T.tl[2] << 2) | (bw << 8);
          r.rbw = 1.0f / (float)bw;
          r.rS = 1.0f / (float)S;
          r.t = t;
          pos.xlo = T.xlo;
          pos.ylo = T.ylo;
        } else {
          large = 1;
        }
      }
    } else if (why == 1) back = 1;
    else if (why == 2) nearc = 1;
    else if (why == 3) guard = 1;
    else if (why == 5) clip = 1;
    else bad = 1;
  }
  // compact the non-empty boxes and take the exclusive prefix of their sizes
  const unsigned ne = __ballot_sync(kAll, npx > 0);
  int pre = npx;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(kAll, pre, o);
    if (lane >= o) pre += v;
  }
  const int total = __shfl_sync(kAll, pre, 31);
  const int start = pre - npx;
  if (npx > 0) {
    const int cpos = __popc(ne & ((1u << lane) - 1u));
    s_tri[wbase + cpos] = r;
    s_pos[wbase + cpos] = pos;
    s_start[wbase + cpos] = start;
  }
  __syncwarp();
  const unsigned le = (lane == 31) ? kAll : ((2u << lane) - 1u);
  int carry = 0;
  for (int w0 = 0; w0 < total; w0 += 32) {
    const unsigned b = (npx > 0 && start >= w0 && start < w0 + 32) ? (1u << (start - w0)) : 0u;
    const unsigned bits = __reduce_or_sync(kAll, b);
    const int slot = w0 + lane;
    if (slot < total) {
      const int o = carry + __popc(bits & le) - 1;
      const TriS& q = s_tri[wbase + o];
      const int local = slot - s_start[wbase + o];
      const int bwq = q.tl_bw >> 8;
      const int dy = (int)(((float)local + 0.5f) * q.rbw);
      const int dx = local - dy * bwq;
      int e[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) e[j] = q.c[j] + q.gx[j] * dx + q.gy[j] * dy;
      if ((e[0] + (q.tl_bw & 1) > 0) && (e[1] + ((q.tl_bw >> 1) & 1) > 0) && (e[2] + ((q.tl_bw >> 2) & 1) > 0)) {
        const TriPos p = s_pos[wbase + o];
        const int S = e[0] + e[1] + e[2];
        red_max_vis(vis + (size_t)(p.ylo + dy) * W + (p.xlo + dx), vis_key(depth_key32(q.q, e, S, q.rS), q.t));
      }
    }
    carry += __popc(bits);
  }
  rc.fb += front | (back << 16);
  rc.ng += nearc | (guard << 16);
  rc.lc += large | (clip << 16);
  rc.bad |= bad;
  // large boxes: the warp strides over each one's screen box
  unsigned lm = __ballot_sync(kAll, large);
  while (lm) {
    const int l = __ffs(lm) - 1;
    lm &= lm - 1;
    const int tq = __shfl_sync(kAll, t, l);
    Tri T;
    int idx[3];
    if (load_tri(s, it.cam, tq, T, idx) != 0) continue;
    const int bw = T.xhi - T.xlo + 1, bh = T.yhi - T.ylo + 1;
    const int npq = bw * bh;
    for (int p = lane; p < npq; p += 32) {
      const int yy = p / bw;
      raster_pixel(T, tq, T.xlo + (p - yy * bw), T.ylo + yy, W, vis);
    }
  }
  // triangles clipped at the near plane (items with a vertex nearer than
  // znear only)
  if constexpr (FULL) {
    unsigned cm = __ballot_sync(kAll, clip);
    while (cm) {
      const int l = __ffs(cm) - 1;
      cm &= cm - 1;
      raster_clipped(s, it.cam, __shfl_sync(kAll, t, l), vis);
    }
  }
  __syncwarp();   // the records are reused by the next round
}

// Raster unit: 32 * it.raster_rounds triangles of one shell in rounds of 32;
// this warp runs rounds [r0, r1).
template <bool FULL>
static __device__ __forceinline__ void unit_raster(const DItem& it, const DShell* sh, int u, WsHeader* hdr, char* smem,
                                                   int r0, int r1) {
  int i = 0;
  while (i + 1 < it.k && u >= it.raster_pre[i + 1]) ++i;
  const DShell& s = sh[i];
  const int per_unit = 32 * it.raster_rounds;
  const int base = (u - it.raster_pre[i]) * per_unit;
  unsigned long long* vis = it.vis + (size_t)i * it.cam.W * it.cam.H;
  RasterCounts rc = {0, 0, 0, 0};
  const int rounds = min(r1, min(per_unit, s.nt - base + 31) / 32);
  for (int r = r0; r < rounds; ++r) raster_round<FULL>(it, s, base + 32 * r, vis, smem, rc);
  warp_count(&hdr->front, rc.fb & 0xFFFFu);
  warp_count(&hdr->back, rc.fb >> 16);
  warp_count(&hdr->nearc, rc.ng & 0xFFFFu);
  warp_count(&hdr->guard, rc.ng >> 16);
  warp_count(&hdr->large, rc.lc & 0xFFFFu);
  warp_count(&hdr->clipped, rc.lc >> 16);
  if (__any_sync(0xffffffffu, rc.bad) && (threadIdx.x & 31) == 0) record_error(hdr, VS_ERR_INVALID_ARG);
}

// ----------------------------------------------------------------------------
// SHADE (+ adjoint)
// ----------------------------------------------------------------------------
// The part of triangle setup shading needs: snapped positions and 1/w,
// after the same validity checks as the raster (0 = usable).
// The vertices' UVs are loaded alongside their snapped positions (both
// need only the indices), so the two loads overlap instead of chaining.
__device__ __forceinline__ int load_tri_shade(const DShell& s, int t, Tri& T, int idx[3], float2 uv[3]) {
  const int* ip = s.tris + 3 * (size_t)t;
  idx[0] = __ldg(ip);
  idx[1] = __ldg(ip + 1);
  idx[2] = __ldg(ip + 2);
  if ((unsigned)idx[0] >= (unsigned)s.nv || (unsigned)idx[1] >= (unsigned)s.nv || (unsigned)idx[2] >= (unsigned)s.nv)
    return 4;
  int4 v[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    v[j] = __ldcg(s.vsetup + idx[j]);
    uv[j] = __ldg(s.uv + idx[j]);
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    if (v[j].x == kInvalidX) return 2;
    T.X[j] = v[j].x;
    T.Y[j] = v[j].y;
    T.iw[j] = __int_as_float(v[j].z);
  }
  const long long a2 = (long long)(T.X[1] - T.X[0]) * (T.Y[2] - T.Y[0]) -
                       (long long)(T.X[2] - T.X[0]) * (T.Y[1] - T.Y[0]);
  return a2 < 0 ? 0 : 1;
}

// Shading a fragment of a triangle clipped at the near plane: the part used
// for the pixel (the only part, or of two the second if it covers the pixel
// under the fill rule, else the first) and its per-vertex UVs.  Rare: kept
// out of line.
static __device__ __forceinline__ bool clipped_part(const DShell& s, const DCam& c, const int idx[3], int px, int py,
                                                 Tri& T, float2 uv[3]) {
  Tri part[2];
  float2 puv[2][3];
  const int n = clip_tri(s.pos, s.uv, c, idx, part, puv);
  if (n == 0) return false;
  int k = 0;
  if (n == 2) {
    long long e[3];
    edge_values(part[1], px, py, e);
    if (covered(part[1], e)) k = 1;
  }
  T = part[k];
  uv[0] = puv[k][0];
  uv[1] = puv[k][1];
  uv[2] = puv[k][2];
  return true;
}

template <int DEG, int VEC, bool KEEP = false>
__device__ __forceinline__ Frag fetch_sh(const DShell& s, const Footprint& f, const float3 v) {
  constexpr int NCH = 1 + 3 * (DEG + 1) * (DEG + 1);
  float Y[16];
  sh_basis(DEG, v.x, v.y, v.z, Y);
  float val[NCH];
  bilinear_f16<NCH, VEC, KEEP>(reinterpret_cast<const __half*>(s.tex), s.tw, s.pitch, f, val);
  return decode_sh<DEG>(val, Y);
}

// The same with the basis already evaluated (sY: the pixel's NB values).
template <int DEG, int VEC>
__device__ __forceinline__ Frag fetch_sh_basis(const DShell& s, const Footprint& f, const float* sY) {
  constexpr int NB = (DEG + 1) * (DEG + 1), NCH = 1 + 3 * NB;
  float Y[16];
#pragma unroll
  for (int m = 0; m < NB; ++m) Y[m] = sY[m];
  float val[NCH];
  bilinear_f16<NCH, VEC>(reinterpret_cast<const __half*>(s.tex), s.tw, s.pitch, f, val);
  return decode_sh<DEG>(val, Y);
}

// Texel load width of the compiled SH classes: 256-bit loads from degree 1
// (texels of 16 or more channels), 128-bit for degree 0.
template <int TC>
__host__ __device__ constexpr int sh_vec() {
  return TC == TC_SH0 ? 8 : 16;
}

template <int DEG>
__device__ __forceinline__ Frag fetch_baked_v(const DShell& s, int ix, float fx, int iy, float fy, const float3 v) {
  float Y[16];
  sh_basis(DEG, v.x, v.y, v.z, Y);
  return fetch_baked<DEG>(s, ix, fx, iy, fy, Y);
}

// Colour and opacity of one fragment; f = its clamped footprint and (ix +
// fx, iy + fy) the unclamped texel coordinate (baked bands derive their own
// footprints from it); v = unit ray direction (SH formats only).  KEEP: FP16
// texel loads mark their lines evict_last (forward-only kernels).
template <int TC, bool KEEP = false>
__device__ __forceinline__ Frag fetch_frag(const DShell& s, const Footprint& f, int ix, float fx, int iy, float fy,
                                           const float3 v) {
  if constexpr (TC == TC_RGBA) {
    float c[4];
    bilinear_rgba<4>(reinterpret_cast<const float*>(s.tex), s.tw, s.pitch, f, c);
    return {c[0], c[1], c[2], c[3]};
  } else if constexpr (TC >= TC_U80) {
    return fetch_baked_v<TC - TC_U80>(s, ix, fx, iy, fy, v);
  } else if constexpr (TC >= TC_SH0) {
    return fetch_sh<TC - TC_SH0, sh_vec<TC>(), KEEP>(s, f, v);
  }
  if (s.fmt == VS_TEX_SH_U8) {
    switch (s.degree) {
      case 0: return fetch_baked_v<0>(s, ix, fx, iy, fy, v);
      case 1: return fetch_baked_v<1>(s, ix, fx, iy, fy, v);
      case 2: return fetch_baked_v<2>(s, ix, fx, iy, fy, v);
      default: return fetch_baked_v<3>(s, ix, fx, iy, fy, v);
    }
  }
  if (s.fmt == VS_TEX_RGBA_F32) {
    float c[4];
    if (s.vec == 4) bilinear_rgba<4>(reinterpret_cast<const float*>(s.tex), s.tw, s.pitch, f, c);
    else bilinear_rgba<1>(reinterpret_cast<const float*>(s.tex), s.tw, s.pitch, f, c);
    return {c[0], c[1], c[2], c[3]};
  }
#define VS_CASE(D, V) \
  case D * 16 + V: return fetch_sh<D, V, KEEP>(s, f, v);
  switch (s.degree * 16 + s.vec) {
    VS_CASE(0, 1) VS_CASE(0, 2) VS_CASE(0, 4) VS_CASE(0, 8)
    VS_CASE(1, 1) VS_CASE(1, 2) VS_CASE(1, 4) VS_CASE(1, 8)
    VS_CASE(2, 1) VS_CASE(2, 2) VS_CASE(2, 4) VS_CASE(2, 8)
    VS_CASE(3, 1) VS_CASE(3, 2) VS_CASE(3, 4) VS_CASE(3, 8)
    default: return {0.f, 0.f, 0.f, 0.f};
  }
#undef VS_CASE
}

// Texel class of a kernel: TC_ANY decides per shell at run time; the others
// are compiled for one format (RGBA with 16-byte texel loads and gradient
// reductions, SH of one degree with 16-byte loads, or baked bytes of one
// degree), which keeps the kernel small (one fetch and one scatter body
// instead of all of them).  is_sh: the format needs the ray direction.
template <int TC>
__device__ __forceinline__ bool is_sh(const DShell& s) {
  if constexpr (TC == TC_ANY) return s.fmt != VS_TEX_RGBA_F32;
  else return TC >= TC_SH0;
}

// Scatter of one fragment's adjoint.  d = (d0, d1, d2, d3) from the
// per-pixel pass: RGBA: dL/d(r, g, b, alpha) of the texel values; SH:
// dL/dz_r, dL/dz_g, dL/dz_b (z the pre-sigmoid colour sums) and dL/da (a
// the alpha logit).  SH values get dz_ch * Y_m (v = unit ray direction).
template <int DEG, int GV>
__device__ __forceinline__ void scatter_sh(const DShell& s, const Footprint& f, const float3 v, const float4 d) {
  constexpr int NB = (DEG + 1) * (DEG + 1);
  constexpr int NCH = 1 + 3 * NB;
  float Y[16];
  sh_basis(DEG, v.x, v.y, v.z, Y);
  float dval[NCH];
  dval[0] = d.w;
#pragma unroll
  for (int m = 0; m < NB; ++m) {
    dval[1 + 3 * m] = d.x * Y[m];
    dval[2 + 3 * m] = d.y * Y[m];
    dval[3 + 3 * m] = d.z * Y[m];
  }
  scatter_grad<NCH, GV>(s.grad, s.tw, s.gpitch, f, dval);
}

template <int TC>
__device__ __forceinline__ void scatter_frag(const DShell& s, const Footprint& f, const float3 v, const float4 d) {
  if constexpr (TC == TC_RGBA) {
    const float dval[4] = {d.x, d.y, d.z, d.w};
    scatter_grad<4, 4>(s.grad, s.tw, s.gpitch, f, dval);
    return;
  } else if constexpr (TC >= TC_U80) {
    return;   // baked shells have no adjoint (refused on the host)
  } else if constexpr (TC >= TC_SH0) {
    scatter_sh<TC - TC_SH0, 4>(s, f, v, d);
    return;
  }
  if (s.fmt == VS_TEX_SH_U8) return;
  if (s.fmt == VS_TEX_RGBA_F32) {
    const float dval[4] = {d.x, d.y, d.z, d.w};
    if (s.gvec == 4) scatter_grad<4, 4>(s.grad, s.tw, s.gpitch, f, dval);
    else if (s.gvec == 2) scatter_grad<4, 2>(s.grad, s.tw, s.gpitch, f, dval);
    else scatter_grad<4, 1>(s.grad, s.tw, s.gpitch, f, dval);
    return;
  }
#define VS_CASE(D, V) \
  case D * 16 + V: scatter_sh<D, V>(s, f, v, d); return;
  switch (s.degree * 16 + s.gvec) {
    VS_CASE(0, 1) VS_CASE(0, 2) VS_CASE(0, 4)
    VS_CASE(1, 1) VS_CASE(1, 2) VS_CASE(1, 4)
    VS_CASE(2, 1) VS_CASE(2, 2) VS_CASE(2, 4)
    VS_CASE(3, 1) VS_CASE(3, 2) VS_CASE(3, 4)
    default: return;
  }
#undef VS_CASE
}

// A footprint kept in shared memory between the fetch and the scatter:
// x0 | y0 << 16 (texture sides <= 65536), and the fractions with the sign
// bit set when the second tap equals the first (clamped at an edge).
__device__ __forceinline__ void pack_footprint(const Footprint& f, unsigned& xy, float2& fr) {
  xy = (unsigned)f.x0 | ((unsigned)f.y0 << 16);
  fr.x = __uint_as_float(__float_as_uint(f.fx) | (f.x1 == f.x0 ? 0x80000000u : 0u));
  fr.y = __uint_as_float(__float_as_uint(f.fy) | (f.y1 == f.y0 ? 0x80000000u : 0u));
}

__device__ __forceinline__ Footprint unpack_footprint(unsigned xy, float2 fr) {
  Footprint f;
  f.x0 = (int)(xy & 0xffffu);
  f.y0 = (int)(xy >> 16);
  const unsigned bx = __float_as_uint(fr.x), by = __float_as_uint(fr.y);
  f.x1 = f.x0 + ((bx >> 31) ? 0 : 1);
  f.y1 = f.y0 + ((by >> 31) ? 0 : 1);
  f.fx = __uint_as_float(bx & 0x7fffffffu);
  f.fy = __uint_as_float(by & 0x7fffffffu);
  return f;
}

// alpha_w of the fragments [0, total) of a shading round (lane-strided),
// from the packed (shell, triangle) entries.
static __device__ __noinline__ void atten_pass(const DCam& cam, const DShell* sh, int pbase, const int* sent,
                                        const unsigned short* spl, float* saw, int total) {
  const int lane = threadIdx.x & 31;
  for (int j = lane; j < total; j += 32) {
    const int e = sent[j];
    const int i = e >> kTriBits, t = e & (kMaxTris - 1);
    const DShell& s = sh[i];
    saw[j] = 1.0f;
    if (t >= s.nt) continue;
    const int* ip = s.tris + 3 * (size_t)t;
    const int idx[3] = {__ldg(ip), __ldg(ip + 1), __ldg(ip + 2)};
    if ((unsigned)idx[0] >= (unsigned)s.nv || (unsigned)idx[1] >= (unsigned)s.nv || (unsigned)idx[2] >= (unsigned)s.nv)
      continue;
    const int pp = pbase + (spl[j] & 31);
    const int y = pp / cam.W, x = pp - y * cam.W;
    saw[j] = alpha_atten(s.pos, idx, ray_dir(cam, x, y));
  }
}

// Per-layer buffers (Figs. S1/S3): record of shell i at pixel p, 12 floats =
// unit face normal, u, v | opacity, blending weight T_i alpha_i, r | g, b, 0, 0.
__device__ __forceinline__ float* layer_rec(const DItem& it, int i, int p) {
  return it.layers + 12 * ((size_t)i * it.cam.W * it.cam.H + p);
}

// The geometric part of a fragment's record: face normal and the UV at the
// pixel (from the unclamped texel coordinate: u = (x + 1/2) / W).
__device__ __forceinline__ void layer_geom(const DItem& it, const DShell& s, const int idx[3], int i, int p, int ix,
                                           float fx, int iy, float fy) {
  const float3 n = face_cross(s.pos, idx);
  const float r = rsqrtf(n.x * n.x + n.y * n.y + n.z * n.z);
  float* L = layer_rec(it, i, p);
  const float u = __fdiv_rn(__fadd_rn(__fadd_rn((float)ix, 0.5f), fx), (float)s.tw);
  const float v = __fdiv_rn(__fadd_rn(__fadd_rn((float)iy, 0.5f), fy), (float)s.th);
  *reinterpret_cast<float4*>(L) = make_float4(n.x * r, n.y * r, n.z * r, u);
  L[4] = v;
}

// Markers in the lane word of a fragment-list entry.
constexpr unsigned kBadFrag = 0x8000u;    // unusable triangle: invisible, no adjoint
constexpr unsigned kClipFrag = 0x4000u;   // triangle to clip at the near plane (pending)

// One fragment of a triangle clipped at the near plane (list entry j): the
// part used at its pixel, footprint, texel fetch; like the fetch loop of
// shade_round, out of line because it is rare.
template <bool BWD, int TC>
static __device__ __forceinline__ void shade_clipped(const DItem& it, const DShell* sh, int pbase, int j, const int* sent,
                                                  unsigned short* spl, float4* sfrag, unsigned* sxy, float2* sfxy,
                                                  unsigned* nfrag, unsigned* bad) {
  const int e = sent[j];
  const DShell& s = sh[e >> kTriBits];
  const int* ip = s.tris + 3 * (size_t)(e & (kMaxTris - 1));
  const int idx[3] = {__ldg(ip), __ldg(ip + 1), __ldg(ip + 2)};   // checked in range by load_tri_shade
  const int pp = pbase + (spl[j] & 31);
  const int W = it.cam.W;
  const int y = pp / W, x = pp - y * W;
  Tri T;
  float2 uv[3];
  Frag fr = {0.f, 0.f, 0.f, 0.f};
  spl[j] &= (unsigned short)~kClipFrag;
  if (!clipped_part(s, it.cam, idx, 256 * x + 128, 256 * y + 128, T, uv)) {
    *bad = 1;
    spl[j] |= (unsigned short)kBadFrag;
  } else {
    int ix, iy;
    float fx, fy;
    texel_coords(T, uv, s.tw, s.th, 256 * x + 128, 256 * y + 128, ix, fx, iy, fy);
    const Footprint f = clamp_footprint(ix, fx, iy, fy, s.tw, s.th);
    if constexpr (BWD) {
      unsigned xy;
      float2 fxy;
      pack_footprint(f, xy, fxy);
      sxy[j] = xy;
      sfxy[j] = fxy;
    }
    float3 v = make_float3(0.f, 0.f, 1.f);
    if (is_sh<TC>(s)) v = ray_dir(it.cam, x, y);
    fr = fetch_frag<TC, !BWD>(s, f, ix, fx, iy, fy, v);
    if (it.layers) layer_geom(it, s, idx, e >> kTriBits, pp, ix, fx, iy, fy);
    ++*nfrag;
  }
  sfrag[j] = make_float4(fr.r, fr.g, fr.b, fr.a);
}

// Shading round: 32 consecutive pixels, one per lane.
//  1. each lane reads its pixel's k visibility words (independent loads)
//     into a per-shell hit table.  The round then runs in passes over
//     consecutive lane ranges whose fragments fit the warp's list (one
//     pass when the list holds 32 K; kFragCap >= kMaxShells, so every pass
//     takes at least one pixel); each pass compacts its lanes' hits into
//     the list, pixel-major with shells ascending;
//  2. the warp shades the list 32 fragments at a time, every lane busy:
//     perspective-correct UV, bilinear fetch at texel centres (Fig. 5), SH
//     decode with the ray direction (and, with the flag, alpha_w first);
//     the adjoint keeps each footprint in shared memory;
//  3. each lane of the pass composites its pixel front to back from shared
//     memory (Eq. 6 with Eq. 1's transmittance).  For the adjoint it then
//     runs back to front with B_i = A_i . g, A_i the colour seen from in
//     front of shell i (B_i = alpha_i (c_i . g) + (1 - alpha_i) B_{i+1},
//     B_k = bg . g): dL/dc_i = T_i alpha_i g, dL/dalpha_i = T_i (c_i . g -
//     B_{i+1}), taken through alpha_w and the sigmoids to the texel-value
//     space in place;
//  4. (adjoint) the warp scatters dL/d(texel) from the stored footprints --
//     no global loads, only reductions.  SH classes of degree 1-3 scatter
//     cooperatively: each lane owns one 16-byte chunk of one tap's texel, so
//     one reduction instruction writes whole contiguous texel rows of a
//     fragment (4 taps x up to 8 chunks); the other classes give each lane
//     a fragment.
// FROM_HITS: hits come from the public int32 buffer (standalone backward)
// instead of the visibility words.
//
// Shared memory of the warp (shade_warp_bytes), C = frag_cap(K, BWD):
//   hit  int    [32 K]  triangle per (shell, lane) of the round (1); own
//                       space only when C < 32 K, else it is the frag area,
//                       which the single pass overwrites after the fill
//   frag float4 [C]  rgb + raw alpha (2 -> 3), then the adjoint d (3 -> 4)
//   ent  u32    [C]  shell << 27 | triangle (1 -> 2), then x0 | y0 << 16
//   aw   float  [C]  alpha_w (2 -> 3)
//   pl   u16    [C]  lane | shell << 5 | kBadFrag / kClipFrag
// adjoint only:
//   fxy  float2 [C]  footprint fractions (2 -> 4)
//   T    float  [C]  transmittance in front of the fragment (3)
//   Y    float  [32 NB]  SH basis of the round's pixels, NB = pixel_basis
//                    (SH classes of degree 1-3; 1 -> 2, 4)
static_assert(kMaxShells <= 16, "shell index takes 4 bits of the lane word");
static_assert(kFragCap >= kMaxShells, "a pixel's fragments must fit one pass");

template <bool BWD, bool FROM_HITS, int TC, bool FULL>
__device__ __forceinline__ void shade_round(const DItem& it, const DShell* sh, int pbase, char* wb, int K,
                                            unsigned& nfrag, unsigned& bad, float& loss_acc) {
  const unsigned kAll = 0xffffffffu;
  const int W = it.cam.W, H = it.cam.H;
  const int HW = W * H;
  const int k = it.k;
  const int lane = threadIdx.x & 31;
  const int C = frag_cap(K, BWD);
  const bool own_table = C < 32 * K;
  int* scratch = reinterpret_cast<int*>(wb);
  char* lb = own_table ? wb + 128 * (size_t)K : wb;
  float4* sfrag = reinterpret_cast<float4*>(lb);
  int* sent = reinterpret_cast<int*>(lb + 16 * C);
  unsigned* sxy = reinterpret_cast<unsigned*>(sent);
  float* saw = reinterpret_cast<float*>(lb + 20 * C);
  unsigned short* spl = reinterpret_cast<unsigned short*>(lb + 24 * C);
  float2* sfxy = reinterpret_cast<float2*>(lb + 26 * C);   // BWD only
  float* sT = reinterpret_cast<float*>(lb + 34 * C);       // BWD only
  constexpr int NB = pixel_basis(TC, BWD);
  float* sY = reinterpret_cast<float*>(lb + 38 * C);       // NB > 0 only
  const int p = pbase + lane;
  const bool pix_ok = p < HW;
  if constexpr (NB > 0) {   // SH basis of this lane's pixel, shared by its fragments
    if (pix_ok) {
      const int y = p / W, x = p - y * W;
      const float3 v = ray_dir(it.cam, x, y);
      float Yb[16];
      sh_basis(TC - TC_SH0, v.x, v.y, v.z, Yb);
#pragma unroll
      for (int m = 0; m < NB; ++m) sY[lane * NB + m] = Yb[m];
    }
  }

  // 1. hits of this pixel
  unsigned mask = 0;
  // eight shells at a time: all loads of a group are in flight together
  for (int i0 = 0; i0 < k; i0 += 8) {
    int tt[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const int i = i0 + d;
      tt[d] = -1;
      if (i < k && pix_ok) {
        if (FROM_HITS) tt[d] = __ldg(it.hits + (size_t)i * HW + p);
        else tt[d] = load_vis_tri(it.vis + (size_t)i * HW + p);
      }
    }
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const int i = i0 + d;
      if (i < k) {
        if (!FROM_HITS && it.hits && pix_ok) it.hits[(size_t)i * HW + p] = tt[d];
        scratch[i * 32 + lane] = tt[d];
        if (tt[d] >= 0) mask |= 1u << i;
      }
    }
  }
  const int cnt = __popc(mask);
  int pre = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(kAll, pre, o);
    if (lane >= o) pre += v;
  }
  const int start = pre - cnt;
  const bool atten = (it.flags & VS_FLAG_ALPHA_ATTEN) != 0;
  int clip_pending = 0;
  if constexpr (FULL) {   // per-layer buffers: every shell's record starts at zero
    if (it.layers && pix_ok)
      for (int i = 0; i < k; ++i) {
        float4* L = reinterpret_cast<float4*>(layer_rec(it, i, p));
        L[0] = L[1] = L[2] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
  }
  __syncwarp();

  for (int l0 = 0; l0 < 32;) {
    // lanes [l0, l1) whose fragments fit the list; pre is nondecreasing
    const int f0 = __shfl_sync(kAll, start, l0);
    const int l1 = __popc(__ballot_sync(kAll, pre - f0 <= C));
    const int nf = __shfl_sync(kAll, pre, l1 - 1) - f0;
    const bool mine = lane >= l0 && lane < l1;
    const int s0 = start - f0;          // this lane's first list slot
    if (mine) {
      unsigned m = mask;
      int c = s0;
      while (m) {
        const int i = __ffs(m) - 1;
        m &= m - 1;
        sent[c] = (i << kTriBits) | (scratch[i * 32 + lane] & (kMaxTris - 1));
        spl[c] = (unsigned short)(lane | (i << 5));
        ++c;
      }
    }
    __syncwarp();

    // 2a. transparency attenuation, in a pass of its own so that the fetch
    //     loop below keeps its registers
    if (atten) {
      atten_pass(it.cam, sh, pbase, sent, spl, saw, nf);
      __syncwarp();
    }

    // 2b. fragments, 32 at a time
    for (int j0 = 0; j0 < nf; j0 += 32) {
      const int j = j0 + lane;
      if (j < nf) {
        const int e = sent[j];
        const int i = e >> kTriBits, t = e & (kMaxTris - 1);
        const int pp = pbase + (spl[j] & 31);
        const DShell& s = sh[i];
        Frag fr = {0.f, 0.f, 0.f, 0.f};
        Tri Tr;
        int idx[3];
        const int y = pp / W, x = pp - y * W;
        float2 uv[3];
        const int r = t < s.nt ? load_tri_shade(s, t, Tr, idx, uv) : 4;
        if (FULL && r == 2) {
          // a vertex nearer than znear (or off the guard band): the triangle
          // is clipped; shaded by the pass below
          clip_pending = 1;
          spl[j] |= (unsigned short)kClipFrag;
        } else if (r != 0) {
          bad = 1;
          spl[j] |= (unsigned short)kBadFrag;   // invisible, and no adjoint
        } else {
          int ix, iy;
          float fx, fy;
          texel_coords(Tr, uv, s.tw, s.th, 256 * x + 128, 256 * y + 128, ix, fx, iy, fy);
          const Footprint f = clamp_footprint(ix, fx, iy, fy, s.tw, s.th);
          if constexpr (BWD) {
            unsigned xy;
            float2 fxy;
            pack_footprint(f, xy, fxy);
            sxy[j] = xy;      // the entry is not read again
            sfxy[j] = fxy;
          }
          if constexpr (NB > 0) {
            fr = fetch_sh_basis<TC - TC_SH0, sh_vec<TC>()>(s, f, sY + (spl[j] & 31) * NB);
          } else {
            float3 v = make_float3(0.f, 0.f, 1.f);
            if (is_sh<TC>(s)) v = ray_dir(it.cam, x, y);
            fr = fetch_frag<TC, !BWD>(s, f, ix, fx, iy, fy, v);
          }
          if constexpr (FULL) {
            if (it.layers) layer_geom(it, s, idx, i, pp, ix, fx, iy, fy);
          }
          ++nfrag;
        }
        // raw opacity here; the composite applies alpha_w
        sfrag[j] = make_float4(fr.r, fr.g, fr.b, fr.a);
        if (!atten) saw[j] = 1.0f;
      }
    }
    __syncwarp();
    // 2c. fragments of triangles clipped at the near plane (rare; out of line)
    if (FULL && __any_sync(kAll, clip_pending)) {
      for (int j = lane; j < nf; j += 32)
        if (spl[j] & kClipFrag) shade_clipped<BWD, TC>(it, sh, pbase, j, sent, spl, sfrag, sxy, sfxy, &nfrag, &bad);
      __syncwarp();
    }

    // 3. composite the pass's pixels
    if (mine) {
      float T = 1.0f, Cr = 0.f, Cg = 0.f, Cb = 0.f;
      for (int c = 0; c < cnt; ++c) {
        const float4 f = sfrag[s0 + c];
        if constexpr (BWD) sT[s0 + c] = T;
        const float a = f.w * saw[s0 + c];
        const float ta = T * a;
        if constexpr (FULL) {
          if (it.layers && !(spl[s0 + c] & kBadFrag)) {
            float* L = layer_rec(it, (spl[s0 + c] >> 5) & 15, p);
            L[5] = a;
            L[6] = ta;
            L[7] = f.x;
            L[8] = f.y;
            L[9] = f.z;
          }
        }
        Cr = fmaf(ta, f.x, Cr);
        Cg = fmaf(ta, f.y, Cg);
        Cb = fmaf(ta, f.z, Cb);
        T = T * (1.0f - a);
      }
      const float outr = fmaf(T, it.bg[0], Cr), outg = fmaf(T, it.bg[1], Cg), outb = fmaf(T, it.bg[2], Cb);
      if (pix_ok && it.out) it.out[p] = make_float4(outr, outg, outb, 1.0f - T);
      if constexpr (BWD) {
        float gr = 0.f, gg = 0.f, gb = 0.f;
        if (pix_ok) {
          const float* gp = it.grad_rgb + 3 * (size_t)p;
          gr = __ldg(gp);
          gg = __ldg(gp + 1);
          gb = __ldg(gp + 2);
          if (it.flags & VS_FLAG_LOSS_L2) {
            const float dr = outr - gr, dg = outg - gg, db = outb - gb;
            const float inv = 1.0f / (3.0f * (float)HW);
            loss_acc += (dr * dr + dg * dg + db * db) * inv;
            gr = 2.0f * inv * dr;
            gg = 2.0f * inv * dg;
            gb = 2.0f * inv * db;
          } else if (it.flags & VS_FLAG_LOSS_L1) {
            const float dr = outr - gr, dg = outg - gg, db = outb - gb;
            const float inv = 1.0f / (3.0f * (float)HW);
            loss_acc += (fabsf(dr) + fabsf(dg) + fabsf(db)) * inv;
            gr = dr > 0.0f ? inv : (dr < 0.0f ? -inv : 0.0f);
            gg = dg > 0.0f ? inv : (dg < 0.0f ? -inv : 0.0f);
            gb = db > 0.0f ? inv : (db < 0.0f ? -inv : 0.0f);
          }
        }
        // back to front; the colour and opacity of each fragment are
        // replaced by the adjoint in texel-value space
        float B = it.bg[0] * gr + it.bg[1] * gg + it.bg[2] * gb;
        for (int c = cnt - 1; c >= 0; --c) {
          const float4 f = sfrag[s0 + c];
          const float aw = saw[s0 + c];
          const float a = f.w * aw;
          const float cg = f.x * gr + f.y * gg + f.z * gb;
          const float Tc = sT[s0 + c];
          const float ta = Tc * a;
          // dL/d(raw alpha): alpha_w is a constant of the texels
          const float ga = Tc * (cg - B) * aw;
          const DShell& s = sh[(spl[s0 + c] >> 5) & 15];
          float4 d;
          if (!is_sh<TC>(s)) {
            d = make_float4(ta * gr, ta * gg, ta * gb, ga);
          } else {
            d = make_float4(ta * gr * (f.x * (1.0f - f.x)), ta * gg * (f.y * (1.0f - f.y)),
                            ta * gb * (f.z * (1.0f - f.z)), ga * (f.w * (1.0f - f.w)));
          }
          sfrag[s0 + c] = d;
          B = fmaf(a, cg - B, B);
        }
      }
    }
    if constexpr (NB > 0) {
      __syncwarp();
      // 4. adjoint scatter, cooperative: lane = (fragment, 16-byte chunk l
      //    of the texel's NCH values), looping over the 4 taps, so one
      //    reduction instruction writes FPI fragments' texel rows as
      //    contiguous chunks.  Each value is w_q * (d_c * Y_m), as in
      //    scatter_sh.
      constexpr int NCH = 1 + 3 * NB, NL = (NCH + 3) / 4;
      constexpr int CPT = NL <= 4 ? 4 : (NL <= 8 ? 8 : 16);   // lanes per fragment
      constexpr int FPI = 32 / CPT;                            // fragments per step
      const int l = lane % CPT, fs = lane / CPT;
      // Channel c = 4 l + e >= 1 holds colour (c - 1) % 3 of basis function
      // (c - 1) / 3: with rot = (4 l - 1) mod 3 (2 for l = 0), channel e has
      // colour (rot + e) % 3 and basis mA while rot + e < 3, else mB.
      // Channel 0 is the alpha logit; channels >= NCH are padding (0).
      const int rot = (4 * l + 2) % 3;
      const int mA = l == 0 ? 0 : (4 * l - 1) / 3;
      const int mB = l == 0 ? 0 : min(mA + 1, NB - 1);
      const bool k1 = 4 * l + 1 < NCH, k2 = 4 * l + 2 < NCH, k3 = 4 * l + 3 < NCH;
      if (l < NL) {
        for (int j = fs; j < nf; j += FPI) {
          const unsigned pl = spl[j];
          if (pl & kBadFrag) continue;
          const DShell& s = sh[(pl >> 5) & 15];
          const float4 d = sfrag[j];
          const float* Y = sY + (pl & 31) * NB;
          const float yA = Y[mA], yB = Y[mB];
          const float c0 = rot == 0 ? d.x : (rot == 1 ? d.y : d.z);
          const float c1 = rot == 0 ? d.y : (rot == 1 ? d.z : d.x);
          const float c2 = rot == 0 ? d.z : (rot == 1 ? d.x : d.y);
          const float dv0 = l == 0 ? d.w : c0 * yA;
          const float dv1 = c1 * (rot < 2 ? yA : yB);
          const float dv2 = c2 * (rot < 1 ? yA : yB);
          const float dv3 = c0 * yB;
          const Footprint f = unpack_footprint(sxy[j], sfxy[j]);
          const size_t r0 = (size_t)f.y0 * s.tw, r1 = (size_t)f.y1 * s.tw;
          float* g = s.grad + 4 * l;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int xq = (q & 1) ? f.x1 : f.x0;
            const float w = ((q & 1) ? f.fx : 1.0f - f.fx) * ((q & 2) ? f.fy : 1.0f - f.fy);
            red_add_v4f32(g + (((q & 2) ? r1 : r0) + xq) * s.gpitch, w * dv0, k1 ? w * dv1 : 0.0f,
                          k2 ? w * dv2 : 0.0f, k3 ? w * dv3 : 0.0f);
          }
        }
      }
    } else if constexpr (BWD) {
      __syncwarp();
      // 4. adjoint scatter, 32 fragments at a time
      for (int j0 = 0; j0 < nf; j0 += 32) {
        const int j = j0 + lane;
        if (j < nf) {
          const unsigned pl = spl[j];
          if (pl & kBadFrag) continue;
          const DShell& s = sh[(pl >> 5) & 15];
          const Footprint f = unpack_footprint(sxy[j], sfxy[j]);
          float3 v = make_float3(0.f, 0.f, 1.f);
          if (is_sh<TC>(s)) {
            const int pp = pbase + (int)(pl & 31);
            const int y = pp / W, x = pp - y * W;
            v = ray_dir(it.cam, x, y);
          }
          scatter_frag<TC>(s, f, v, sfrag[j]);
        }
      }
    }
    __syncwarp();   // the list is rebuilt by the next pass
    l0 = l1;
  }
}

// Shading unit: 32 * it.shade_rounds consecutive pixels in rounds of 32;
// this warp runs rounds [r0, r1).  `wb` is the warp's shared-memory slice.
template <bool BWD, bool FROM_HITS, int TC, bool FULL>
__device__ __forceinline__ void unit_shade(const DItem& it, const DShell* sh, int u, WsHeader* hdr, char* wb, int K,
                                           int r0, int r1) {
  const unsigned kAll = 0xffffffffu;
  const int HW = it.cam.W * it.cam.H;
  unsigned nfrag = 0, bad = 0;
  float loss = 0.0f;
  for (int r = r0; r < r1; ++r) {
    const int pbase = (u * it.shade_rounds + r) * 32;
    if (pbase >= HW) break;
    shade_round<BWD, FROM_HITS, TC, FULL>(it, sh, pbase, wb, K, nfrag, bad, loss);
  }
  const int lane = threadIdx.x & 31;
  if (!FROM_HITS) warp_count(&hdr->frags, nfrag);
  if (__any_sync(kAll, bad) && lane == 0) record_error(hdr, VS_ERR_INVALID_ARG);
  if constexpr (BWD) {
    if (it.loss && (it.flags & (VS_FLAG_LOSS_L2 | VS_FLAG_LOSS_L1))) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(kAll, loss, o);
      if (lane == 0 && loss != 0.0f) atomicAdd(it.loss, loss);
    }
  }
}

extern __shared__ __align__(16) char vs_smem[];

// Shared-memory slice of the calling warp (every phase carves the same way).
__device__ __forceinline__ char* warp_smem(int K, bool bwd, int tc) {
  return vs_smem + (threadIdx.x >> 5) * warp_slice_bytes(K, bwd, tc);
}

template <bool BWD, bool FROM_HITS, int TC, bool FULL>
__global__ void __launch_bounds__(kThreads, BWD ? VS_BWD_BLOCKS : VS_FWD_BLOCKS) k_shade(TableRef tb, int item) {
  const DItem& it = tb.items[item];
  const int w = threadIdx.x >> 5;
  unit_shade<BWD, FROM_HITS, TC, FULL>(it, tb.shells + it.shell0, blockIdx.x, tb.hdr, warp_smem(tb.kmax, BWD, TC), tb.kmax, w,
                             w + 1);
}

// Bounded wait (one lane) for `target` completions; false on timeout or
// abort.  A timeout records VS_ERR_TIMEOUT and raises the abort flag so that
// every warp leaves the persistent loop.
static __device__ bool wait_done(const int* ctr, int target, long long limit, WsHeader* hdr) {
  for (long long n = 0;; ++n) {
    if (ld_acquire(ctr) >= target) return true;
    if (*(volatile int*)&hdr->abort) return false;
    if (n >= limit) {
      record_error(hdr, VS_ERR_TIMEOUT);
      atomicExch(&hdr->abort, 1);
      return false;
    }
    __nanosleep(200);
  }
}

// Persistent kernel over all items; every WARP takes units on its own, so a
// slow unit never holds up the other warps of its block.  Units are
// dispensed in a skewed global order: stage s holds the SETUP units of item
// s, the RASTER units of item s-1 and the SHADE units of item s-2, so that
// an item's visibility words are written, resolved and read within a few
// stages (while still in L2).  A unit waits only for the previous phase of
// its own item, whose units were all dispensed in an earlier stage to warps
// that are already running, so the wait always ends (and is bounded anyway).
template <bool BWD, int TC, bool FULL>
__global__ void __launch_bounds__(pers_threads(BWD), BWD ? VS_PERS_BWD_BLOCKS : VS_PERS_FWD_BLOCKS) k_persistent(TableRef tb, long long spin_limit) {
  const unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  WsHeader* hdr = tb.hdr;
  char* smem = warp_smem(tb.kmax, BWD, TC);
  for (;;) {
    int g = 0;
    if (lane == 0) g = *(volatile int*)&hdr->abort ? tb.total : (int)atomicAdd(&hdr->next_unit, 1u);
    g = __shfl_sync(kAll, g, 0);
    if (g >= tb.total) break;
    // stage: last s with stage_pre[s] <= g
    int lo = 0, hi = tb.n + NPH - 2;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(tb.stage_pre + mid) <= g) lo = mid; else hi = mid - 1;
    }
    int rel = g - __ldg(tb.stage_pre + lo);
    int ph = 0, j = lo;
    for (ph = 0; ph < NPH; ++ph) {
      j = lo - ph;
      const int cnt = (j >= 0 && j < tb.n) ? tb.items[j].units[ph] : 0;
      if (rel < cnt) break;
      rel -= cnt;
    }
    const DItem& it = tb.items[j];
    const int u = rel;
    int ok = 1;
    if (lane == 0 && ph > 0) {
      int target = it.units[ph - 1];
      long long lim = spin_limit;
      if (ph == PH_SHADE && it.stall && u == 0) { target += 1; lim = 4096; }
      ok = wait_done(tb.done + j * NPH + ph - 1, target, lim, hdr) ? 1 : 0;
    }
    ok = __shfl_sync(kAll, ok, 0);
    __syncwarp();   // orders every lane's reads after lane 0's acquire
    if (!ok) break;
    const DShell* sh = tb.shells + it.shell0;
    switch (ph) {
      case PH_SETUP: unit_setup(it, sh, u); break;
      case PH_RASTER: unit_raster<FULL>(it, sh, u, hdr, smem, 0, it.raster_rounds); break;
      default:
        unit_shade<BWD, false, TC, FULL>(it, sh, u, hdr, smem, tb.kmax, 0, it.shade_rounds);
    }
    __syncwarp();
    if (lane == 0) {
      __threadfence();
      atomicAdd(tb.done + j * NPH + ph, 1);
    }
  }
}

}  // namespace vsd
