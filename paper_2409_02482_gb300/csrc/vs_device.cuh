// Device-side building blocks of the k-shell renderer (sm_103a).
//
// Everything a kernel needs is here as __device__ functions so that the
// per-phase kernels of vs_render and the persistent kernel of
// vs_render_batch run the very same arithmetic (batched forward output is
// bit-identical to the plain launches).  The file is compiled with
// --fmad=false: no multiply-add is fused unless written as fmaf(), so the
// arithmetic does not depend on where a function gets inlined.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "vs.h"

namespace vsd {

// ----------------------------------------------------------------------------
// tuning constants and table layout
// ----------------------------------------------------------------------------
constexpr int kThreads = 256;          // threads per block, all kernels
constexpr int kWarps = kThreads / 32;  // a work unit is run by one warp
constexpr int kSetupPerUnit = 1024;    // vertices per setup unit
constexpr int kRasterPerUnit = 256;    // triangles per raster unit of the plain launches
constexpr int kClearPerUnit = 16384;   // visibility words cleared per unit
constexpr int kShadePixels = 256;      // pixels per shading unit of the plain launches
// The plain raster/shade launches run one unit per block, one 32-wide round
// per warp, so their units are kWarps rounds; the persistent kernel takes
// any size per item (DItem::raster_rounds, shade_rounds).
static_assert(kRasterPerUnit == 32 * kWarps && kShadePixels == 32 * kWarps, "plain units = one round per warp");
constexpr int kSmallMaxPixels = 64;    // bbox pixels walked by the warp's pair loop
constexpr int kMaxShells = VS_MAX_SHELLS;
constexpr int kTriBits = 27;           // triangle index bits in a packed fragment
constexpr int kMaxTris = 1 << kTriBits;

// Texel classes: a kernel compiled for TC_ANY decides the format per shell at
// run time; the others serve batches whose shells all share one format with
// 16-byte-aligned texels (and gradients); SH classes of degree >= 1 also want
// 32-byte-aligned texels for their 256-bit loads.
enum : int { TC_ANY = 0, TC_RGBA = 1, TC_SH0 = 2, TC_U80 = 6 };   // TC_SH0 / TC_U80 + degree
constexpr int kNumTc = TC_U80 + 4;

// SH basis values per pixel that an adjoint shading warp keeps for the
// round's fragments (compiled SH classes of degree 1-3: evaluated once per
// pixel instead of once per fragment in the fetch, and read again by the
// cooperative scatter), else 0.  The forward kernels evaluate it per
// fragment: measured faster there, the larger slice costing more L1 than the
// evaluation.
__host__ __device__ constexpr int pixel_basis(int tc, bool bwd) {
  return (bwd && tc >= TC_SH0 + 1 && tc <= TC_SH0 + 3) ? (tc - TC_SH0 + 1) * (tc - TC_SH0 + 1) : 0;
}

// Dynamic shared memory of a shading warp for up to K shells: a fragment
// list of frag_cap(K, bwd) entries -- [frag float4][entry u32][alpha_w
// float][lane|shell u16] and, for the adjoint only, [fractions float2][T
// float] -- and, when the list is shorter than a round's worst case (32 K),
// the round's hit table (32 K ints) in front of it, and behind it, for the
// adjoint, the SH basis of the round's 32 pixels (pixel_basis values each;
// carved in shade_round).
// The forward list holds the worst case (one pass per round).  The adjoint
// list is capped at kFragCap: a round whose fragments do not fit runs in
// several passes, and the smaller slice leaves more of the SM's unified
// L1/shared storage to L1.
#ifndef VS_FRAG_CAP
#define VS_FRAG_CAP 128
#endif
constexpr int kFragCap = VS_FRAG_CAP;
static_assert(kFragCap % 32 == 0, "fragment list in whole 32-wide rounds");
__host__ __device__ constexpr int frag_cap(int K, bool bwd) {
  return (bwd && kFragCap < 32 * K) ? kFragCap : 32 * K;
}
__host__ __device__ constexpr size_t shade_warp_bytes(int K, bool bwd, int tc) {
  return ((frag_cap(K, bwd) < 32 * K ? 128 * (size_t)K : 0) + (bwd ? 38 : 26) * (size_t)frag_cap(K, bwd) +
          128 * (size_t)pixel_basis(tc, bwd) + 15) &
         ~(size_t)15;
}
constexpr size_t kRasterWarpBytes = 32 * (64 + 8 + 4);   // TriS, TriPos, start per triangle
__host__ __device__ constexpr size_t warp_slice_bytes(int K, bool bwd, int tc) {
  return shade_warp_bytes(K, bwd, tc) > kRasterWarpBytes ? shade_warp_bytes(K, bwd, tc) : kRasterWarpBytes;
}
__host__ __device__ constexpr size_t block_smem_bytes(int K, bool bwd, int tc) {
  return warp_slice_bytes(K, bwd, tc) * kWarps;
}

// Block shape of the persistent kernel, per direction.  Its warps take units
// on their own, so the block size only sets the register budget: the SM's
// 64K registers are shared by (warps per block) x (resident blocks) warps.
// The fused forward + adjoint runs 5-warp blocks, 4 per SM: 20 warps at 96
// registers (measured 0.7 % faster on the C2 fitting step than 24 warps at
// 80 registers, which spill ~2x more; 16 warps at 128 registers, no spill,
// 4 % slower).  The forward keeps 8-warp blocks, 3 per SM (24 warps at 80
// registers: 7 % faster than 20 warps at 96).
#ifndef VS_PERS_BWD_WARPS
#define VS_PERS_BWD_WARPS 5
#endif
#ifndef VS_PERS_FWD_WARPS
#define VS_PERS_FWD_WARPS 8
#endif
__host__ __device__ constexpr int pers_warps(bool bwd) { return bwd ? VS_PERS_BWD_WARPS : VS_PERS_FWD_WARPS; }
__host__ __device__ constexpr int pers_threads(bool bwd) { return 32 * pers_warps(bwd); }
__host__ __device__ constexpr size_t pers_smem_bytes(int K, bool bwd, int tc) {
  return warp_slice_bytes(K, bwd, tc) * pers_warps(bwd);
}


// Phases of one item.  Large triangles are rasterized by the whole block
// inside the raster unit that met them.
enum { PH_SETUP = 0, PH_RASTER = 1, PH_SHADE = 2, NPH = 3 };

constexpr int kInvalidX = -2147483647 - 1;   // vertex marker: culled
enum { VTX_NEAR = 1, VTX_GUARD = 2 };

struct alignas(16) DCam {
  float m[12];                 // world -> camera [R | t], row-major
  float fx, fy, cx, cy, znear;
  int32_t W, H;
  float rfx, rfy;              // 1 / fx, 1 / fy (ray directions only)
  int32_t pad[3];
};

struct alignas(16) DShell {
  const float* pos;            // [nv, 3]
  const float2* uv;            // [nv]
  const int32_t* tris;         // [nt, 3]
  const void* tex;             // [th, tw, pitch]
  float* grad;                 // [th, tw, gpitch] FP32 (backward) or null
  int4* vsetup;                // [nv] (X, Y, bits(1/w), q) -- workspace
  int32_t nv, nt, tw, th;
  int32_t fmt, degree, pitch;
  int32_t vec;                 // texel load width in values (1, 2, 4, 8)
  int32_t gvec;                // gradient atomic width in floats (1, 2, 4)
  int32_t wide;                // texels 32-byte aligned (base and pitch): 256-bit loads
  int4* pad5;                  // unused
  // VS_TEX_SH_U8: byte offset of band l in tex, resolution shift per band,
  // decode value = vmin + vscale * q
  long long boff[4];
  float vmin, vscale;
  int32_t bshift;
  int32_t gpitch;              // FP32 values per gradient texel (>= the value count)
};

struct alignas(16) DItem {
  DCam cam;
  float4* out;                 // [H*W]
  int32_t* hits;               // [k, H*W] or null
  const float* grad_rgb;       // [H*W, 3] gradient or target, or null
  float* loss;                 // scalar or null
  unsigned long long* vis;     // [k, H*W] -- workspace
  float* layers;               // [k, H*W, 12] per-layer buffers or null
  int32_t k, shell0, pad0, clear_units;
  int32_t flags, do_bwd, stall;
  int32_t raster_rounds;       // raster unit = 32 * raster_rounds triangles
  int32_t shade_rounds;        // shading unit = 32 * shade_rounds pixels
  int32_t units[4];            // per phase (3 used)
  int32_t setup_pre[kMaxShells + 1];
  int32_t raster_pre[kMaxShells + 1];
  float bg[4];
};

// Workspace header (first 256 bytes).  status and the counters persist
// across calls until vs_read_stats resets them; next_unit and abort are
// reset by every call's table upload.
struct alignas(16) WsHeader {
  int32_t status;
  int32_t abort;
  uint32_t next_unit;
  int32_t pad;
  unsigned long long frags, front, back, nearc, guard, large;
  unsigned long long launches;  // kernels enqueued by the calls (host-declared)
  unsigned long long clipped;   // triangles clipped at the near plane
  int32_t kernel_class;         // shading kernels of the last call (host-declared)
  int32_t pad1;
  unsigned long long reserved[21];
};
static_assert(sizeof(WsHeader) == 256, "header is 256 bytes");

// ----------------------------------------------------------------------------
// small helpers
// ----------------------------------------------------------------------------
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Fire-and-forget reductions (no value returned, so no wait on the result).
__device__ __forceinline__ void red_max_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.max.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// L2 eviction priority.  The fused forward + adjoint kernel streams, per
// view, ~2 GB of texel reads and FP32 gradient reductions and 36 MB of
// per-shell visibility words (k = 7 at 800^2) through the 129 MB L2.  A
// gradient texel's 128-byte line is reduced into by the neighbouring
// fragments of several shading rounds; the reductions mark it evict_last so
// that it stays in L2 between them instead of making another DRAM round trip.
// The visibility words and the texel reads of the adjoint keep the default
// priority.  (Measured on the C2 step against other assignments: words
// evict_last until an evict_first read, gradients normal -- 1.7 % slower;
// texel reads evict_first -- 11 % slower, evict_last -- 0.6 % slower.  The
// forward-only kernels keep texel lines evict_last: there they are the
// lines that neighbouring fragments reuse.)
__device__ __forceinline__ unsigned long long l2_evict_last() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void red_max_vis(unsigned long long* p, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.max.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void clear_vis2(uint4* p) { *p = make_uint4(0, 0, 0, 0); }
__device__ __forceinline__ void red_add_f32(float* p, float v) {
  asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add_v2f32(float* p, float a, float b) {
  asm volatile("red.relaxed.gpu.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}
// Gradient reductions (16 bytes of a gradient texel), evict_last (above).
__device__ __forceinline__ void red_add_v4f32(float* p, float a, float b, float c, float d) {
  asm volatile("red.relaxed.gpu.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(a),
               "f"(b), "f"(c), "f"(d), "l"(l2_evict_last())
               : "memory");
}

__device__ __forceinline__ void record_error(WsHeader* h, int code) {
  atomicCAS(&h->status, 0, code);
}

__device__ __forceinline__ void warp_count(unsigned long long* ctr, unsigned v) {
  v = __reduce_add_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(ctr, (unsigned long long)v);
}

// ----------------------------------------------------------------------------
// vertex stage: fixed FP32 transform, 1/256 px snap, depth key
// ----------------------------------------------------------------------------
// Each product and sum is rounded to FP32 in this order; the CPU oracle runs
// the same sequence, so the snapped integers agree bit for bit.
// World -> camera space (pinned FP32 sequence).
__device__ __forceinline__ float3 cam_xyz(const float* p, const DCam& c) {
  const float x = p[0], y = p[1], z = p[2];
  const float xc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c.m[0], x), __fmul_rn(c.m[1], y)),
                                       __fmul_rn(c.m[2], z)), c.m[3]);
  const float yc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c.m[4], x), __fmul_rn(c.m[5], y)),
                                       __fmul_rn(c.m[6], z)), c.m[7]);
  const float zc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c.m[8], x), __fmul_rn(c.m[9], y)),
                                       __fmul_rn(c.m[10], z)), c.m[11]);
  return make_float3(xc, yc, zc);
}

// Camera space (zc >= znear) -> (X, Y, bits(1/w), depth key), or the guard
// marker off the +-32768 px band.
__device__ __forceinline__ int4 project_cam(float xc, float yc, float zc, const DCam& c) {
  const float iw = __frcp_rn(zc);
  const float sx = __fadd_rn(__fmul_rn(__fmul_rn(c.fx, xc), iw), c.cx);
  const float sy = __fadd_rn(__fmul_rn(__fmul_rn(c.fy, yc), iw), c.cy);
  const float X = __fmul_rn(sx, 256.0f), Y = __fmul_rn(sy, 256.0f);
  if (!(fabsf(X) < 8388608.0f && fabsf(Y) < 8388608.0f)) return make_int4(kInvalidX, 0, 0, VTX_GUARD);
  const float qf = __fmul_rn(iw, __fmul_rn(c.znear, 1073741824.0f));
  return make_int4(__float2int_rn(X), __float2int_rn(Y), __float_as_int(iw), (int)__float2uint_rn(qf));
}

__device__ __forceinline__ int4 setup_vertex(const float* p, const DCam& c) {
  const float3 pc = cam_xyz(p, c);
  if (!(pc.z >= c.znear)) return make_int4(kInvalidX, 0, 0, VTX_NEAR);
  return project_cam(pc.x, pc.y, pc.z, c);
}

// ----------------------------------------------------------------------------
// triangle stage: integer edge functions, top-left rule, exact depth key
// ----------------------------------------------------------------------------
struct Tri {
  int X[3], Y[3];
  unsigned q[3];
  float iw[3];
  int tl[3];        // 1 if edge j (opposite vertex j) is a top or left edge
  int xlo, xhi, ylo, yhi;
};

// 0 = front-facing and valid; 1 = back-facing or zero area; 2 = every
// vertex nearer than znear; 3 = off the guard band; 5 = one or two vertices
// nearer than znear (to be clipped, clip_tri).
__device__ __forceinline__ int make_tri(const int4 v0, const int4 v1, const int4 v2, int W, int H,
                                        Tri& t) {
  if (v0.x == kInvalidX || v1.x == kInvalidX || v2.x == kInvalidX) {
    const int nn = (v0.x == kInvalidX && (v0.w & VTX_NEAR)) + (v1.x == kInvalidX && (v1.w & VTX_NEAR)) +
                   (v2.x == kInvalidX && (v2.w & VTX_NEAR));
    return nn == 3 ? 2 : (nn > 0 ? 5 : 3);
  }
  t.X[0] = v0.x; t.X[1] = v1.x; t.X[2] = v2.x;
  t.Y[0] = v0.y; t.Y[1] = v1.y; t.Y[2] = v2.y;
  const long long a2 = (long long)(t.X[1] - t.X[0]) * (t.Y[2] - t.Y[0]) -
                       (long long)(t.X[2] - t.X[0]) * (t.Y[1] - t.Y[0]);
  if (a2 >= 0) return 1;
  t.q[0] = (unsigned)v0.w; t.q[1] = (unsigned)v1.w; t.q[2] = (unsigned)v2.w;
  t.iw[0] = __int_as_float(v0.z); t.iw[1] = __int_as_float(v1.z); t.iw[2] = __int_as_float(v2.z);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int a = (j + 2) % 3, b = (j + 1) % 3;
    const int gx = t.Y[a] - t.Y[b];   // d e_j / d px
    const int gy = t.X[b] - t.X[a];   // d e_j / d py
    t.tl[j] = (gx > 0) || (gx == 0 && gy > 0);
  }
  const int mnx = min(t.X[0], min(t.X[1], t.X[2])), mxx = max(t.X[0], max(t.X[1], t.X[2]));
  const int mny = min(t.Y[0], min(t.Y[1], t.Y[2])), mxy = max(t.Y[0], max(t.Y[1], t.Y[2]));
  // pixel centres 256 x + 128 within [mn, mx]
  t.xlo = max(0, -((128 - mnx) >> 8));
  t.xhi = min(W - 1, (mxx - 128) >> 8);
  t.ylo = max(0, -((128 - mny) >> 8));
  t.yhi = min(H - 1, (mxy - 128) >> 8);
  return 0;
}

// Near-plane clipping of a mesh triangle with one or two vertices nearer
// than znear (the oracle's definition, same FP32 operations): in camera
// space, Sutherland-Hodgman against z = znear with the vertices in order;
// the point on a crossing edge comes from its (inside, outside) ends, t =
// (znear - z_out) / (z_in - z_out), x = x_out + t (x_in - x_out) (y and the
// UVs alike), z = znear, so triangles sharing the edge get the same point;
// the points are projected and snapped like vertices; the 3- or 4-gon is
// split into (P0, P1, P2) and (P0, P2, P3).  Returns the number of
// rasterizable parts (0..2) with their per-vertex UVs.  Rare: kept out of
// line so that the common path keeps its registers.
static __device__ __forceinline__ int clip_tri(const float* pos, const float2* uvs, const DCam& c, const int idx[3], Tri part[2],
                                     float2 puv[2][3]) {
  float3 pc[3];
  float2 uv[3];
  bool in[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    pc[j] = cam_xyz(pos + 3 * (size_t)idx[j], c);
    uv[j] = uvs ? __ldg(uvs + idx[j]) : make_float2(0.f, 0.f);
    in[j] = pc[j].z >= c.znear;
  }
  int4 pv[4];
  float2 pu[4];
  int n = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int b = (a + 1) % 3;
    if (in[a]) {
      pv[n] = project_cam(pc[a].x, pc[a].y, pc[a].z, c);
      pu[n] = uv[a];
      ++n;
    }
    if (in[a] != in[b]) {
      const int i = in[a] ? a : b, o = in[a] ? b : a;
      const float t = __fdiv_rn(__fsub_rn(c.znear, pc[o].z), __fsub_rn(pc[i].z, pc[o].z));
      const float x = __fadd_rn(pc[o].x, __fmul_rn(t, __fsub_rn(pc[i].x, pc[o].x)));
      const float y = __fadd_rn(pc[o].y, __fmul_rn(t, __fsub_rn(pc[i].y, pc[o].y)));
      const float u = __fadd_rn(uv[o].x, __fmul_rn(t, __fsub_rn(uv[i].x, uv[o].x)));
      const float w = __fadd_rn(uv[o].y, __fmul_rn(t, __fsub_rn(uv[i].y, uv[o].y)));
      pv[n] = project_cam(x, y, c.znear, c);
      pu[n] = make_float2(u, w);
      ++n;
    }
  }
  int m = 0;
  if (n >= 3 && make_tri(pv[0], pv[1], pv[2], c.W, c.H, part[m]) == 0) {
    puv[m][0] = pu[0]; puv[m][1] = pu[1]; puv[m][2] = pu[2];
    ++m;
  }
  if (n == 4 && make_tri(pv[0], pv[2], pv[3], c.W, c.H, part[m]) == 0) {
    puv[m][0] = pu[0]; puv[m][1] = pu[2]; puv[m][2] = pu[3];
    ++m;
  }
  return m;
}

__device__ __forceinline__ void edge_values(const Tri& t, int px, int py, long long e[3]) {
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int a = (j + 2) % 3, b = (j + 1) % 3;
    e[j] = (long long)(t.X[b] - t.X[a]) * (py - t.Y[a]) - (long long)(t.Y[b] - t.Y[a]) * (px - t.X[a]);
  }
}

__device__ __forceinline__ bool covered(const Tri& t, const long long e[3]) {
  return (e[0] + t.tl[0] > 0) && (e[1] + t.tl[1] > 0) && (e[2] + t.tl[2] > 0);
}

// floor(sum_j e_j q_j / S) exactly, S = sum_j e_j, for e_j >= 0 (S > 0,
// S < 2^51) and q_j < 2^31; rS ~ 1/S in FP32.  The quotient lies between min
// q and max q, so it fits in 32 bits; the FP32 estimate (a sum of positive
// terms, relative error ~6 ulp) is within ~2^10 of it, which bounds the
// residual R = N - Q S below 2^62 and lets R be computed exactly in
// wrapping 64-bit arithmetic; two correction steps make the quotient exact.
__device__ __forceinline__ unsigned depth_key_r(const unsigned q[3], const long long e[3],
                                                unsigned long long S, float rS) {
  const unsigned long long N = (unsigned long long)e[0] * q[0] + (unsigned long long)e[1] * q[1] +
                               (unsigned long long)e[2] * q[2];   // mod 2^64
  const float est = fmaf((float)e[0], (float)q[0],
                         fmaf((float)e[1], (float)q[1], (float)e[2] * (float)q[2])) * rS;
  const unsigned qmin = min(q[0], min(q[1], q[2])), qmax = max(q[0], max(q[1], q[2]));
  unsigned Q = (unsigned)fminf(fmaxf(est, (float)qmin), (float)qmax);
  Q = min(max(Q, qmin), qmax);
  long long R = (long long)(N - (unsigned long long)Q * S);
  Q = (unsigned)((long long)Q + (long long)floorf((float)R * rS));
  R = (long long)(N - (unsigned long long)Q * S);
#pragma unroll 1
  for (int i = 0; i < 4 && R < 0; ++i) { --Q; R += (long long)S; }
#pragma unroll 1
  for (int i = 0; i < 4 && R >= (long long)S; ++i) { ++Q; R -= (long long)S; }
  return Q;
}

__device__ __forceinline__ unsigned depth_key(const Tri& t, const long long e[3]) {
  const unsigned long long S = (unsigned long long)(e[0] + e[1] + e[2]);
  return depth_key_r(t.q, e, S, 1.0f / (float)S);
}

__device__ __forceinline__ unsigned long long vis_key(unsigned K, int tri) {
  return ((unsigned long long)K << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)tri);
}

__device__ __forceinline__ int vis_tri(unsigned long long key) {
  return key ? (int)(0xFFFFFFFFu - (unsigned)(key & 0xFFFFFFFFull)) : -1;
}

// The triangle of a visibility word from its low 32 bits alone (the word is
// little-endian, so they sit at its address): an empty word is 0, and a
// written one holds ~triangle there, which is never 0 because triangle ids
// stay below 2^31.  Half the registers of loading the whole word.
__device__ __forceinline__ int load_vis_tri(const unsigned long long* p) {
  const unsigned lo = __ldcg(reinterpret_cast<const unsigned*>(p));
  return lo ? (int)(0xFFFFFFFFu - lo) : -1;
}

// ----------------------------------------------------------------------------
// float-float arithmetic (Dekker 1971 / Knuth TAOCP 4.2.2): used for UV
// interpolation over triangles that span many texels
// ----------------------------------------------------------------------------
struct ff { float hi, lo; };

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff quick_two_sum(float a, float b) {   // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  ff t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = quick_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  ff p = two_prod(a.hi, b.hi);
  p.lo = __fadd_rn(p.lo, __fadd_rn(__fmul_rn(a.hi, b.lo), __fmul_rn(a.lo, b.hi)));
  return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  ff p = two_prod(a.hi, b);
  p.lo = __fadd_rn(p.lo, __fmul_rn(a.lo, b));
  return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ff ll_to_ff(long long v) {
  const float hi = __ll2float_rn(v);
  const float lo = __ll2float_rn(v - __float2ll_rn(hi));
  return {hi, lo};
}
__device__ __forceinline__ ff int_to_ff(int v) {   // the same split for |v| < 2^31
  const float hi = __int2float_rn(v);
  const float lo = __int2float_rn(v - __float2int_rn(hi));
  return {hi, lo};
}
// a / b with rb = 1/b.hi rounded: the quotient estimate and one correction
// step on the float-float remainder (relative error near 2^-44).
__device__ __forceinline__ ff ff_div_r(ff a, ff b, float rb) {
  const float q1 = __fmul_rn(a.hi, rb);
  const ff r = ff_add(a, ff_mul_f({-b.hi, -b.lo}, q1));
  const float q2 = __fmul_rn(r.hi, rb);
  return quick_two_sum(q1, q2);
}

// ----------------------------------------------------------------------------
// attribute interpolation and the bilinear footprint
// ----------------------------------------------------------------------------
struct Footprint {
  int x0, x1, y0, y1;  // clamped tap columns / rows
  float fx, fy;        // weight of column x1 / row y1
};

// Integer part and fraction of (X0 - 1/2) + delta, with delta given as a
// float-float; the fraction is returned rounded to FP32.
__device__ __forceinline__ void split_coord(float X0, ff delta, int& i, float& f) {
  const float a = __fsub_rn(X0, 0.5f);
  const float base = floorf(a);
  const float frac0 = __fsub_rn(a, base);          // exact, in [0, 1)
  ff s = ff_add({frac0, 0.0f}, delta);
  float fl = floorf(s.hi);
  if (s.hi == fl && s.lo < 0.0f) fl = __fsub_rn(fl, 1.0f);
  f = __fadd_rn(__fsub_rn(s.hi, fl), s.lo);
  if (f >= 1.0f) { f = __fsub_rn(f, 1.0f); fl = __fadd_rn(fl, 1.0f); }
  if (f < 0.0f) f = 0.0f;
  i = (int)base + (int)fl;
}

// Same for a plain FP32 delta of a few texels at most: the sum with the
// fraction in [0, 1) keeps an absolute error below 2^-20 texel.
__device__ __forceinline__ void split_coord_f(float X0, float delta, int& i, float& f) {
  const float a = __fsub_rn(X0, 0.5f);
  const float base = floorf(a);
  const float s = __fadd_rn(__fsub_rn(a, base), delta);
  const float fl = floorf(s);
  f = __fsub_rn(s, fl);
  i = (int)base + (int)fl;
}

// Perspective-correct UV of pixel centre (px, py) mapped to texel space
// (x = u W - 1/2, y = v H - 1/2), interpolated relative to vertex 0, as an
// integer part and a fraction (unclamped).  Three paths by the triangle's
// span in texels: up to 8, plain FP32 (error ~10 2^-24 span); up to 32 with
// edge values below 2^24, one rounding per weight and error-free
// transformations after it (error <= 2 2^-24 span); beyond, float-float.
__device__ __forceinline__ void texel_coords(const Tri& t, const float2 uv[3], int tw, int th, int px, int py,
                                             int& ix, float& fx, int& iy, float& fy) {
  // exact edge values at the pixel: 32-bit arithmetic when every vertex lies
  // within 2^14 units (64 px) of it (products below 2^29), else 64-bit; the
  // same integers either way
  bool near = true;
#pragma unroll
  for (int j = 0; j < 3; ++j)
    near = near && abs(t.X[j] - px) < (1 << 14) && abs(t.Y[j] - py) < (1 << 14);
  int e32[3];
  long long e[3];
  if (near) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int a = (j + 2) % 3, b = (j + 1) % 3;
      e32[j] = (t.X[b] - t.X[a]) * (py - t.Y[a]) - (t.Y[b] - t.Y[a]) * (px - t.X[a]);
      e[j] = e32[j];
    }
  } else {
    edge_values(t, px, py, e);
  }
  const float W = (float)tw, H = (float)th;
  const float X0 = __fmul_rn(uv[0].x, W), X1 = __fmul_rn(uv[1].x, W), X2 = __fmul_rn(uv[2].x, W);
  const float Y0 = __fmul_rn(uv[0].y, H), Y1 = __fmul_rn(uv[1].y, H), Y2 = __fmul_rn(uv[2].y, H);
  const float d1x = __fsub_rn(X1, X0), d2x = __fsub_rn(X2, X0);
  const float d1y = __fsub_rn(Y1, Y0), d2y = __fsub_rn(Y2, Y0);
  const float span = fmaxf(fmaxf(fabsf(d1x), fabsf(d2x)), fmaxf(fabsf(d1y), fabsf(d2y)));
  if (span <= 8.0f) {
    float ef[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) ef[j] = near ? __int2float_rn(e32[j]) : __ll2float_rn(e[j]);
    const float w0 = __fmul_rn(ef[0], t.iw[0]);
    const float w1 = __fmul_rn(ef[1], t.iw[1]);
    const float w2 = __fmul_rn(ef[2], t.iw[2]);
    const float rD = __fdividef(1.0f, __fadd_rn(__fadd_rn(w0, w1), w2));
    const float l1 = __fmul_rn(w1, rD), l2 = __fmul_rn(w2, rD);
    split_coord_f(X0, __fmaf_rn(l1, d1x, __fmul_rn(l2, d2x)), ix, fx);
    split_coord_f(Y0, __fmaf_rn(l1, d1y, __fmul_rn(l2, d2y)), iy, fy);
  } else if (span <= 32.0f && near && abs(e32[0]) < (1 << 24) && abs(e32[1]) < (1 << 24) &&
             abs(e32[2]) < (1 << 24)) {
    // Edge values below 2^24 convert to float exactly, so each weight
    // w_j = e_j (1/w_j) carries one rounding (relative 2^-24); everything
    // after it -- the sum of the weights, the vertex differences, the
    // numerators and the quotient with one correction step -- is kept to
    // ~2^-44 by error-free transformations.  The weights' roundings move
    // the offset by at most 2 * 2^-24 * span: 2^-18 texel at span 32.
    const float w0 = __fmul_rn(__int2float_rn(e32[0]), t.iw[0]);
    const float w1 = __fmul_rn(__int2float_rn(e32[1]), t.iw[1]);
    const float w2 = __fmul_rn(__int2float_rn(e32[2]), t.iw[2]);
    const ff s01 = two_sum(w0, w1);
    const ff s012 = two_sum(s01.hi, w2);
    const float Sh = s012.hi, Sl = __fadd_rn(s012.lo, s01.lo);
    const float r = __frcp_rn(Sh);
    auto offset = [&](float A0, float A1, float A2) {
      const ff d1 = two_sum(A1, -A0), d2 = two_sum(A2, -A0);
      const ff p1 = two_prod(w1, d1.hi), p2 = two_prod(w2, d2.hi);
      const ff nh = two_sum(p1.hi, p2.hi);
      const float nl = __fmaf_rn(w2, d2.lo, __fmaf_rn(w1, d1.lo, __fadd_rn(__fadd_rn(nh.lo, p1.lo), p2.lo)));
      const float q = __fmul_rn(nh.hi, r);
      const float rem = __fadd_rn(__fmaf_rn(-q, Sh, nh.hi), __fsub_rn(nl, __fmul_rn(q, Sl)));
      return quick_two_sum(q, __fmul_rn(rem, r));
    };
    split_coord(X0, offset(X0, X1, X2), ix, fx);
    split_coord(Y0, offset(Y0, Y1, Y2), iy, fy);
  } else {
    ff ee[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) ee[j] = near ? int_to_ff(e32[j]) : ll_to_ff(e[j]);
    const ff w0 = ff_mul_f(ee[0], t.iw[0]);
    const ff w1 = ff_mul_f(ee[1], t.iw[1]);
    const ff w2 = ff_mul_f(ee[2], t.iw[2]);
    const ff D = ff_add(ff_add(w0, w1), w2);
    const float rD = __frcp_rn(D.hi);
    const ff ex1 = two_sum(X1, -X0), ex2 = two_sum(X2, -X0);
    const ff ey1 = two_sum(Y1, -Y0), ey2 = two_sum(Y2, -Y0);
    split_coord(X0, ff_div_r(ff_add(ff_mul(w1, ex1), ff_mul(w2, ex2)), D, rD), ix, fx);
    split_coord(Y0, ff_div_r(ff_add(ff_mul(w1, ey1), ff_mul(w2, ey2)), D, rD), iy, fy);
  }
}

// The two taps per axis, clamped to the image (clamp-to-edge).
__device__ __forceinline__ Footprint clamp_footprint(int ix, float fx, int iy, float fy, int w, int h) {
  Footprint f;
  f.fx = fx;
  f.fy = fy;
  f.x0 = min(max(ix, 0), w - 1);
  f.x1 = min(max(ix + 1, 0), w - 1);
  f.y0 = min(max(iy, 0), h - 1);
  f.y1 = min(max(iy + 1, 0), h - 1);
  return f;
}

// Bilinear footprint (taps and weights) of pixel centre (px, py).
__device__ __forceinline__ Footprint footprint(const Tri& t, const float2 uv[3], int tw, int th, int px, int py) {
  int ix, iy;
  float fx, fy;
  texel_coords(t, uv, tw, th, px, py, ix, fx, iy, fy);
  return clamp_footprint(ix, fx, iy, fy, tw, th);
}

// Texel coordinate of an image 2^s times smaller: from X = ix + fx at full
// resolution, X' = (X + 1/2) / 2^s - 1/2 = q + (m + 1/2 + fx) / 2^s - 1/2 with
// ix = q 2^s + m.  The sum m + 1/2 + fx < 2^s + 1 loses at most s bits of fx,
// which the division by 2^s gives back: the fraction keeps about 2^-24.
__device__ __forceinline__ void coarser_coord(int ix, float fx, int s, int& ixs, float& fxs) {
  if (s == 0) {
    ixs = ix;
    fxs = fx;
    return;
  }
  const int q = ix >> s;                     // floor division (arithmetic shift)
  const int m = ix - (q << s);
  const float t = __fmul_rn(__fadd_rn(__fadd_rn((float)m, 0.5f), fx), __int_as_float((127 - s) << 23)) - 0.5f;
  const float fl = floorf(t);
  ixs = q + (int)fl;
  fxs = __fsub_rn(t, fl);
}

// ----------------------------------------------------------------------------
// real spherical harmonics, l <= 3 (orthonormal; l = 1 band ~ (y, z, x))
// Constants are the closed-form normalisations:
//   0.2820947917738782 = 1/(2 sqrt(pi))        0.4886025119029199 = sqrt(3/(4 pi))
//   1.0925484305920792 = sqrt(15/pi)/2          0.31539156525252005 = sqrt(5/pi)/4
//   0.5462742152960396 = sqrt(15/pi)/4          0.5900435899266435 = sqrt(35/(2 pi))/4
//   2.890611442640554  = sqrt(105/pi)/2         0.4570457994644658 = sqrt(21/(2 pi))/4
//   0.3731763325901154 = sqrt(7/pi)/4           1.445305721320277  = sqrt(105/pi)/4
// ----------------------------------------------------------------------------
__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float Y[16]) {
  Y[0] = 0.2820947917738782f;
  if (deg < 1) return;
  Y[1] = 0.4886025119029199f * y;
  Y[2] = 0.4886025119029199f * z;
  Y[3] = 0.4886025119029199f * x;
  if (deg < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = 1.0925484305920792f * (x * y);
  Y[5] = 1.0925484305920792f * (y * z);
  Y[6] = 0.31539156525252005f * (2.0f * zz - xx - yy);
  Y[7] = 1.0925484305920792f * (x * z);
  Y[8] = 0.5462742152960396f * (xx - yy);
  if (deg < 3) return;
  Y[9] = 0.5900435899266435f * y * (3.0f * xx - yy);
  Y[10] = 2.890611442640554f * (x * y) * z;
  Y[11] = 0.4570457994644658f * y * (4.0f * zz - xx - yy);
  Y[12] = 0.3731763325901154f * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
  Y[13] = 0.4570457994644658f * x * (4.0f * zz - xx - yy);
  Y[14] = 1.445305721320277f * z * (xx - yy);
  Y[15] = 0.5900435899266435f * x * (xx - 3.0f * yy);
}

__device__ __forceinline__ float sigmoidf_(float x) { return __fdividef(1.0f, 1.0f + __expf(-x)); }

// Unit world-space ray direction through pixel (x, y).
__device__ __forceinline__ float3 ray_dir(const DCam& c, int x, int y) {
  const float a = ((float)x + 0.5f - c.cx) * c.rfx;
  const float b = ((float)y + 0.5f - c.cy) * c.rfy;
  // world = R^T (a, b, 1)
  float vx = c.m[0] * a + c.m[4] * b + c.m[8];
  float vy = c.m[1] * a + c.m[5] * b + c.m[9];
  float vz = c.m[2] * a + c.m[6] * b + c.m[10];
  const float r = rsqrtf(vx * vx + vy * vy + vz * vz);
  return make_float3(vx * r, vy * r, vz * r);
}

// Transparency attenuation (Sec. 3): alpha_w = 2 sigmoid(10 |v . n|) - 1 for
// unit ray direction v and the unit normal n of the hit face, taken as the
// flat normal (p1 - p0) x (p2 - p0) of the stored triangle.  Grazing rays
// (v . n -> 0) give alpha_w -> 0, head-on rays 2 sigmoid(10) - 1.
// (p1 - p0) x (p2 - p0) of the stored positions of a face (unnormalised).
__device__ __forceinline__ float3 face_cross(const float* pos, const int idx[3]) {
  float p[3][3];
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int d = 0; d < 3; ++d) p[j][d] = __ldg(pos + 3 * (size_t)idx[j] + d);
  const float ax = p[1][0] - p[0][0], ay = p[1][1] - p[0][1], az = p[1][2] - p[0][2];
  const float bx = p[2][0] - p[0][0], by = p[2][1] - p[0][1], bz = p[2][2] - p[0][2];
  return make_float3(ay * bz - az * by, az * bx - ax * bz, ax * by - ay * bx);
}

__device__ __forceinline__ float alpha_atten(const float* pos, const int idx[3], const float3 v) {
  const float3 n = face_cross(pos, idx);
  const float n2 = n.x * n.x + n.y * n.y + n.z * n.z;
  // a face with a projected area has a nonzero normal; guard the rounding case
  const float vn = n2 > 0.0f ? fabsf(n.x * v.x + n.y * v.y + n.z * v.z) * rsqrtf(n2) : 0.0f;
  return 2.0f * sigmoidf_(10.0f * vn) - 1.0f;
}

// ----------------------------------------------------------------------------
// texel fetch + decode.  NCH values per texel, loaded VEC at a time.
// ----------------------------------------------------------------------------
// KEEP: the load marks its L2 line evict_last (the forward-only kernels,
// where texel lines are what neighbouring fragments reuse; measured on the
// C2 forward batch: 2 % faster).  The 256-bit loads do not allocate in L1:
// a texel line is rarely read twice by one SM, and the L1 then keeps the
// triangle indices, snapped vertices and UVs that neighbouring fragments
// share and that every fragment's dependent loads wait for (C2: fused step
// -1.5 %, forward -3.3 %; L1::evict_first instead: +0.2 % / +0.6 %).
template <int VEC, bool KEEP = false>
__device__ __forceinline__ void load_halves(const __half* p, float* out) {
  if constexpr (VEC == 16) {   // one 256-bit load (32-byte aligned)
    unsigned r[8];
    if constexpr (KEEP)
      asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8], %9;"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
          : "l"(p), "l"(l2_evict_last()));
    else
      asm("ld.global.nc.L1::no_allocate.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
          : "l"(p));
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&r[i]));
      out[2 * i] = f.x;
      out[2 * i + 1] = f.y;
    }
  } else if constexpr (VEC == 8) {
    uint4 r;
    if constexpr (KEEP)
      asm("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
          : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
          : "l"(p), "l"(l2_evict_last()));
    else
      r = __ldg(reinterpret_cast<const uint4*>(p));
    const __half2* h = reinterpret_cast<const __half2*>(&r);
#pragma unroll
    for (int i = 0; i < 4; ++i) { float2 f = __half22float2(h[i]); out[2 * i] = f.x; out[2 * i + 1] = f.y; }
  } else if constexpr (VEC == 4) {
    const uint2 r = __ldg(reinterpret_cast<const uint2*>(p));
    const __half2* h = reinterpret_cast<const __half2*>(&r);
#pragma unroll
    for (int i = 0; i < 2; ++i) { float2 f = __half22float2(h[i]); out[2 * i] = f.x; out[2 * i + 1] = f.y; }
  } else if constexpr (VEC == 2) {
    const unsigned r = __ldg(reinterpret_cast<const unsigned*>(p));
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&r));
    out[0] = f.x; out[1] = f.y;
  } else {
    out[0] = __half2float(__ldg(p));
  }
}

// Bilinear mix of the 4 taps' NCH values (fp16 storage), FP32 accumulate.
template <int NCH, int VEC, bool KEEP = false>
__device__ __forceinline__ void bilinear_f16(const __half* tex, int tw, int pitch, const Footprint& f,
                                             float val[NCH]) {
  const float w00 = (1.0f - f.fx) * (1.0f - f.fy), w10 = f.fx * (1.0f - f.fy);
  const float w01 = (1.0f - f.fx) * f.fy, w11 = f.fx * f.fy;
  const __half* p00 = tex + ((size_t)f.y0 * tw + f.x0) * pitch;
  const __half* p10 = tex + ((size_t)f.y0 * tw + f.x1) * pitch;
  const __half* p01 = tex + ((size_t)f.y1 * tw + f.x0) * pitch;
  const __half* p11 = tex + ((size_t)f.y1 * tw + f.x1) * pitch;
  constexpr int NL = (NCH + VEC - 1) / VEC;
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    float a[VEC], b[VEC], c[VEC], d[VEC];
    load_halves<VEC, KEEP>(p00 + l * VEC, a);
    load_halves<VEC, KEEP>(p10 + l * VEC, b);
    load_halves<VEC, KEEP>(p01 + l * VEC, c);
    load_halves<VEC, KEEP>(p11 + l * VEC, d);
#pragma unroll
    for (int i = 0; i < VEC; ++i) {
      const int ch = l * VEC + i;
      if (ch < NCH) val[ch] = fmaf(w11, d[i], fmaf(w01, c[i], fmaf(w10, b[i], w00 * a[i])));
    }
  }
}

template <int VEC>
__device__ __forceinline__ void bilinear_rgba(const float* tex, int tw, int pitch, const Footprint& f,
                                              float val[4]) {
  const float w00 = (1.0f - f.fx) * (1.0f - f.fy), w10 = f.fx * (1.0f - f.fy);
  const float w01 = (1.0f - f.fx) * f.fy, w11 = f.fx * f.fy;
  const float* p[4] = {tex + ((size_t)f.y0 * tw + f.x0) * pitch, tex + ((size_t)f.y0 * tw + f.x1) * pitch,
                       tex + ((size_t)f.y1 * tw + f.x0) * pitch, tex + ((size_t)f.y1 * tw + f.x1) * pitch};
  float t[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if constexpr (VEC == 4) {
      const float4 r = __ldg(reinterpret_cast<const float4*>(p[q]));
      t[q][0] = r.x; t[q][1] = r.y; t[q][2] = r.z; t[q][3] = r.w;
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) t[q][i] = __ldg(p[q] + i);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) val[i] = fmaf(w11, t[3][i], fmaf(w01, t[2][i], fmaf(w10, t[1][i], w00 * t[0][i])));
}

// Fragment colour and opacity.
struct Frag {
  float r, g, b, a;
};

template <int DEG>
__device__ __forceinline__ Frag decode_sh(const float* val, const float Y[16]) {
  constexpr int NB = (DEG + 1) * (DEG + 1);
  float z[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int m = 0; m < NB; ++m) {
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) z[ch] = fmaf(val[1 + 3 * m + ch], Y[m], z[ch]);
  }
  return {sigmoidf_(z[0]), sigmoidf_(z[1]), sigmoidf_(z[2]), sigmoidf_(val[0])};
}

// ----------------------------------------------------------------------------
// baked texels (VS_TEX_SH_U8): RGBA SH bytes, band l at (tw, th) >> l * bshift
// ----------------------------------------------------------------------------
// Byte c of w as a float, exactly: the byte placed under the exponent of
// 2^23 (one byte permute: 0x4B0000bb is 2^23 + bb) minus 2^23 -- no
// integer-to-float conversion (a quarter-rate instruction) per byte.
__device__ __forceinline__ float byte_of(unsigned w, int c) {
  return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u | (unsigned)c)) - 8388608.0f;
}

// Band L of a baked texel at full-resolution texel coordinate (ix + fx,
// iy + fy): the band's own footprint, its 2L + 1 coefficient quadruples
// bilinearly combined, decoded (vmin + vscale q) and added into
// z_c += value * Y_m.
template <int L>
__device__ __forceinline__ void baked_band(const DShell& s, int ix, float fx, int iy, float fy, const float Y[16],
                                           float z[4]) {
  constexpr int NC = 2 * L + 1;
  constexpr int STRIDE = L == 0 ? 4 : (L == 1 ? 16 : 32);
  const int sh = L * s.bshift;
  int bx, by;
  float bfx, bfy;
  coarser_coord(ix, fx, sh, bx, bfx);
  coarser_coord(iy, fy, sh, by, bfy);
  const int w = s.tw >> sh, h = s.th >> sh;
  const Footprint f = clamp_footprint(bx, bfx, by, bfy, w, h);
  const float w00 = (1.0f - f.fx) * (1.0f - f.fy), w10 = f.fx * (1.0f - f.fy);
  const float w01 = (1.0f - f.fx) * f.fy, w11 = f.fx * f.fy;
  const unsigned char* base = reinterpret_cast<const unsigned char*>(s.tex) + s.boff[L];
  const unsigned char* p[4] = {base + ((size_t)f.y0 * w + f.x0) * STRIDE, base + ((size_t)f.y0 * w + f.x1) * STRIDE,
                               base + ((size_t)f.y1 * w + f.x0) * STRIDE, base + ((size_t)f.y1 * w + f.x1) * STRIDE};
  unsigned q[4][8];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if constexpr (L == 0) {
      q[t][0] = __ldg(reinterpret_cast<const unsigned*>(p[t]));
    } else {
      const uint4 a = __ldg(reinterpret_cast<const uint4*>(p[t]));
      q[t][0] = a.x; q[t][1] = a.y; q[t][2] = a.z; q[t][3] = a.w;
      if constexpr (L >= 2) {
        const uint4 b = __ldg(reinterpret_cast<const uint4*>(p[t]) + 1);
        q[t][4] = b.x; q[t][5] = b.y; q[t][6] = b.z; q[t][7] = b.w;
      }
    }
  }
#pragma unroll
  for (int m = 0; m < NC; ++m)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float b = fmaf(w11, byte_of(q[3][m], c),
                           fmaf(w01, byte_of(q[2][m], c), fmaf(w10, byte_of(q[1][m], c), w00 * byte_of(q[0][m], c))));
      const float val = fmaf(s.vscale, b, s.vmin);
      z[c] = fmaf(val, Y[L * L + m], z[c]);
    }
}

// Colour and opacity of a baked fragment: every channel is
// sigmoid(sum_m sh_{m,c} Y_m(v)) (opacity view dependent too).
template <int DEG>
__device__ __forceinline__ Frag fetch_baked(const DShell& s, int ix, float fx, int iy, float fy, const float Y[16]) {
  float z[4] = {0.f, 0.f, 0.f, 0.f};
  baked_band<0>(s, ix, fx, iy, fy, Y, z);
  if constexpr (DEG >= 1) baked_band<1>(s, ix, fx, iy, fy, Y, z);
  if constexpr (DEG >= 2) baked_band<2>(s, ix, fx, iy, fy, Y, z);
  if constexpr (DEG >= 3) baked_band<3>(s, ix, fx, iy, fy, Y, z);
  return {sigmoidf_(z[0]), sigmoidf_(z[1]), sigmoidf_(z[2]), sigmoidf_(z[3])};
}

// ----------------------------------------------------------------------------
// gradient scatter: dval (NCH values) * tap weight into 4 texels
// ----------------------------------------------------------------------------
template <int NCH, int GV>
__device__ __forceinline__ void scatter_grad(float* grad, int tw, int pitch, const Footprint& f,
                                             const float* dval) {
  const float w[4] = {(1.0f - f.fx) * (1.0f - f.fy), f.fx * (1.0f - f.fy), (1.0f - f.fx) * f.fy,
                      f.fx * f.fy};
  const int xs[4] = {f.x0, f.x1, f.x0, f.x1}, ys[4] = {f.y0, f.y0, f.y1, f.y1};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float* g = grad + ((size_t)ys[q] * tw + xs[q]) * pitch;
    constexpr int NL = (NCH + GV - 1) / GV;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      if constexpr (GV == 4) {
        red_add_v4f32(g + 4 * l, w[q] * dval[4 * l],
                      (4 * l + 1 < NCH) ? w[q] * dval[4 * l + 1] : 0.0f,
                      (4 * l + 2 < NCH) ? w[q] * dval[4 * l + 2] : 0.0f,
                      (4 * l + 3 < NCH) ? w[q] * dval[4 * l + 3] : 0.0f);
      } else if constexpr (GV == 2) {
        red_add_v2f32(g + 2 * l, w[q] * dval[2 * l], (2 * l + 1 < NCH) ? w[q] * dval[2 * l + 1] : 0.0f);
      } else {
        red_add_f32(g + l, w[q] * dval[l]);
      }
    }
  }
}

}  // namespace vsd
