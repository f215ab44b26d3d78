// Kernels of the k-shell renderer (sm_103a): per-phase kernels for the plain
// per-view path and the persistent multi-item kernel, built from the same
// device functions.
//
// Phases of one (object, view) item -- the hot path of the paper's baked
// real-time renderer (Sec. 3 "Baking Textures": rasterize every mesh in a
// fixed order and blend in the frame buffer) and of its texture fitting
// (Sec. 3 "Texturing Meshes"):
//   SETUP  clear the per-shell visibility words; transform + snap vertices
//   RASTER one thread per triangle: cull, edge functions, exact depth key,
//          64-bit atomicMax (key << 32 | ~triangle) per (shell, pixel):
//          nearest hit per shell, ties to the lower triangle (Fig. 3c);
//          triangles with large screen boxes are queued for LARGE
//   LARGE  one warp per queued triangle, lanes over its box
//   SHADE  one thread per pixel: per shell in order, perspective-correct UV,
//          bilinear fetch at texel centres (Fig. 5), SH decode with the ray
//          direction, front-to-back over (Eq. 6 with Eq. 1's
//          transmittance); optionally the adjoint w.r.t. texels.

#include <cuda_runtime.h>

#include "vs_device.cuh"
#include "vs_kernels.h"

namespace vsd {

// ----------------------------------------------------------------------------
// SETUP
// ----------------------------------------------------------------------------
__device__ void unit_setup(const DItem& it, const DShell* sh, int u) {
  if (u < it.clear_units) {
    const size_t total = (size_t)it.k * it.cam.W * it.cam.H;
    const size_t beg = (size_t)u * kClearPerUnit;
    const size_t end = min(total, beg + (size_t)kClearPerUnit);
    uint4* p = reinterpret_cast<uint4*>(it.vis + beg);
    const size_t n2 = (end - beg) >> 1;
    for (size_t i = threadIdx.x; i < n2; i += blockDim.x) p[i] = make_uint4(0, 0, 0, 0);
    if (((end - beg) & 1) && threadIdx.x == 0) it.vis[end - 1] = 0ull;
    if (u == 0 && (int)threadIdx.x < it.k) it.large_count[threadIdx.x] = 0;
    return;
  }
  u -= it.clear_units;
  int i = 0;
  while (i + 1 < it.k && u >= it.setup_pre[i + 1]) ++i;
  const DShell& s = sh[i];
  const int v0 = (u - it.setup_pre[i]) * kSetupPerUnit;
  const int v1 = min(v0 + kSetupPerUnit, s.nv);
  for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) s.vsetup[v] = setup_vertex(s.pos + 3 * (size_t)v, it.cam);
}

// ----------------------------------------------------------------------------
// RASTER / LARGE
// ----------------------------------------------------------------------------
// Loads triangle t of shell s; 0 = front-facing and rasterizable, 1..3 =
// culled (back/zero-area, near, guard band), 4 = index out of range.
__device__ __forceinline__ int load_tri(const DShell& s, const DCam& c, int t, Tri& T) {
  const int* ip = s.tris + 3 * (size_t)t;
  const int i0 = __ldg(ip), i1 = __ldg(ip + 1), i2 = __ldg(ip + 2);
  if ((unsigned)i0 >= (unsigned)s.nv || (unsigned)i1 >= (unsigned)s.nv || (unsigned)i2 >= (unsigned)s.nv) return 4;
  return make_tri(__ldcg(s.vsetup + i0), __ldcg(s.vsetup + i1), __ldcg(s.vsetup + i2), c.W, c.H, T);
}

__device__ __forceinline__ void raster_pixel(const Tri& T, int t, int x, int y, int W, unsigned long long* vis) {
  long long e[3];
  edge_values(T, 256 * x + 128, 256 * y + 128, e);
  if (covered(T, e)) atomicMax(vis + (size_t)y * W + x, vis_key(depth_key(T, e), t));
}

__device__ void unit_raster(const DItem& it, const DShell* sh, int u, WsHeader* hdr) {
  int i = 0;
  while (i + 1 < it.k && u >= it.raster_pre[i + 1]) ++i;
  const DShell& s = sh[i];
  const int t = (u - it.raster_pre[i]) * kRasterPerUnit + threadIdx.x;
  const int W = it.cam.W, H = it.cam.H;
  unsigned front = 0, back = 0, nearc = 0, guard = 0, large = 0, bad = 0;
  if (t < s.nt) {
    Tri T;
    const int why = load_tri(s, it.cam, t, T);
    if (why == 0) {
      front = 1;
      const int bw = T.xhi - T.xlo + 1, bh = T.yhi - T.ylo + 1;
      if (bw > 0 && bh > 0) {
        unsigned long long* vis = it.vis + (size_t)i * W * H;
        if (bw * bh <= kSmallMaxPixels) {
          for (int y = T.ylo; y <= T.yhi; ++y)
            for (int x = T.xlo; x <= T.xhi; ++x) raster_pixel(T, t, x, y, W, vis);
        } else {
          large = 1;
          const int slot = atomicAdd(it.large_count + i, 1);
          if (slot < s.nt) s.large[slot] = t;
        }
      }
    } else if (why == 1) back = 1;
    else if (why == 2) nearc = 1;
    else if (why == 3) guard = 1;
    else bad = 1;
  }
  warp_count(&hdr->front, front);
  warp_count(&hdr->back, back);
  warp_count(&hdr->nearc, nearc);
  warp_count(&hdr->guard, guard);
  warp_count(&hdr->large, large);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) record_error(hdr, VS_ERR_INVALID_ARG);
}

__device__ void unit_large(const DItem& it, const DShell* sh, int u) {
  const int NW = kLargeUnits * (kThreads / 32);
  const int gw = u * (kThreads / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int W = it.cam.W, H = it.cam.H;
  for (int i = 0; i < it.k; ++i) {
    const DShell& s = sh[i];
    const int n = min(__ldcg(it.large_count + i), s.nt);
    unsigned long long* vis = it.vis + (size_t)i * W * H;
    for (int b = gw; b < n; b += NW) {
      const int t = __ldcg(s.large + b);
      Tri T;
      if (load_tri(s, it.cam, t, T) != 0) continue;
      const int bw = T.xhi - T.xlo + 1, bh = T.yhi - T.ylo + 1;
      const int npx = bw * bh;
      for (int p = lane; p < npx; p += 32) raster_pixel(T, t, T.xlo + p % bw, T.ylo + p / bw, W, vis);
    }
  }
}

// ----------------------------------------------------------------------------
// SHADE (+ adjoint)
// ----------------------------------------------------------------------------
template <int DEG, int VEC>
__device__ __forceinline__ Frag fetch_sh(const DShell& s, const Footprint& f, const float Y[16]) {
  constexpr int NCH = 1 + 3 * (DEG + 1) * (DEG + 1);
  float val[NCH];
  bilinear_f16<NCH, VEC>(reinterpret_cast<const __half*>(s.tex), s.tw, s.pitch, f, val);
  return decode_sh<DEG>(val, Y);
}

__device__ __noinline__ Frag fetch_frag(const DShell& s, const Footprint& f, const float Y[16]) {
  if (s.fmt == VS_TEX_RGBA_F32) {
    float v[4];
    if (s.vec == 4) bilinear_rgba<4>(reinterpret_cast<const float*>(s.tex), s.tw, s.pitch, f, v);
    else bilinear_rgba<1>(reinterpret_cast<const float*>(s.tex), s.tw, s.pitch, f, v);
    return {v[0], v[1], v[2], v[3]};
  }
#define VS_CASE(D, V) \
  case D * 16 + V: return fetch_sh<D, V>(s, f, Y);
  switch (s.degree * 16 + s.vec) {
    VS_CASE(0, 1) VS_CASE(0, 2) VS_CASE(0, 4) VS_CASE(0, 8)
    VS_CASE(1, 1) VS_CASE(1, 2) VS_CASE(1, 4) VS_CASE(1, 8)
    VS_CASE(2, 1) VS_CASE(2, 2) VS_CASE(2, 4) VS_CASE(2, 8)
    VS_CASE(3, 1) VS_CASE(3, 2) VS_CASE(3, 4) VS_CASE(3, 8)
    default: return {0.f, 0.f, 0.f, 0.f};
  }
#undef VS_CASE
}

// dL/d(values) of one fragment, scattered into its 4 texels.
template <int DEG, int GV>
__device__ __forceinline__ void adjoint_sh(const DShell& s, const Footprint& f, const float Y[16],
                                           const Frag& fr, float gcr, float gcg, float gcb, float ga) {
  constexpr int NB = (DEG + 1) * (DEG + 1);
  constexpr int NCH = 1 + 3 * NB;
  float dval[NCH];
  dval[0] = ga * fr.a * (1.0f - fr.a);
  const float dz[3] = {gcr * fr.r * (1.0f - fr.r), gcg * fr.g * (1.0f - fr.g), gcb * fr.b * (1.0f - fr.b)};
#pragma unroll
  for (int m = 0; m < NB; ++m)
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) dval[1 + 3 * m + ch] = dz[ch] * Y[m];
  scatter_grad<NCH, GV>(s.grad, s.tw, s.pitch, f, dval);
}

__device__ __noinline__ void adjoint_frag(const DShell& s, const Footprint& f, const float Y[16],
                                          const Frag& fr, float gcr, float gcg, float gcb, float ga) {
  if (s.fmt == VS_TEX_RGBA_F32) {
    const float dval[4] = {gcr, gcg, gcb, ga};
    if (s.gvec == 4) scatter_grad<4, 4>(s.grad, s.tw, s.pitch, f, dval);
    else if (s.gvec == 2) scatter_grad<4, 2>(s.grad, s.tw, s.pitch, f, dval);
    else scatter_grad<4, 1>(s.grad, s.tw, s.pitch, f, dval);
    return;
  }
#define VS_CASE(D, V) \
  case D * 16 + V: adjoint_sh<D, V>(s, f, Y, fr, gcr, gcg, gcb, ga); return;
  switch (s.degree * 16 + s.gvec) {
    VS_CASE(0, 1) VS_CASE(0, 2) VS_CASE(0, 4)
    VS_CASE(1, 1) VS_CASE(1, 2) VS_CASE(1, 4)
    VS_CASE(2, 1) VS_CASE(2, 2) VS_CASE(2, 4)
    VS_CASE(3, 1) VS_CASE(3, 2) VS_CASE(3, 4)
    default: return;
  }
#undef VS_CASE
}

// One thread per pixel.  FROM_HITS: the hits come from the public int32
// buffer (standalone backward) instead of the visibility words.
template <bool BWD, bool FROM_HITS>
__device__ void unit_shade(const DItem& it, const DShell* sh, int u, WsHeader* hdr) {
  const int W = it.cam.W, H = it.cam.H;
  const int HW = W * H;
  const int p = u * kShadePerUnit + threadIdx.x;
  unsigned nfrag = 0, bad = 0;
  float loss = 0.0f;
  if (p < HW) {
    const int y = p / W, x = p - y * W;
    const int px = 256 * x + 128, py = 256 * y + 128;
    float Y[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) Y[m] = 0.0f;
    if (it.maxdeg >= 0) {
      const float3 v = ray_dir(it.cam, x, y);
      sh_basis(it.maxdeg, v.x, v.y, v.z, Y);
    }
    float Cr = 0.f, Cg = 0.f, Cb = 0.f, T = 1.0f;
    // per-shell state kept for the adjoint
    Frag sf[BWD ? kMaxShells : 1];
    Footprint sfp[BWD ? kMaxShells : 1];
    float sT[BWD ? kMaxShells : 1];
    unsigned mask = 0;
    for (int i = 0; i < it.k; ++i) {
      const DShell& s = sh[i];
      int tri;
      if (FROM_HITS) {
        tri = __ldg(it.hits + (size_t)i * HW + p);
      } else {
        tri = vis_tri(__ldcg(it.vis + (size_t)i * HW + p));
        if (it.hits) it.hits[(size_t)i * HW + p] = tri;
      }
      if (tri < 0) continue;
      Tri Tr;
      if (tri >= s.nt || load_tri(s, it.cam, tri, Tr) != 0) { bad = 1; continue; }
      const int* ip = s.tris + 3 * (size_t)tri;
      const float2 uv[3] = {__ldg(s.uv + __ldg(ip)), __ldg(s.uv + __ldg(ip + 1)), __ldg(s.uv + __ldg(ip + 2))};
      const Footprint f = footprint(Tr, uv, s.tw, s.th, px, py);
      const Frag fr = fetch_frag(s, f, Y);
      ++nfrag;
      const float ta = T * fr.a;
      Cr = fmaf(ta, fr.r, Cr);
      Cg = fmaf(ta, fr.g, Cg);
      Cb = fmaf(ta, fr.b, Cb);
      if constexpr (BWD) {
        sf[i] = fr;
        sfp[i] = f;
        sT[i] = T;
        mask |= 1u << i;
      }
      T = T * (1.0f - fr.a);
    }
    const float outr = fmaf(T, it.bg[0], Cr), outg = fmaf(T, it.bg[1], Cg), outb = fmaf(T, it.bg[2], Cb);
    if (it.out) it.out[p] = make_float4(outr, outg, outb, 1.0f - T);
    if constexpr (BWD) {
      const float* gp = it.grad_rgb + 3 * (size_t)p;
      float gr = __ldg(gp), gg = __ldg(gp + 1), gb = __ldg(gp + 2);
      if (it.flags & VS_FLAG_LOSS_L2) {
        const float dr = outr - gr, dg = outg - gg, db = outb - gb;
        const float inv = 1.0f / (3.0f * (float)HW);
        loss = (dr * dr + dg * dg + db * db) * inv;
        gr = 2.0f * inv * dr;
        gg = 2.0f * inv * dg;
        gb = 2.0f * inv * db;
      }
      float Ar = it.bg[0], Ag = it.bg[1], Ab = it.bg[2];
      for (int i = it.k - 1; i >= 0; --i) {
        if (!((mask >> i) & 1u)) continue;
        const Frag fr = sf[i];
        const float Ti = sT[i];
        const float ta = Ti * fr.a;
        const float ga = Ti * ((fr.r - Ar) * gr + (fr.g - Ag) * gg + (fr.b - Ab) * gb);
        Ar = fmaf(fr.a, fr.r - Ar, Ar);
        Ag = fmaf(fr.a, fr.g - Ag, Ag);
        Ab = fmaf(fr.a, fr.b - Ab, Ab);
        adjoint_frag(sh[i], sfp[i], Y, fr, ta * gr, ta * gg, ta * gb, ga);
      }
    }
  }
  if (!FROM_HITS) warp_count(&hdr->frags, nfrag);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) record_error(hdr, VS_ERR_INVALID_ARG);
  if constexpr (BWD) {
    if (it.loss && (it.flags & VS_FLAG_LOSS_L2)) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
      if ((threadIdx.x & 31) == 0) atomicAdd(it.loss, loss);
    }
  }
}

// ----------------------------------------------------------------------------
// kernels
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_upload(char* ws, const __grid_constant__ UploadChunk c) {
  uint4* dst = reinterpret_cast<uint4*>(ws + c.dst_off);
  for (uint32_t i = threadIdx.x; i < c.nbytes / 16; i += blockDim.x) dst[i] = c.data[i];
  if (c.reset && threadIdx.x == 0) {
    WsHeader* h = reinterpret_cast<WsHeader*>(ws);
    h->next_unit = 0;
    h->abort = 0;
  }
}

__global__ void __launch_bounds__(kThreads) k_setup(TableRef tb, int item) {
  const DItem& it = tb.items[item];
  unit_setup(it, tb.shells + it.shell0, blockIdx.x);
}

__global__ void __launch_bounds__(kThreads) k_raster(TableRef tb, int item) {
  const DItem& it = tb.items[item];
  unit_raster(it, tb.shells + it.shell0, blockIdx.x, tb.hdr);
}

__global__ void __launch_bounds__(kThreads) k_large(TableRef tb, int item) {
  const DItem& it = tb.items[item];
  unit_large(it, tb.shells + it.shell0, blockIdx.x);
}

template <bool BWD, bool FROM_HITS>
__global__ void __launch_bounds__(kThreads) k_shade(TableRef tb, int item) {
  const DItem& it = tb.items[item];
  unit_shade<BWD, FROM_HITS>(it, tb.shells + it.shell0, blockIdx.x, tb.hdr);
}

// Bounded wait (one thread) for `target` completions; false on timeout or
// abort.  A timeout records VS_ERR_TIMEOUT and raises the abort flag so that
// every block leaves the persistent loop.
__device__ bool wait_done(const int* ctr, int target, long long limit, WsHeader* hdr) {
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

// Persistent kernel over all items.  Units are dispensed in the global order
// (phase, item, unit); a unit of phase p > 0 waits only for the phase p-1
// units of its own item, all of which were dispensed earlier to blocks that
// are already running, so the wait always ends (and is bounded anyway).
__global__ void __launch_bounds__(kThreads) k_persistent(TableRef tb, long long spin_limit) {
  __shared__ int s_unit, s_ok;
  WsHeader* hdr = tb.hdr;
  for (;;) {
    if (threadIdx.x == 0) {
      s_unit = *(volatile int*)&hdr->abort ? tb.total : (int)atomicAdd(&hdr->next_unit, 1u);
    }
    __syncthreads();
    const int g = s_unit;
    if (g >= tb.total) break;
    int ph = 0;
    while (ph + 1 < NPH && g >= tb.phase_start[ph + 1]) ++ph;
    const int* pre = tb.unit_pre + ph * (tb.n + 1);
    const int rel = g - tb.phase_start[ph];
    int lo = 0, hi = tb.n - 1;   // last item with pre[item] <= rel
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(pre + mid) <= rel) lo = mid; else hi = mid - 1;
    }
    const int j = lo;
    const int u = rel - __ldg(pre + j);
    const DItem& it = tb.items[j];
    if (threadIdx.x == 0) {
      bool ok = true;
      if (ph > 0) {
        int target = it.units[ph - 1];
        long long lim = spin_limit;
        if (ph == PH_SHADE && it.stall && u == 0) { target += 1; lim = 4096; }
        ok = wait_done(tb.done + j * NPH + ph - 1, target, lim, hdr);
      }
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) break;
    const DShell* sh = tb.shells + it.shell0;
    switch (ph) {
      case PH_SETUP: unit_setup(it, sh, u); break;
      case PH_RASTER: unit_raster(it, sh, u, hdr); break;
      case PH_LARGE: unit_large(it, sh, u); break;
      default:
        if (it.do_bwd) unit_shade<true, false>(it, sh, u, hdr);
        else unit_shade<false, false>(it, sh, u, hdr);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(tb.done + j * NPH + ph, 1);
    }
  }
}

}  // namespace vsd

// ----------------------------------------------------------------------------
// host-side launchers (C++ linkage, used by vs_api.cu)
// ----------------------------------------------------------------------------
namespace vsk {

cudaError_t upload(char* ws, const UploadChunk& c, cudaStream_t st) {
  vsd::k_upload<<<1, vsd::kThreads, 0, st>>>(ws, c);
  return cudaGetLastError();
}

cudaError_t plain_forward(const TableRef& tb, const int units[4], cudaStream_t st) {
  if (units[0]) vsd::k_setup<<<units[0], vsd::kThreads, 0, st>>>(tb, 0);
  if (units[1]) vsd::k_raster<<<units[1], vsd::kThreads, 0, st>>>(tb, 0);
  if (units[2]) vsd::k_large<<<units[2], vsd::kThreads, 0, st>>>(tb, 0);
  if (units[3]) vsd::k_shade<false, false><<<units[3], vsd::kThreads, 0, st>>>(tb, 0);
  return cudaGetLastError();
}

cudaError_t plain_backward(const TableRef& tb, const int units[4], cudaStream_t st) {
  if (units[0]) vsd::k_setup<<<units[0], vsd::kThreads, 0, st>>>(tb, 0);
  if (units[3]) vsd::k_shade<true, true><<<units[3], vsd::kThreads, 0, st>>>(tb, 0);
  return cudaGetLastError();
}

cudaError_t persistent(const TableRef& tb, int grid, long long spin_limit, cudaStream_t st) {
  vsd::k_persistent<<<grid, vsd::kThreads, 0, st>>>(tb, spin_limit);
  return cudaGetLastError();
}

cudaError_t persistent_occupancy(int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, vsd::k_persistent, vsd::kThreads, 0);
}

}  // namespace vsk
