// Host side of the C ABI declared in include/vs.h: argument checking,
// workspace layout, the item table and kernel launches.  No device memory is
// ever allocated here; the caller's workspace is the only scratch.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>

#include <nvtx3/nvToolsExt.h>
#include <string>
#include <tuple>
#include <vector>

#include "vs.h"
#include "vs_device.cuh"
#include "vs_kernels.h"
#include "vs_ntex.h"

using namespace vsd;

struct vs_ctx {
  int device;
  int num_sms;
  int persist_blocks[2][kNumTc][VS_MAX_SHELLS + 1];   // [backward][texel class][most shells] blocks per SM
  int persist_blocks_full[2][VS_MAX_SHELLS + 1];      // the full variant (generic class)
  std::mutex tune_mu;                          // guards tune / tune_set
  vs_tuning tune[2][VS_MAX_SHELLS + 1];        // [backward][most shells]
  bool tune_set[2][VS_MAX_SHELLS + 1];
};

struct vs_object {
  int32_t k;
  vs_shell_desc shells[VS_MAX_SHELLS];
  // bounding sphere per shell (world space), read from the positions on the
  // first render; decides whether a camera needs the clipping kernels
  std::mutex bounds_mu;
  bool bounded;
  double center[VS_MAX_SHELLS][3], radius[VS_MAX_SHELLS];
};

namespace {

thread_local std::string g_err;

// NVTX range named after a public call (header-only NVTX3: without a tool
// attached -- nsys, ncu --nvtx -- the push and pop cost a few nanoseconds).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

vs_status fail(vs_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

vs_status cuda_fail(cudaError_t e, const char* what) {
  return fail(VS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int nch_of(const vs_shell_desc& s) {
  if (s.format == VS_TEX_SH_U8) return 4 * (s.sh_degree + 1) * (s.sh_degree + 1);
  return s.format == VS_TEX_RGBA_F32 ? 4 : 1 + 3 * (s.sh_degree + 1) * (s.sh_degree + 1);
}

// Layout of a baked (VS_TEX_SH_U8) buffer: band l at (w, h) >> l s, texels of
// 4, 16, 32, 32 bytes, bands on 256-byte boundaries.
struct BakedLayout {
  int64_t offset[4];
  int32_t w[4], h[4], stride[4];
  int64_t total;
};

vs_status baked_layout(int32_t tw, int32_t th, int32_t degree, int32_t shift, BakedLayout& L) {
  static const int32_t kStride[4] = {4, 16, 32, 32};
  if (degree < 0 || degree > 3) return fail(VS_ERR_INVALID_ARG, "SH degree %d out of [0, 3]", degree);
  if (shift < 0 || shift > 3) return fail(VS_ERR_INVALID_ARG, "band_shift %d out of [0, 3]", shift);
  if (tw < 1 || th < 1 || tw > 65536 || th > 65536)
    return fail(VS_ERR_INVALID_ARG, "texture %dx%d out of [1, 65536]", tw, th);
  const int32_t div = 1 << (degree * shift);
  if (tw % div || th % div)
    return fail(VS_ERR_INVALID_ARG, "texture %dx%d not divisible by 2^(degree * band_shift) = %d", tw, th, div);
  std::memset(&L, 0, sizeof L);
  int64_t off = 0;
  for (int l = 0; l <= degree; ++l) {
    L.offset[l] = off;
    L.w[l] = tw >> (l * shift);
    L.h[l] = th >> (l * shift);
    L.stride[l] = kStride[l];
    off += ((int64_t)L.w[l] * L.h[l] * kStride[l] + 255) / 256 * 256;
  }
  L.total = off;
  return VS_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int gcd_pow2(uint64_t a, int cap) {  // largest power of two <= cap dividing a
  int g = 1;
  while (g < cap && (a % (uint64_t)(2 * g)) == 0) g *= 2;
  return g;
}

// The binding (_abi.py) mirrors these layouts field by field.
static_assert(sizeof(vs_shell_desc) == 88 && offsetof(vs_shell_desc, grad_pitch) == 80, "vs_shell_desc layout");
static_assert(sizeof(vs_camera) == 76, "vs_camera layout");

vs_status check_shell(const vs_shell_desc& s, int i) {
  if (!s.pos || !s.uv || !s.tris || !s.texels) return fail(VS_ERR_INVALID_ARG, "shell %d: NULL array", i);
  if (s.num_verts < 3 || s.num_verts > (1 << 30)) return fail(VS_ERR_INVALID_ARG, "shell %d: num_verts %d out of [3, 2^30]", i, s.num_verts);
  if (s.num_tris < 1 || s.num_tris >= kMaxTris) return fail(VS_ERR_INVALID_ARG, "shell %d: num_tris %d out of [1, 2^27)", i, s.num_tris);
  if (s.tex_w < 1 || s.tex_h < 1 || s.tex_w > 65536 || s.tex_h > 65536)
    return fail(VS_ERR_INVALID_ARG, "shell %d: texture %dx%d out of [1, 65536]", i, s.tex_w, s.tex_h);
  if (s.format != VS_TEX_RGBA_F32 && s.format != VS_TEX_SH_F16 && s.format != VS_TEX_SH_U8)
    return fail(VS_ERR_INVALID_ARG, "shell %d: unknown format %d", i, s.format);
  if (s.format == VS_TEX_SH_U8) {
    BakedLayout L;
    if (baked_layout(s.tex_w, s.tex_h, s.sh_degree, s.band_shift, L) != VS_OK)
      return fail(VS_ERR_INVALID_ARG, "shell %d: %s", i, g_err.c_str());
    if (!std::isfinite(s.value_min) || !std::isfinite(s.value_max) || !(s.value_min < s.value_max))
      return fail(VS_ERR_INVALID_ARG, "shell %d: decode range [%g, %g] not finite and increasing", i,
                  (double)s.value_min, (double)s.value_max);
    if ((uintptr_t)s.pos % 4 || (uintptr_t)s.uv % 8 || (uintptr_t)s.tris % 4 || (uintptr_t)s.texels % 16)
      return fail(VS_ERR_INVALID_ARG, "shell %d: misaligned array (pos 4 B, uv 8 B, tris 4 B, texels 16 B)", i);
    return VS_OK;
  }
  if (s.format == VS_TEX_SH_F16 && (s.sh_degree < 0 || s.sh_degree > 3)) return fail(VS_ERR_INVALID_ARG, "shell %d: SH degree %d out of [0, 3]", i, s.sh_degree);
  if (s.texel_pitch < nch_of(s)) return fail(VS_ERR_INVALID_ARG, "shell %d: texel_pitch %d < %d values", i, s.texel_pitch, nch_of(s));
  if (s.grad_pitch != 0 && s.grad_pitch < nch_of(s))
    return fail(VS_ERR_INVALID_ARG, "shell %d: grad_pitch %d < %d values", i, s.grad_pitch, nch_of(s));
  size_t esz = s.format == VS_TEX_RGBA_F32 ? 4 : 2;
  if ((uintptr_t)s.pos % 4 || (uintptr_t)s.uv % 8 || (uintptr_t)s.tris % 4 || (uintptr_t)s.texels % esz)
    return fail(VS_ERR_INVALID_ARG, "shell %d: misaligned array (pos 4 B, uv 8 B, tris 4 B, texels %zu B)", i, esz);
  return VS_OK;
}

vs_status check_camera(const vs_camera* c) {
  if (!c) return fail(VS_ERR_INVALID_ARG, "camera is NULL");
  if (c->width < 1 || c->height < 1 || c->width > VS_MAX_IMAGE_SIDE || c->height > VS_MAX_IMAGE_SIDE)
    return fail(VS_ERR_INVALID_ARG, "image %dx%d out of [1, %d]", c->width, c->height, VS_MAX_IMAGE_SIDE);
  if (!(c->znear > 0.0f) || !(c->fx != 0.0f) || !(c->fy != 0.0f))
    return fail(VS_ERR_INVALID_ARG, "camera needs znear > 0 and nonzero focal lengths");
  for (int i = 0; i < 12; ++i)
    if (!(c->world_to_cam[i] == c->world_to_cam[i])) return fail(VS_ERR_INVALID_ARG, "camera matrix has NaN");
  return VS_OK;
}

// ---------------------------------------------------------------------------
// planning: workspace layout + the host copy of the item table
// ---------------------------------------------------------------------------
struct ItemReq {
  const vs_object* obj;
  const vs_camera* cam;
  float* out;
  int32_t* hits;
  const float* grad_rgb;
  float* const* grad_tex;
  float* loss;
  float* layers = nullptr;   // per-layer buffers [k, H, W, 12] or null
  int index = 0;             // the item's position in the caller's array
};

// Dispatch order of a batch, for L2 locality: items grouped by object (in
// the order objects first appear), and within an object a greedy
// nearest-neighbour chain of camera centres from its first item, so that
// consecutive items -- shaded at overlapping times by the persistent
// kernel's skewed stages -- see nearby surface and share gradient and texel
// lines in L2.  Outputs do not depend on the order (each item writes its
// own buffers); gradient sums only through the FP32 rounding order of their
// atomics, which is unordered anyway.  Groups larger than kChainMax keep the
// caller's order (the chain costs O(n^2) on the host).
constexpr int kChainMax = 4096;

void order_for_locality(std::vector<ItemReq>& req) {
  const int n = (int)req.size();
  std::vector<ItemReq> out;
  out.reserve(n);
  std::vector<char> taken(n, 0);
  auto eye = [](const vs_camera& c, double e[3]) {   // -R^T t
    for (int a = 0; a < 3; ++a)
      e[a] = -(c.world_to_cam[0 * 4 + a] * (double)c.world_to_cam[0 * 4 + 3] +
               c.world_to_cam[1 * 4 + a] * (double)c.world_to_cam[1 * 4 + 3] +
               c.world_to_cam[2 * 4 + a] * (double)c.world_to_cam[2 * 4 + 3]);
  };
  for (int j0 = 0; j0 < n; ++j0) {
    if (taken[j0]) continue;
    std::vector<int> grp;
    for (int j = j0; j < n; ++j)
      if (!taken[j] && req[j].obj == req[j0].obj) grp.push_back(j);
    for (int j : grp) taken[j] = 1;
    if ((int)grp.size() > kChainMax) {
      for (int j : grp) out.push_back(req[j]);
      continue;
    }
    std::vector<double> E(3 * grp.size());
    for (size_t q = 0; q < grp.size(); ++q) eye(*req[grp[q]].cam, &E[3 * q]);
    std::vector<char> used(grp.size(), 0);
    size_t cur = 0;
    used[0] = 1;
    out.push_back(req[grp[0]]);
    for (size_t step = 1; step < grp.size(); ++step) {
      size_t best = 0;
      double bd = -1.0;
      for (size_t q = 0; q < grp.size(); ++q) {
        if (used[q]) continue;
        const double dx = E[3 * q] - E[3 * cur], dy = E[3 * q + 1] - E[3 * cur + 1], dz = E[3 * q + 2] - E[3 * cur + 2];
        const double d = dx * dx + dy * dy + dz * dz;
        if (bd < 0.0 || d < bd) {
          bd = d;
          best = q;
        }
      }
      used[best] = 1;
      cur = best;
      out.push_back(req[grp[best]]);
    }
  }
  req.swap(out);
}

// Work-unit sizes of one plan, in 32-wide rounds.  The plain launches run
// one round per warp of a block, so they always use kWarps rounds.
struct UnitShape {
  int raster_rounds = kWarps;
  int shade_rounds = kWarps;
};

struct Plan {
  bool full = false;             // the full kernels: a shell may reach nearer than znear
                                 // (clipping) or per-layer buffers are written
  size_t off_items, off_shells, off_done, off_stage, table_end, total;
  std::vector<DItem> items;
  std::vector<DShell> shells;
  std::vector<int> stage_pre;    // [n + 3]
  int total_units;
  int tc;                        // texel class of the kernels (vsd::TC_*)
};

// Bounding spheres of an object's shells, from one read of its positions
// (the first render with the object; positions are not expected to change
// afterwards -- reload the object if they do).
vs_status ensure_bounds(const vs_object* cobj) {
  vs_object* obj = const_cast<vs_object*>(cobj);
  std::lock_guard<std::mutex> g(obj->bounds_mu);
  if (obj->bounded) return VS_OK;
  std::vector<float> p;
  for (int i = 0; i < obj->k; ++i) {
    const vs_shell_desc& d = obj->shells[i];
    p.resize(3 * (size_t)d.num_verts);
    cudaError_t e = cudaMemcpy(p.data(), d.pos, p.size() * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading vertex positions for the shell bounds");
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (size_t v = 0; v < (size_t)d.num_verts; ++v)
      for (int c = 0; c < 3; ++c) {
        lo[c] = std::min(lo[c], (double)p[3 * v + c]);
        hi[c] = std::max(hi[c], (double)p[3 * v + c]);
      }
    double r2 = 0.0;
    for (int c = 0; c < 3; ++c) obj->center[i][c] = 0.5 * (lo[c] + hi[c]);
    for (size_t v = 0; v < (size_t)d.num_verts; ++v) {
      double q = 0.0;
      for (int c = 0; c < 3; ++c) q += (p[3 * v + c] - obj->center[i][c]) * (p[3 * v + c] - obj->center[i][c]);
      r2 = std::max(r2, q);
    }
    obj->radius[i] = std::sqrt(r2);
  }
  obj->bounded = true;
  return VS_OK;
}

// Whether a shell of the object may come nearer than znear in this camera
// (camera depth of its bounding sphere, with a margin far above the FP32
// rounding of the vertex transform); true while the bounds are unknown.
bool needs_clip(const vs_object& o, const vs_camera& c) {
  if (!o.bounded) return true;
  const float* m = c.world_to_cam;
  const double n = std::sqrt((double)m[8] * m[8] + (double)m[9] * m[9] + (double)m[10] * m[10]);
  for (int i = 0; i < o.k; ++i) {
    const double* ce = o.center[i];
    const double z = m[8] * ce[0] + m[9] * ce[1] + m[10] * ce[2] + m[11];
    const double scale = n * (std::fabs(ce[0]) + std::fabs(ce[1]) + std::fabs(ce[2]) + o.radius[i]) +
                         std::fabs((double)m[11]) + c.znear;
    if (z - n * o.radius[i] < (double)c.znear + 1e-5 * scale) return true;
  }
  return false;
}

// Fills the plan; with ws == nullptr only sizes are computed.
vs_status make_plan(const ItemReq* req, int n, const float* bg, int do_bwd, bool clear_vis, uint32_t flags,
                    char* ws, Plan& P, UnitShape shape = UnitShape()) {
  if ((flags & VS_FLAG_LOSS_L1) && (flags & VS_FLAG_LOSS_L2))
    return fail(VS_ERR_INVALID_ARG, "VS_FLAG_LOSS_L1 and VS_FLAG_LOSS_L2 are exclusive");
  P.full = false;
  for (int j = 0; j < n; ++j) P.full = P.full || needs_clip(*req[j].obj, *req[j].cam) || req[j].layers;
  const int raster_per_unit = 32 * shape.raster_rounds;
  const int shade_per_unit = 32 * shape.shade_rounds;
  size_t off = sizeof(WsHeader);
  int S = 0;
  for (int j = 0; j < n; ++j) S += req[j].obj->k;
  P.off_items = off;
  off = align256(off + sizeof(DItem) * (size_t)n);
  P.off_shells = off;
  off = align256(off + sizeof(DShell) * (size_t)S);
  P.off_done = off;
  off = align256(off + sizeof(int) * (size_t)n * NPH);
  P.off_stage = off;
  off = align256(off + sizeof(int) * (size_t)(n + NPH));
  P.table_end = off;
  P.items.assign(n, DItem{});
  P.shells.assign(S, DShell{});
  P.stage_pre.assign((size_t)n + NPH, 0);
  int sidx = 0;
  for (int j = 0; j < n; ++j) {
    const vs_object& o = *req[j].obj;
    const vs_camera& c = *req[j].cam;
    DItem& it = P.items[j];
    std::memcpy(it.cam.m, c.world_to_cam, sizeof it.cam.m);
    it.cam.fx = c.fx; it.cam.fy = c.fy; it.cam.cx = c.cx; it.cam.cy = c.cy; it.cam.znear = c.znear;
    it.cam.W = c.width; it.cam.H = c.height;
    it.cam.rfx = 1.0f / c.fx; it.cam.rfy = 1.0f / c.fy;
    it.out = reinterpret_cast<float4*>(req[j].out);
    it.hits = req[j].hits;
    it.layers = req[j].layers;
    it.grad_rgb = req[j].grad_rgb;
    it.loss = req[j].loss;
    it.k = o.k;
    it.shell0 = sidx;
    it.flags = (int)flags;
    it.do_bwd = do_bwd;
    it.stall = (flags & VS_FLAG_TEST_STALL) ? 1 : 0;
    it.raster_rounds = shape.raster_rounds;
    it.shade_rounds = shape.shade_rounds;
    it.bg[0] = bg ? bg[0] : 0.f; it.bg[1] = bg ? bg[1] : 0.f; it.bg[2] = bg ? bg[2] : 0.f;
    const size_t HW = (size_t)c.width * c.height;
    it.setup_pre[0] = 0;
    it.raster_pre[0] = 0;
    for (int i = 0; i < o.k; ++i) {
      const vs_shell_desc& d = o.shells[i];
      DShell& s = P.shells[sidx + i];
      s.pos = d.pos; s.uv = reinterpret_cast<const float2*>(d.uv); s.tris = d.tris; s.tex = d.texels;
      s.grad = (do_bwd && req[j].grad_tex) ? req[j].grad_tex[i] : nullptr;
      s.nv = d.num_verts; s.nt = d.num_tris; s.tw = d.tex_w; s.th = d.tex_h;
      s.fmt = d.format; s.degree = d.format != VS_TEX_RGBA_F32 ? d.sh_degree : 0; s.pitch = d.texel_pitch;
      if (d.format == VS_TEX_SH_U8) {
        BakedLayout L;
        baked_layout(d.tex_w, d.tex_h, d.sh_degree, d.band_shift, L);   // checked at load
        for (int l = 0; l < 4; ++l) s.boff[l] = L.offset[l];
        s.bshift = d.band_shift;
        s.vmin = d.value_min;
        s.vscale = (d.value_max - d.value_min) / 255.0f;
        s.pitch = 0;
      }
      const int esz = d.format == VS_TEX_RGBA_F32 ? 4 : 2;
      const uint64_t tex_align = (uint64_t)(uintptr_t)d.texels | (uint64_t)d.texel_pitch * esz;
      s.vec = d.format == VS_TEX_RGBA_F32 ? (gcd_pow2(tex_align, 16) >= 16 ? 4 : 1) : gcd_pow2(tex_align, 16) / 2;
      s.wide = gcd_pow2(tex_align, 32) >= 32;
      s.gpitch = d.grad_pitch > 0 ? d.grad_pitch : d.texel_pitch;
      if (s.grad) {
        const uint64_t ga = (uint64_t)(uintptr_t)s.grad | (uint64_t)s.gpitch * 4;
        s.gvec = gcd_pow2(ga, 16) / 4;
        if (s.gvec < 1) s.gvec = 1;
      } else {
        s.gvec = 1;
      }
      s.vsetup = reinterpret_cast<int4*>(ws ? ws + off : nullptr);
      off = align256(off + sizeof(int4) * (size_t)d.num_verts);
      it.setup_pre[i + 1] = it.setup_pre[i] + (d.num_verts + kSetupPerUnit - 1) / kSetupPerUnit;
      it.raster_pre[i + 1] = it.raster_pre[i] + (d.num_tris + raster_per_unit - 1) / raster_per_unit;
    }
    it.vis = reinterpret_cast<unsigned long long*>(ws ? ws + off : nullptr);
    if (clear_vis) off = align256(off + sizeof(unsigned long long) * o.k * HW);
    const size_t vis_words = (size_t)o.k * HW;
    it.clear_units = clear_vis ? (int)((vis_words + kClearPerUnit - 1) / kClearPerUnit) : 0;
    it.units[PH_SETUP] = it.clear_units + it.setup_pre[o.k];
    it.units[PH_RASTER] = clear_vis ? it.raster_pre[o.k] : 0;
    it.units[PH_SHADE] = (int)((HW + shade_per_unit - 1) / shade_per_unit);
    sidx += o.k;
  }
  P.total = align256(off);
  // texel class: one compiled format when every shell shares it with
  // 16-byte-aligned texels (and, for the adjoint, gradients); SH of degree
  // >= 1 also with 32-byte-aligned texels (256-bit loads)
  int tc = -1;
  for (const DShell& sh : P.shells) {
    int c = TC_ANY;
    if (sh.fmt == VS_TEX_RGBA_F32 && sh.vec == 4 && (!do_bwd || sh.gvec == 4)) c = TC_RGBA;
    else if (sh.fmt == VS_TEX_SH_F16 && sh.vec == 8 && (!do_bwd || sh.gvec == 4) && (sh.degree == 0 || sh.wide))
      c = TC_SH0 + sh.degree;
    else if (sh.fmt == VS_TEX_SH_U8) c = TC_U80 + sh.degree;
    tc = (tc < 0 || tc == c) ? c : TC_ANY;
  }
  P.tc = tc < 0 ? TC_ANY : tc;
  if (P.full) P.tc = TC_ANY;   // the full kernels exist for the generic class
  // skewed stages: stage s = SETUP(s), RASTER(s-1), SHADE(s-2)
  long long g = 0;
  for (int st = 0; st < n + NPH - 1; ++st) {
    P.stage_pre[st] = (int)std::min<long long>(g, 0x7FFFFFFF);
    for (int ph = 0; ph < NPH; ++ph) {
      const int j = st - ph;
      if (j >= 0 && j < n) g += P.items[j].units[ph];
    }
  }
  P.stage_pre[n + NPH - 1] = (int)std::min<long long>(g, 0x7FFFFFFF);
  P.total_units = (int)std::min<long long>(g, 0x7FFFFFFF);
  if (g > 0x7FFFFFFF) return fail(VS_ERR_OVERFLOW, "too many work units (%lld)", g);
  return VS_OK;
}

TableRef table_ref(const Plan& P, char* ws) {
  TableRef t;
  t.hdr = reinterpret_cast<WsHeader*>(ws);
  t.items = reinterpret_cast<DItem*>(ws + P.off_items);
  t.shells = reinterpret_cast<DShell*>(ws + P.off_shells);
  t.done = reinterpret_cast<int*>(ws + P.off_done);
  t.stage_pre = reinterpret_cast<const int*>(ws + P.off_stage);
  t.n = (int)P.items.size();
  t.total = P.total_units;
  t.kmax = 1;
  for (const DItem& it : P.items) t.kmax = std::max(t.kmax, (int)it.k);
  return t;
}

size_t upload_chunks(const Plan& P) {
  const size_t bytes = P.table_end - P.off_items;
  return std::max<size_t>(1, (bytes + kUploadBytes - 1) / kUploadBytes);
}

// Copies the table (items, shells, zeroed completion counters, stage
// prefixes) into the workspace through kernel parameters; `kernels` is the
// number of compute kernels the call enqueues after the upload.
vs_status upload_table(const Plan& P, char* ws, int kernels, cudaStream_t st) {
  std::vector<char> blob(P.table_end - P.off_items, 0);
  std::memcpy(blob.data(), P.items.data(), sizeof(DItem) * P.items.size());
  std::memcpy(blob.data() + (P.off_shells - P.off_items), P.shells.data(), sizeof(DShell) * P.shells.size());
  std::memcpy(blob.data() + (P.off_stage - P.off_items), P.stage_pre.data(), sizeof(int) * P.stage_pre.size());
  static thread_local UploadChunk chunk;
  const size_t nchunks = upload_chunks(P);
  size_t pos = 0;
  for (size_t c = 0; c < nchunks; ++c) {
    const size_t nb = std::min(blob.size() - pos, (size_t)kUploadBytes);
    chunk.dst_off = (uint32_t)(P.off_items + pos);
    chunk.nbytes = (uint32_t)nb;
    chunk.reset = c == 0 ? 1 : 0;
    chunk.launches = c == 0 ? (int32_t)(nchunks + kernels) : 0;
    chunk.kernel_class = 1 + P.tc + (P.full ? 16 : 0);
    std::memcpy(chunk.data, blob.data() + pos, nb);
    cudaError_t e = vsk::upload(ws, chunk, st);
    if (e != cudaSuccess) return cuda_fail(e, "table upload launch");
    pos += nb;
  }
  return VS_OK;
}

vs_status check_ws(const Plan& P, void* ws, size_t ws_bytes) {
  if (!ws) return fail(VS_ERR_WORKSPACE, "workspace is NULL");
  if ((uintptr_t)ws % 256) return fail(VS_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (ws_bytes < P.total) return fail(VS_ERR_WORKSPACE, "workspace has %zu bytes, needs %zu", ws_bytes, P.total);
  if (P.table_end - P.off_items > ((size_t)1 << 31)) return fail(VS_ERR_OVERFLOW, "item table too large");
  if ((long long)P.total_units > 0x7FFFFFFFll) return fail(VS_ERR_OVERFLOW, "too many work units");
  return VS_OK;
}

vs_status check_item(const vs_ctx* ctx, const vs_object* obj, const vs_camera* cam) {
  if (!ctx) return fail(VS_ERR_INVALID_ARG, "ctx is NULL");
  if (!obj) return fail(VS_ERR_INVALID_ARG, "object is NULL");
  return check_camera(cam);
}

vs_status set_device(const vs_ctx* ctx) {
  cudaError_t e = cudaSetDevice(ctx->device);
  return e == cudaSuccess ? VS_OK : cuda_fail(e, "cudaSetDevice");
}

// ---------------------------------------------------------------------------
// batch tuning
// ---------------------------------------------------------------------------
bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

vs_status check_tuning(const vs_tuning* t) {
  if (!t) return fail(VS_ERR_INVALID_ARG, "tuning is NULL");
  if (!pow2_in(t->raster_tris, 32, 2048))
    return fail(VS_ERR_INVALID_ARG, "raster_tris %d is not a power of two in [32, 2048]", t->raster_tris);
  if (!pow2_in(t->shade_pixels, 32, 4096))
    return fail(VS_ERR_INVALID_ARG, "shade_pixels %d is not a power of two in [32, 4096]", t->shade_pixels);
  if (t->blocks_per_sm < 0 || t->blocks_per_sm > 64)
    return fail(VS_ERR_INVALID_ARG, "blocks_per_sm %d out of [0, 64]", t->blocks_per_sm);
  if (t->reserved != 0) return fail(VS_ERR_INVALID_ARG, "reserved field must be 0");
  return VS_OK;
}

vs_tuning default_tuning() {
  vs_tuning t{};
  t.raster_tris = VS_TUNING_DEFAULT_RASTER_TRIS;
  t.shade_pixels = VS_TUNING_DEFAULT_SHADE_PIXELS;
  return t;
}

vs_tuning lookup_tuning(vs_ctx* ctx, int bwd, int kmax) {
  std::lock_guard<std::mutex> g(ctx->tune_mu);
  return ctx->tune_set[bwd][kmax] ? ctx->tune[bwd][kmax] : default_tuning();
}

UnitShape shape_of(const vs_tuning& t) {
  UnitShape u;
  u.raster_rounds = t.raster_tris / 32;
  u.shade_rounds = t.shade_pixels / 32;
  return u;
}

// Checks every item of a batch (before anything is enqueued) and fills the
// plan requests; makes the context's device current and bounds the objects.
vs_status check_batch(const vs_ctx* ctx, const vs_batch_item* items, int n, int do_backward,
                      std::vector<ItemReq>& req, int* kmax) {
  if (!ctx || !items) return fail(VS_ERR_INVALID_ARG, "NULL argument");
  if (n < 1) return fail(VS_ERR_INVALID_ARG, "n = %d < 1", n);
  req.assign(n, ItemReq{});
  *kmax = 1;
  for (int j = 0; j < n; ++j) {
    const vs_batch_item& b = items[j];
    vs_status s = check_item(ctx, b.obj, &b.cam);
    if (s != VS_OK) return fail(s, "item %d: %s", j, g_err.c_str());
    if (!b.out_rgba || (uintptr_t)b.out_rgba % 16) return fail(VS_ERR_INVALID_ARG, "item %d: out_rgba NULL or not 16-byte aligned", j);
    if (do_backward) {
      for (int i = 0; i < b.obj->k; ++i)
        if (b.obj->shells[i].format == VS_TEX_SH_U8)
          return fail(VS_ERR_UNSUPPORTED, "item %d, shell %d: baked bytes (VS_TEX_SH_U8) have no gradient", j, i);
      if (!b.grad_rgb || !b.grad_texels) return fail(VS_ERR_INVALID_ARG, "item %d: backward needs grad_rgb and grad_texels", j);
      for (int i = 0; i < b.obj->k; ++i)
        if (!b.grad_texels[i] || (uintptr_t)b.grad_texels[i] % 4) return fail(VS_ERR_INVALID_ARG, "item %d: grad_texels[%d] NULL or misaligned", j, i);
    }
    req[j] = ItemReq{b.obj, &b.cam, b.out_rgba, b.hits, b.grad_rgb, b.grad_texels, b.loss, nullptr, j};
    *kmax = std::max(*kmax, (int)b.obj->k);
  }
  vs_status s = set_device(ctx);
  if (s != VS_OK) return s;
  for (int j = 0; j < n; ++j)
    if ((s = ensure_bounds(items[j].obj)) != VS_OK) return s;
  order_for_locality(req);
  return VS_OK;
}

// Checks the batch and builds its plan (shared by vs_render_batch and the
// autotuner).
vs_status plan_batch(const vs_ctx* ctx, const vs_batch_item* items, int n, const float* bg, int do_backward,
                     void* workspace, size_t ws_bytes, uint32_t flags, const vs_tuning& t, Plan& P, int* kmax) {
  std::vector<ItemReq> req;
  vs_status s = check_batch(ctx, items, n, do_backward, req, kmax);
  if (s != VS_OK) return s;
  if ((s = make_plan(req.data(), n, bg, do_backward ? 1 : 0, true, flags, static_cast<char*>(workspace), P,
                     shape_of(t))) != VS_OK)
    return s;
  return check_ws(P, workspace, ws_bytes);
}

// Enqueues a planned batch: table upload + one persistent launch.
vs_status launch_batch(vs_ctx* ctx, const Plan& P, void* workspace, int do_backward, int kmax, const vs_tuning& t,
                       cudaStream_t st) {
  char* ws = static_cast<char*>(workspace);
  vs_status s = upload_table(P, ws, 1, st);
  if (s != VS_OK) return s;
  const int most = P.full ? ctx->persist_blocks_full[do_backward ? 1 : 0][kmax]
                         : ctx->persist_blocks[do_backward ? 1 : 0][P.tc][kmax];
  const int bps = t.blocks_per_sm == 0 ? most : std::min(t.blocks_per_sm, most);
  const long long spin_limit = 1ll << 24;   // ~ seconds with 200 ns sleeps
  cudaError_t e = vsk::persistent(table_ref(P, ws), do_backward != 0, P.tc, P.full, ctx->num_sms * bps, spin_limit,
                                  st);
  return e == cudaSuccess ? VS_OK : cuda_fail(e, "vs_render_batch launch");
}

// Cost function of vs_autotune_batch: shortest of `repeats` timed launches.
struct AutotuneJob {
  vs_ctx* ctx;
  const vs_batch_item* items;
  int n;
  const float* bg;
  int do_backward;
  void* ws;
  size_t ws_bytes;
  uint32_t flags;
  cudaStream_t st;
  int repeats;
  cudaEvent_t ev[2];
  vs_status status;       // first failure, reported after the search
  std::string error;
};

double autotune_cost(const vs_tuning* t, void* user) {
  AutotuneJob& J = *static_cast<AutotuneJob*>(user);
  if (J.status != VS_OK) return NAN;
  Plan P;
  int kmax = 1;
  auto bail = [&](vs_status s) {
    J.status = s;
    J.error = g_err;
    return (double)NAN;
  };
  vs_status s = plan_batch(J.ctx, J.items, J.n, J.bg, J.do_backward, J.ws, J.ws_bytes, J.flags, *t, P, &kmax);
  if (s != VS_OK) return bail(s);
  float best = INFINITY;
  for (int r = 0; r <= J.repeats; ++r) {
    cudaError_t e = cudaEventRecord(J.ev[0], J.st);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaEventRecord"));
    if ((s = launch_batch(J.ctx, P, J.ws, J.do_backward, kmax, *t, J.st)) != VS_OK) return bail(s);
    if ((e = cudaEventRecord(J.ev[1], J.st)) != cudaSuccess) return bail(cuda_fail(e, "cudaEventRecord"));
    if ((e = cudaEventSynchronize(J.ev[1])) != cudaSuccess) return bail(cuda_fail(e, "cudaEventSynchronize"));
    int32_t dev_status = 0;
    if ((e = cudaMemcpy(&dev_status, J.ws, sizeof dev_status, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return bail(cuda_fail(e, "cudaMemcpy"));
    if (dev_status != VS_OK) return bail(fail(dev_status, "a tuning launch recorded device status %d", dev_status));
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, J.ev[0], J.ev[1])) != cudaSuccess) return bail(cuda_fail(e, "cudaEventElapsedTime"));
    if (r > 0) best = std::min(best, ms);   // launch 0 is the untimed warm-up
  }
  return best;
}

}  // namespace

// ===========================================================================
extern "C" {

const char* vs_last_error(void) { return g_err.c_str(); }

vs_status vs_baked_layout(int32_t tex_w, int32_t tex_h, int32_t sh_degree, int32_t band_shift, int64_t band_offset[4],
                          int32_t band_w[4], int32_t band_h[4], int32_t band_stride[4], int64_t* total_bytes) {
  BakedLayout L;
  vs_status s = baked_layout(tex_w, tex_h, sh_degree, band_shift, L);
  if (s != VS_OK) return s;
  for (int l = 0; l < 4; ++l) {
    if (band_offset) band_offset[l] = L.offset[l];
    if (band_w) band_w[l] = L.w[l];
    if (band_h) band_h[l] = L.h[l];
    if (band_stride) band_stride[l] = L.stride[l];
  }
  if (total_bytes) *total_bytes = L.total;
  return VS_OK;
}

vs_status vs_create(vs_ctx** ctx, int device) {
  if (!ctx) return fail(VS_ERR_INVALID_ARG, "ctx is NULL");
  *ctx = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= n) return fail(VS_ERR_CUDA, "device %d not present (%d devices)", device, n);
  if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  vs_ctx* c = new (std::nothrow) vs_ctx{};
  if (!c) return fail(VS_ERR_INVALID_ARG, "out of host memory");
  c->device = device;
  if ((e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaDeviceGetAttribute");
  }
  if ((e = vsk::configure_kernels()) != cudaSuccess) {
    delete c;
    return cuda_fail(e, "kernel configuration");
  }
  for (int b = 0; b < 2; ++b)
    for (int tc = 0; tc < kNumTc; ++tc)
      for (int K = 1; K <= VS_MAX_SHELLS; ++K) {
        int& nb = c->persist_blocks[b][tc][K];
        if ((e = vsk::persistent_occupancy(b == 1, tc, false, K, &nb)) != cudaSuccess) {
          delete c;
          return cuda_fail(e, "occupancy query");
        }
        if (nb < 1) nb = 1;
      }
  for (int b = 0; b < 2; ++b)
    for (int K = 1; K <= VS_MAX_SHELLS; ++K) {
      int& nb = c->persist_blocks_full[b][K];
      if ((e = vsk::persistent_occupancy(b == 1, TC_ANY, true, K, &nb)) != cudaSuccess) {
        delete c;
        return cuda_fail(e, "occupancy query");
      }
      if (nb < 1) nb = 1;
    }
  *ctx = c;
  g_err.clear();
  return VS_OK;
}

vs_status vs_destroy(vs_ctx* ctx) {
  delete ctx;
  return VS_OK;
}

vs_status vs_load_shells(vs_ctx* ctx, const vs_shell_desc* shells, int32_t k, vs_object** out) {
  if (!ctx || !shells || !out) return fail(VS_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (k < 1 || k > VS_MAX_SHELLS) return fail(VS_ERR_INVALID_ARG, "k = %d out of [1, %d]", k, VS_MAX_SHELLS);
  for (int i = 0; i < k; ++i) {
    vs_status s = check_shell(shells[i], i);
    if (s != VS_OK) return s;
  }
  vs_object* o = new (std::nothrow) vs_object{};
  if (!o) return fail(VS_ERR_INVALID_ARG, "out of host memory");
  o->k = k;
  std::memcpy(o->shells, shells, sizeof(vs_shell_desc) * k);
  *out = o;
  return VS_OK;
}

vs_status vs_free_shells(vs_ctx* ctx, vs_object* obj) {
  (void)ctx;
  delete obj;
  return VS_OK;
}

vs_status vs_workspace_size(vs_ctx* ctx, const vs_object* const* objs, const vs_camera* cams, int32_t n_items,
                            uint32_t flags, size_t* bytes) {
  (void)ctx;
  if (!objs || !cams || !bytes) return fail(VS_ERR_INVALID_ARG, "NULL argument");
  if (n_items < 1) return fail(VS_ERR_INVALID_ARG, "n_items = %d < 1", n_items);
  std::vector<ItemReq> req(n_items);
  for (int j = 0; j < n_items; ++j) {
    if (!objs[j]) return fail(VS_ERR_INVALID_ARG, "object %d is NULL", j);
    vs_status s = check_camera(&cams[j]);
    if (s != VS_OK) return s;
    req[j] = ItemReq{objs[j], &cams[j], nullptr, nullptr, nullptr, nullptr, nullptr};
  }
  Plan P;
  vs_status s = make_plan(req.data(), n_items, nullptr, 1, true, flags, nullptr, P);
  if (s != VS_OK) return s;
  *bytes = P.total;
  return VS_OK;
}

vs_status vs_render(vs_ctx* ctx, const vs_object* obj, const vs_camera* cam, const float* bg, float* out_rgba,
                    int32_t* hits, void* workspace, size_t ws_bytes, uint32_t flags, vs_stream_t stream) {
  NvtxRange nvtx_range("vs_render");
  vs_status s = check_item(ctx, obj, cam);
  if (s != VS_OK) return s;
  if (!out_rgba) return fail(VS_ERR_INVALID_ARG, "out_rgba is NULL");
  if ((uintptr_t)out_rgba % 16) return fail(VS_ERR_INVALID_ARG, "out_rgba must be 16-byte aligned");
  ItemReq r{obj, cam, out_rgba, hits, nullptr, nullptr, nullptr};
  Plan P;
  char* ws = static_cast<char*>(workspace);
  if ((s = set_device(ctx)) != VS_OK) return s;
  if ((s = ensure_bounds(obj)) != VS_OK) return s;
  if ((s = make_plan(&r, 1, bg, 0, true, flags & ~VS_FLAG_TEST_STALL, ws, P)) != VS_OK) return s;
  if ((s = check_ws(P, workspace, ws_bytes)) != VS_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if ((s = upload_table(P, ws, vsk::plain_forward_launches(P.items[0].units), st)) != VS_OK) return s;
  cudaError_t e = vsk::plain_forward(table_ref(P, ws), P.items[0].units, P.tc, P.full, st);
  return e == cudaSuccess ? VS_OK : cuda_fail(e, "vs_render launch");
}

vs_status vs_render_layers(vs_ctx* ctx, const vs_object* obj, const vs_camera* cam, const float* bg, float* out_rgba,
                           int32_t* hits, float* layers, void* workspace, size_t ws_bytes, uint32_t flags,
                           vs_stream_t stream) {
  NvtxRange nvtx_range("vs_render_layers");
  vs_status s = check_item(ctx, obj, cam);
  if (s != VS_OK) return s;
  if (!out_rgba || !layers) return fail(VS_ERR_INVALID_ARG, "out_rgba and layers are required");
  if ((uintptr_t)out_rgba % 16 || (uintptr_t)layers % 16)
    return fail(VS_ERR_INVALID_ARG, "out_rgba and layers must be 16-byte aligned");
  ItemReq r{obj, cam, out_rgba, hits, nullptr, nullptr, nullptr, layers};
  Plan P;
  char* ws = static_cast<char*>(workspace);
  if ((s = set_device(ctx)) != VS_OK) return s;
  if ((s = ensure_bounds(obj)) != VS_OK) return s;
  if ((s = make_plan(&r, 1, bg, 0, true, flags & ~VS_FLAG_TEST_STALL, ws, P)) != VS_OK) return s;
  if ((s = check_ws(P, workspace, ws_bytes)) != VS_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if ((s = upload_table(P, ws, vsk::plain_forward_launches(P.items[0].units), st)) != VS_OK) return s;
  cudaError_t e = vsk::plain_forward(table_ref(P, ws), P.items[0].units, P.tc, P.full, st);
  return e == cudaSuccess ? VS_OK : cuda_fail(e, "vs_render_layers launch");
}

vs_status vs_render_backward(vs_ctx* ctx, const vs_object* obj, const vs_camera* cam, const float* bg,
                             const int32_t* hits, const float* grad_rgb, float* const* grad_texels, float* loss,
                             void* workspace, size_t ws_bytes, uint32_t flags, vs_stream_t stream) {
  NvtxRange nvtx_range("vs_render_backward");
  vs_status s = check_item(ctx, obj, cam);
  if (s != VS_OK) return s;
  for (int i = 0; i < obj->k; ++i)
    if (obj->shells[i].format == VS_TEX_SH_U8)
      return fail(VS_ERR_UNSUPPORTED, "shell %d: baked bytes (VS_TEX_SH_U8) have no gradient", i);
  if (!hits || !grad_rgb || !grad_texels) return fail(VS_ERR_INVALID_ARG, "hits, grad_rgb and grad_texels are required");
  for (int i = 0; i < obj->k; ++i)
    if (!grad_texels[i] || (uintptr_t)grad_texels[i] % 4) return fail(VS_ERR_INVALID_ARG, "grad_texels[%d] NULL or misaligned", i);
  ItemReq r{obj, cam, nullptr, const_cast<int32_t*>(hits), grad_rgb, grad_texels, loss};
  Plan P;
  char* ws = static_cast<char*>(workspace);
  if ((s = set_device(ctx)) != VS_OK) return s;
  if ((s = ensure_bounds(obj)) != VS_OK) return s;
  if ((s = make_plan(&r, 1, bg, 1, false, flags & ~VS_FLAG_TEST_STALL, ws, P)) != VS_OK) return s;
  if ((s = check_ws(P, workspace, ws_bytes)) != VS_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if ((s = upload_table(P, ws, vsk::plain_backward_launches(P.items[0].units), st)) != VS_OK) return s;
  cudaError_t e = vsk::plain_backward(table_ref(P, ws), P.items[0].units, P.tc, P.full, st);
  return e == cudaSuccess ? VS_OK : cuda_fail(e, "vs_render_backward launch");
}

vs_status vs_render_batch(vs_ctx* ctx, const vs_batch_item* items, int32_t n, const float* bg, int32_t do_backward,
                          void* workspace, size_t ws_bytes, uint32_t flags, vs_stream_t stream) {
  NvtxRange nvtx_range("vs_render_batch");
  if (!ctx || !items) return fail(VS_ERR_INVALID_ARG, "NULL argument");
  if (n < 1) return fail(VS_ERR_INVALID_ARG, "n = %d < 1", n);
  int kmax = 1;
  for (int j = 0; j < n; ++j)
    if (items[j].obj) kmax = std::max(kmax, std::min((int)items[j].obj->k, VS_MAX_SHELLS));
  const vs_tuning t = lookup_tuning(ctx, do_backward ? 1 : 0, kmax);
  std::vector<ItemReq> req;
  vs_status s = check_batch(ctx, items, n, do_backward, req, &kmax);   // makes the device current
  if (s != VS_OK) return s;
  const int bwd = do_backward ? 1 : 0;
  const UnitShape shape = shape_of(t);
  // bytes of the runs [j, j + m): the plan's layout without a workspace
  auto run_bytes = [&](int j, int m, size_t* bytes) {
    Plan Q;
    vs_status r = make_plan(req.data() + j, m, bg, bwd, true, flags, nullptr, Q, shape);
    *bytes = Q.total;
    return r;
  };
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  size_t all = 0;
  if ((s = run_bytes(0, n, &all)) != VS_OK) return s;
  // consecutive runs of items, each the longest that fits the workspace (the
  // whole batch in one launch when it fits)
  int runs = 0;
  for (int j = 0; j < n;) {
    int m = n - j;
    size_t bytes = j == 0 ? all : 0;
    if (j > 0 && (s = run_bytes(j, m, &bytes)) != VS_OK) return s;
    if (bytes > ws_bytes) {
      size_t one = 0;
      if ((s = run_bytes(j, 1, &one)) != VS_OK) return s;
      if (one > ws_bytes || !workspace)
        return fail(VS_ERR_WORKSPACE, "workspace has %zu bytes; item %d alone needs %zu (the batch %zu)", ws_bytes,
                    req[j].index, one, all);
      int lo = 1, hi = m - 1;   // largest m' in [lo, hi] that fits; lo fits
      while (lo < hi) {
        const int mid = lo + (hi - lo + 1) / 2;
        size_t b = 0;
        if ((s = run_bytes(j, mid, &b)) != VS_OK) return s;
        if (b <= ws_bytes) lo = mid; else hi = mid - 1;
      }
      m = lo;
    }
    Plan P;
    if ((s = make_plan(req.data() + j, m, bg, bwd, true, flags, static_cast<char*>(workspace), P, shape)) != VS_OK)
      return s;
    if ((s = check_ws(P, workspace, ws_bytes)) != VS_OK) return s;
    int km = 1;
    for (int q = j; q < j + m; ++q) km = std::max(km, (int)req[q].obj->k);
    if ((s = launch_batch(ctx, P, workspace, do_backward, km, t, st)) != VS_OK)
      return runs ? fail(s, "run %d of the batch (%d items): %s", runs, m, g_err.c_str()) : s;
    ++runs;
    j += m;
  }
  return VS_OK;
}

vs_status vs_set_batch_tuning(vs_ctx* ctx, int32_t do_backward, int32_t k_max, const vs_tuning* t) {
  vs_status s = check_tuning(t);
  if (s != VS_OK) return s;
  if (k_max < 0 || k_max > VS_MAX_SHELLS) return fail(VS_ERR_INVALID_ARG, "k_max %d out of [0, %d]", k_max, VS_MAX_SHELLS);
  if (!ctx) return fail(VS_ERR_INVALID_ARG, "ctx is NULL");
  std::lock_guard<std::mutex> g(ctx->tune_mu);
  const int b = do_backward ? 1 : 0;
  for (int K = (k_max ? k_max : 1); K <= (k_max ? k_max : VS_MAX_SHELLS); ++K) {
    ctx->tune[b][K] = *t;
    ctx->tune_set[b][K] = true;
  }
  return VS_OK;
}

vs_status vs_get_batch_tuning(vs_ctx* ctx, int32_t do_backward, int32_t k_max, vs_tuning* t) {
  if (!t) return fail(VS_ERR_INVALID_ARG, "tuning is NULL");
  if (k_max < 1 || k_max > VS_MAX_SHELLS) return fail(VS_ERR_INVALID_ARG, "k_max %d out of [1, %d]", k_max, VS_MAX_SHELLS);
  if (!ctx) return fail(VS_ERR_INVALID_ARG, "ctx is NULL");
  *t = lookup_tuning(ctx, do_backward ? 1 : 0, k_max);
  return VS_OK;
}

vs_status vs_tune_search(const vs_tuning* start, int32_t max_blocks_per_sm, vs_cost_fn cost, void* user,
                         vs_tuning* best, int32_t* evaluations) {
  if (!start || !cost || !best) return fail(VS_ERR_INVALID_ARG, "NULL argument");
  vs_status s = check_tuning(start);
  if (s != VS_OK) return s;
  if (max_blocks_per_sm < 1 || max_blocks_per_sm > 64)
    return fail(VS_ERR_INVALID_ARG, "max_blocks_per_sm %d out of [1, 64]", max_blocks_per_sm);
  vs_tuning cur = *start;
  if (cur.blocks_per_sm == 0 || cur.blocks_per_sm > max_blocks_per_sm) cur.blocks_per_sm = max_blocks_per_sm;
  std::map<std::tuple<int, int, int>, double> seen;
  int calls = 0;
  bool bad = false;
  auto eval = [&](const vs_tuning& t) -> double {
    const auto key = std::make_tuple(t.raster_tris, t.shade_pixels, t.blocks_per_sm);
    auto f = seen.find(key);
    if (f != seen.end()) return f->second;
    const double c = cost(&t, user);
    ++calls;
    if (!(c >= 0.0)) bad = true;
    seen[key] = c;
    return c;
  };
  double cur_cost = eval(cur);
  static const int kSizes[] = {64, 128, 256, 512, 1024};
  for (int sweep = 0; sweep < 4 && !bad; ++sweep) {
    bool moved = false;
    for (int dim = 0; dim < 3 && !bad; ++dim) {
      const int nv = dim < 2 ? 5 : max_blocks_per_sm;
      vs_tuning pick = cur;
      double pick_cost = cur_cost;
      for (int v = 0; v < nv && !bad; ++v) {
        vs_tuning t = cur;
        if (dim == 0) t.raster_tris = kSizes[v];
        else if (dim == 1) t.shade_pixels = kSizes[v];
        else t.blocks_per_sm = v + 1;
        const double c = eval(t);
        // a move needs a 1% gain, so timing noise does not walk the search
        if (!bad && c < 0.99 * pick_cost) {
          pick = t;
          pick_cost = c;
        }
      }
      if (!bad && (pick.raster_tris != cur.raster_tris || pick.shade_pixels != cur.shade_pixels ||
                   pick.blocks_per_sm != cur.blocks_per_sm)) {
        cur = pick;
        cur_cost = pick_cost;
        moved = true;
      }
    }
    if (!moved) break;
  }
  if (evaluations) *evaluations = calls;
  if (bad) return fail(VS_ERR_INVALID_ARG, "the cost function returned a negative or NaN cost");
  *best = cur;
  return VS_OK;
}

vs_status vs_autotune_batch(vs_ctx* ctx, const vs_batch_item* items, int32_t n, const float* bg, int32_t do_backward,
                            void* workspace, size_t ws_bytes, uint32_t flags, vs_stream_t stream, int32_t repeats,
                            vs_tuning* best) {
  NvtxRange nvtx_range("vs_autotune_batch");
  if (repeats < 1 || repeats > 16) return fail(VS_ERR_INVALID_ARG, "repeats %d out of [1, 16]", repeats);
  if (!ctx || !items) return fail(VS_ERR_INVALID_ARG, "NULL argument");
  if (n < 1) return fail(VS_ERR_INVALID_ARG, "n = %d < 1", n);
  int kmax = 1;
  for (int j = 0; j < n; ++j)
    if (items[j].obj) kmax = std::max(kmax, std::min((int)items[j].obj->k, VS_MAX_SHELLS));
  const int b = do_backward ? 1 : 0;
  const vs_tuning start = lookup_tuning(ctx, b, kmax);
  int most = 1;
  {  // validate the whole batch once before timing anything
    Plan P;
    int km = 1;
    vs_status s = plan_batch(ctx, items, n, bg, do_backward, workspace, ws_bytes, flags, start, P, &km);
    if (s != VS_OK) return s;
    most = P.full ? ctx->persist_blocks_full[b][kmax] : ctx->persist_blocks[b][P.tc][kmax];
  }
  vs_status s = set_device(ctx);
  if (s != VS_OK) return s;
  AutotuneJob J{ctx, items, n, bg, do_backward, workspace, ws_bytes, flags & ~VS_FLAG_TEST_STALL,
                reinterpret_cast<cudaStream_t>(stream), repeats, {nullptr, nullptr}, VS_OK, std::string()};
  cudaError_t e = cudaEventCreate(&J.ev[0]);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
  if ((e = cudaEventCreate(&J.ev[1])) != cudaSuccess) {
    cudaEventDestroy(J.ev[0]);
    return cuda_fail(e, "cudaEventCreate");
  }
  vs_tuning won{};
  s = vs_tune_search(&start, most, autotune_cost, &J, &won, nullptr);
  cudaEventDestroy(J.ev[0]);
  cudaEventDestroy(J.ev[1]);
  if (J.status != VS_OK) return fail(J.status, "%s", J.error.c_str());
  if (s != VS_OK) return s;
  {
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    ctx->tune[b][kmax] = won;
    ctx->tune_set[b][kmax] = true;
  }
  if (best) *best = won;
  return VS_OK;
}

// --- neural texture -----------------------------------------------------------------

}  // extern "C"

namespace {

vs_status check_ntex(const vs_ntex_config* c) {
  if (!c) return fail(VS_ERR_INVALID_ARG, "config is NULL");
  if (c->levels < 1 || c->levels > 16) return fail(VS_ERR_INVALID_ARG, "levels %d out of [1, 16]", c->levels);
  if (c->features < 1 || c->features > 8) return fail(VS_ERR_INVALID_ARG, "features %d out of [1, 8]", c->features);
  if (c->log2_table < 2 || c->log2_table > 24)
    return fail(VS_ERR_INVALID_ARG, "log2_table %d out of [2, 24]", c->log2_table);
  if (c->base_res < 1) return fail(VS_ERR_INVALID_ARG, "base_res %d < 1", c->base_res);
  if (!(c->growth >= 1.0f && c->growth <= 4.0f)) return fail(VS_ERR_INVALID_ARG, "growth out of [1, 4]");
  if ((double)c->base_res * std::pow((double)c->growth, c->levels - 1) > (double)(1 << 20))
    return fail(VS_ERR_INVALID_ARG, "finest level resolution above 2^20");
  if (c->hidden < 1 || c->hidden > 512) return fail(VS_ERR_INVALID_ARG, "hidden %d out of [1, 512]", c->hidden);
  if (c->out_ch < 1 || c->out_ch > 256) return fail(VS_ERR_INVALID_ARG, "out_ch %d out of [1, 256]", c->out_ch);
  if (c->tensor_cores != 0 && c->tensor_cores != 1) return fail(VS_ERR_INVALID_ARG, "tensor_cores must be 0 or 1");
  return VS_OK;
}

vs_status check_ntex_call(vs_ctx* ctx, const vs_ntex_config* cfg, const void* params, int32_t W, int32_t H,
                          const void* texels, int32_t pitch, int32_t ch0, void* ws, size_t ws_bytes) {
  vs_status s = check_ntex(cfg);
  if (s != VS_OK) return s;
  if (!ctx || !params || !texels) return fail(VS_ERR_INVALID_ARG, "NULL argument");
  if (W < 1 || H < 1 || W > 65536 || H > 65536 || (long long)W * H > (1ll << 30))
    return fail(VS_ERR_INVALID_ARG, "texture %dx%d out of range", W, H);
  if (ch0 < 0 || pitch < 1 || ch0 + cfg->out_ch > pitch)
    return fail(VS_ERR_INVALID_ARG, "channels [%d, %d) do not fit pitch %d", ch0, ch0 + cfg->out_ch, pitch);
  if ((uintptr_t)params % 4) return fail(VS_ERR_INVALID_ARG, "params must be 4-byte aligned");
  const int rows = (long long)W * H < vsntex::kNtexChunk ? W * H : vsntex::kNtexChunk;
  if (!ws || (uintptr_t)ws % 256) return fail(VS_ERR_WORKSPACE, "workspace NULL or not 256-byte aligned");
  const size_t need = vsntex::ws_floats(*cfg, rows) * sizeof(float);
  if (ws_bytes < need) return fail(VS_ERR_WORKSPACE, "workspace has %zu bytes, needs %zu", ws_bytes, need);
  return VS_OK;
}

vs_status ntex_status(int r, const char* what) {
  if (r == 0) return VS_OK;
  return cuda_fail((cudaError_t)r, what);
}

}  // namespace

extern "C" {

vs_status vs_ntex_layout(const vs_ntex_config* cfg, int64_t offsets[7], int64_t* total) {
  vs_status s = check_ntex(cfg);
  if (s != VS_OK) return s;
  const int64_t L = cfg->levels, T = 1ll << cfg->log2_table, F = cfg->features, H = cfg->hidden, C = cfg->out_ch;
  const int64_t sz[7] = {L * T * F, H * L * F, H, H * H, H, C * H, C};
  int64_t off = 0;
  for (int i = 0; i < 7; ++i) {
    if (offsets) offsets[i] = off;
    off += sz[i];
  }
  if (total) *total = off;
  return VS_OK;
}

vs_status vs_ntex_workspace_size(const vs_ntex_config* cfg, int32_t tex_w, int32_t tex_h, size_t* bytes) {
  vs_status s = check_ntex(cfg);
  if (s != VS_OK) return s;
  if (!bytes) return fail(VS_ERR_INVALID_ARG, "bytes is NULL");
  if (tex_w < 1 || tex_h < 1) return fail(VS_ERR_INVALID_ARG, "texture %dx%d out of range", tex_w, tex_h);
  const long long N = (long long)tex_w * tex_h;
  const int rows = N < vsntex::kNtexChunk ? (int)N : vsntex::kNtexChunk;
  *bytes = vsntex::ws_floats(*cfg, rows) * sizeof(float);
  return VS_OK;
}

vs_status vs_ntex_forward(vs_ctx* ctx, const vs_ntex_config* cfg, const float* params, int32_t tex_w, int32_t tex_h,
                          void* texels, int32_t dtype, int32_t pitch, int32_t ch0, void* workspace, size_t ws_bytes,
                          vs_stream_t stream) {
  NvtxRange nvtx_range("vs_ntex_forward");
  vs_status s = check_ntex_call(ctx, cfg, params, tex_w, tex_h, texels, pitch, ch0, workspace, ws_bytes);
  if (s != VS_OK) return s;
  if (dtype != 0 && dtype != 1) return fail(VS_ERR_INVALID_ARG, "dtype %d is neither 0 (f32) nor 1 (f16)", dtype);
  if ((s = set_device(ctx)) != VS_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return ntex_status(vsntex::forward(*cfg, params, tex_w, tex_h, texels, dtype, pitch, ch0, workspace, st),
                     "vs_ntex_forward");
}

vs_status vs_ntex_backward(vs_ctx* ctx, const vs_ntex_config* cfg, const float* params, int32_t tex_w, int32_t tex_h,
                           const float* grad_texels, int32_t pitch, int32_t ch0, float* grads, void* workspace,
                           size_t ws_bytes, vs_stream_t stream) {
  NvtxRange nvtx_range("vs_ntex_backward");
  vs_status s = check_ntex_call(ctx, cfg, params, tex_w, tex_h, grad_texels, pitch, ch0, workspace, ws_bytes);
  if (s != VS_OK) return s;
  if (!grads || (uintptr_t)grads % 4) return fail(VS_ERR_INVALID_ARG, "grads NULL or misaligned");
  if ((s = set_device(ctx)) != VS_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return ntex_status(vsntex::backward(*cfg, params, tex_w, tex_h, grad_texels, pitch, ch0, grads, workspace, st),
                     "vs_ntex_backward");
}

vs_status vs_adam_step(vs_ctx* ctx, float* params, const float* grads, float* m, float* v, int64_t n, float lr,
                       float beta1, float beta2, float eps, int32_t step, vs_stream_t stream) {
  NvtxRange nvtx_range("vs_adam_step");
  if (!ctx || !params || !grads || !m || !v) return fail(VS_ERR_INVALID_ARG, "NULL argument");
  if (n < 1 || step < 1) return fail(VS_ERR_INVALID_ARG, "n and step must be >= 1");
  if (!(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f && eps >= 0.0f))
    return fail(VS_ERR_INVALID_ARG, "beta1, beta2 in [0, 1) and eps >= 0 required");
  vs_status s = set_device(ctx);
  if (s != VS_OK) return s;
  return ntex_status(vsntex::adam(params, grads, m, v, n, lr, beta1, beta2, eps, step,
                                  reinterpret_cast<cudaStream_t>(stream)),
                     "vs_adam_step");
}

vs_status vs_read_stats(void* workspace, vs_stream_t stream, int32_t reset, vs_stats* out) {
  if (!workspace || !out) return fail(VS_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  WsHeader h;
  if ((e = cudaMemcpy(&h, workspace, sizeof h, cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
  out->device_status = h.status;
  out->fragments = h.frags;
  out->tris_front = h.front;
  out->tris_culled_back = h.back;
  out->tris_culled_near = h.nearc;
  out->tris_culled_guard = h.guard;
  out->tris_large = h.large;
  out->launches = h.launches;
  out->tris_clipped = h.clipped;
  out->kernel_class = h.kernel_class;
  out->reserved = 0;
  if (reset) {
    if ((e = cudaMemset(workspace, 0, sizeof h)) != cudaSuccess) return cuda_fail(e, "cudaMemset");
  }
  return VS_OK;
}

}  // extern "C"

// ===========================================================================
// Allocation-free forward (vs_render_noalloc).
//
// Some callers cannot allocate device memory: a render loop that must not
// allocate once it is running, or a plug-in inside a framework that owns and
// pools every byte of device memory and lends none out.  They cannot hand vs_render a workspace, so this
// entry point keeps its scratch in a fixed device array instead.  The array
// exists once per GPU that loads the library and stays until the process
// exits; its size is the limit on what one call may render.
// ===========================================================================
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;   // 16 MiB
constexpr int kNoAllocMaxDevices = 64;

std::mutex g_noalloc_mu;
char* g_noalloc_ptr[kNoAllocMaxDevices] = {};

}  // namespace

// The scratch itself.  Host code must not use this name as an address: it is
// a host-side stand-in; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

// Device address of the scratch on `device` (which must be current); looked
// up on the first call for that device and remembered.
vs_status noalloc_scratch(int device, char** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (device < 0 || device >= kNoAllocMaxDevices)
    return fail(VS_ERR_UNSUPPORTED, "vs_render_noalloc supports devices 0..%d", kNoAllocMaxDevices - 1);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_noalloc_ptr[device] = static_cast<char*>(p);
  }
  *out = g_noalloc_ptr[device];
  return VS_OK;
}

}  // namespace

extern "C" vs_status vs_render_noalloc(vs_ctx* ctx, const vs_object* obj, const vs_camera* cam, const float* bg,
                                       float* out_rgba, int32_t* hits, uint32_t flags, vs_stream_t stream) {
  NvtxRange nvtx_range("vs_render_noalloc");
  vs_status s = check_item(ctx, obj, cam);
  if (s != VS_OK) return s;
  if (!out_rgba) return fail(VS_ERR_INVALID_ARG, "out_rgba is NULL");
  if ((uintptr_t)out_rgba % 16) return fail(VS_ERR_INVALID_ARG, "out_rgba must be 16-byte aligned");
  ItemReq r{obj, cam, out_rgba, hits, nullptr, nullptr, nullptr};
  const uint32_t fl = flags & ~VS_FLAG_TEST_STALL;
  Plan P;
  if ((s = set_device(ctx)) != VS_OK) return s;
  if ((s = ensure_bounds(obj)) != VS_OK) return s;
  if ((s = make_plan(&r, 1, bg, 0, true, fl, nullptr, P)) != VS_OK) return s;
  if (P.total > kNoAllocScratchBytes)
    return fail(VS_ERR_OVERFLOW,
                "vs_render_noalloc needs %zu bytes of scratch for this object and camera; its fixed array holds "
                "%zu (use vs_render with a workspace)",
                P.total, kNoAllocScratchBytes);
  char* ws = nullptr;
  if ((s = noalloc_scratch(ctx->device, &ws)) != VS_OK) return s;
  if ((s = make_plan(&r, 1, bg, 0, true, fl, ws, P)) != VS_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: the header (status,
  // counters, work counter) must start at zero; the visibility words are
  // cleared by the setup kernel and the table is rewritten below
  cudaError_t e = cudaMemsetAsync(ws, 0, sizeof(WsHeader), st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(no-alloc header)");
  if ((s = upload_table(P, ws, vsk::plain_forward_launches(P.items[0].units), st)) != VS_OK) return s;
  e = vsk::plain_forward(table_ref(P, ws), P.items[0].units, P.tc, P.full, st);
  return e == cudaSuccess ? VS_OK : cuda_fail(e, "vs_render_noalloc launch");
}
