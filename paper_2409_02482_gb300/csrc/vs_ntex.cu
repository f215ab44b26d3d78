// Neural texture (Sec. 3 "Texturing Meshes"; the supplement's neural texture
// architecture): a 2D multiresolution hash encoding (the trainable
// positional encoding of Mueller et al. 2022) and an MLP of two ReLU hidden
// layers with a linear output, evaluated at the texel centres of the target
// resolution, so that the texture the renderer samples IS the network's
// prediction there ("grounded").  The adjoint takes the renderer's texel
// gradients (vs_render_backward / the fused batch) back to the hash tables
// and MLP parameters; vs_adam_step updates them.
//
// GB300 mapping.  FP32 layers (the default): per chunk of kNtexChunk texels
// the encoding (a 4-corner gather per level, one thread per (texel, level)),
// the three layers as hand-written GEMM kernels on the FP32 pipes with their
// elementwise work fused in (bias and ReLU in the forward's epilogue, the
// ReLU mask and the bias gradient's column sums in the adjoint's), so that
// the activations (64 MB per layer at 2^18 texels) stay within L2 between
// layers and in a bounded workspace.  TF32 layers (cfg.tensor_cores): one
// fused persistent kernel each way, the layers on the tensor cores (tcgen05,
// FP32 accumulators in tensor memory; vs_ntex_tc.cuh).  Both modes take the
// encoding's adjoint in k_table_grad, by 2D tiles of texels (register runs
// down columns, a shared vertex box per tile).

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "vs.h"
#include "vs_ntex.h"

namespace vsn {

constexpr uint32_t kPrime = 2654435761u;
constexpr int kThreads = 256;

struct Enc {
  int L, F, logT, base;
  float growth;
  int res[16];
};

// Level resolutions N_l = floor(N_min b^l), computed on the host in double.
Enc make_enc(const vs_ntex_config& c) {
  Enc e{};
  e.L = c.levels;
  e.F = c.features;
  e.logT = c.log2_table;
  e.base = c.base_res;
  e.growth = c.growth;
  for (int l = 0; l < c.levels; ++l) e.res[l] = (int)std::floor((double)c.base_res * std::pow((double)c.growth, l));
  return e;
}

// Table row of lattice vertex (c0, c1) of level l: dense indexing while the
// level's (N_l + 1)^2 vertices fit the table, else the spatial hash.
__device__ __forceinline__ uint32_t table_row(const Enc& e, int l, uint32_t c0, uint32_t c1) {
  const int n = e.res[l];
  const uint32_t T = 1u << e.logT;
  if ((uint64_t)(n + 1) * (uint64_t)(n + 1) <= T) return c0 + c1 * (uint32_t)(n + 1);
  return (c0 ^ (c1 * kPrime)) & (T - 1u);
}

// Lattice cell of texel coordinate v (of `ext` texels) at resolution n, and
// the fractional position r inside it.  The position p = (v + 1/2) n / ext
// is the fraction (2v + 1) n / (2 ext) of integers, so the cell is an exact
// integer quotient and r = remainder / (2 ext) carries one rounding (two
// with the reciprocal): the encoding's weights do not lose the ~n 2^-24 of
// a cell that a float evaluation of p would at fine levels.  Numerators
// below 2^24 (every texture up to 4096 texels a side with levels up to 2048
// cells) take the quotient from a float estimate corrected by one step.
__device__ __forceinline__ int lattice_cell(int v, int ext, int n, float& r) {
  const unsigned long long num = (unsigned long long)(2 * v + 1) * (unsigned)n;
  const unsigned den = 2u * (unsigned)ext;
  const float rcp = __frcp_rn((float)den);
  int q, rem;
  if (num < (1ull << 24)) {
    q = (int)__fmul_rz((float)num, rcp);
    rem = (int)num - q * (int)den;
    if (rem < 0) {
      --q;
      rem += (int)den;
    } else if (rem >= (int)den) {
      ++q;
      rem -= (int)den;
    }
  } else {
    q = (int)(num / den);
    rem = (int)(num - (unsigned long long)q * den);
  }
  r = __fmul_rn((float)rem, rcp);
  return q;
}

// The four corners of level l at texel (tx, ty): corner c (dx = c & 1,
// dy = c >> 1) has table row row[c] and weight w[c].
__device__ __forceinline__ void corners4(const Enc& e, int l, int tx, int ty, int W, int H, uint32_t row[4],
                                         float w[4]) {
  const int n = e.res[l];
  float rx, ry;
  const int fx = lattice_cell(tx, W, n, rx), fy = lattice_cell(ty, H, n, ry);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int dx = c & 1, dy = c >> 1;
    row[c] = table_row(e, l, (uint32_t)(fx + dx), (uint32_t)(fy + dy));
    w[c] = (dx ? rx : 1.0f - rx) * (dy ? ry : 1.0f - ry);
  }
}

// X[i, l F + f] = sum_corners w table[l, row, f] for texels n0 + i.
__global__ void __launch_bounds__(kThreads) k_encode(const __grid_constant__ Enc e, const float* table, int W, int H,
                                                      int n0, int count, float* X) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)count * e.L) return;
  const int i = (int)(id / e.L), l = (int)(id - (long long)i * e.L);
  const int n = n0 + i, tx = n % W, ty = n / W;
  const size_t lt = (size_t)l << e.logT;
  uint32_t row[4];
  float w[4];
  corners4(e, l, tx, ty, W, H, row, w);
  if (e.F == 2) {   // four 8-byte rows, all in flight; the same sums as below
    const float2* t2 = reinterpret_cast<const float2*>(table) + lt;
    float2 v[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = __ldg(t2 + row[c]);
    float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      a0 = fmaf(w[c], v[c].x, a0);
      a1 = fmaf(w[c], v[c].y, a1);
    }
    *reinterpret_cast<float2*>(X + (size_t)i * e.L * 2 + l * 2) = make_float2(a0, a1);
    return;
  }
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int c = 0; c < 4; ++c) {
    const float* t = table + (lt + row[c]) * e.F;
    for (int f = 0; f < e.F; ++f) acc[f] = fmaf(w[c], __ldg(t + f), acc[f]);
  }
  float* x = X + (size_t)i * e.L * e.F + l * e.F;
  for (int f = 0; f < e.F; ++f) x[f] = acc[f];
}

// The encoding's adjoint, dtable[l, row, f] += w dX[i, l F + f], by 2D
// tiles of texels: a block takes one tile of one level, 256 texel columns
// (one per thread) by the level's tile height.  Down its column a thread
// sums, in registers, the contributions of consecutive texels in the same
// lattice cell row (the x weights are constant down a column) and adds the
// cell's four corners when the cell row changes: into a shared-memory copy
// of the tile's vertex box, which is added to the table once per tile, or,
// at levels where a vertex meets few texels (the box would take more
// atomics than the texels' corners), straight into the table.  A coarse
// level thus takes a few atomics per tile instead of four per texel.
// Element (l, i, f) of dX (texel n0 + i) sits at dX[l sl + i si + f].
constexpr int kTgThreads = 256;
constexpr int kTgSmem = 12288;   // floats of the vertex box (48 KB)

struct TgPlan {
  int L, tiles_x, y_first, nrows;
  int ty[16];       // tile rows of level l
  int direct[16];   // 1: corners straight into the table
  int pre[17];      // first block of level l
};

// dst[0 .. F) += v[0 .. F) with vector reductions where F allows (8- and
// 16-byte aligned rows).
template <int F>
__device__ __forceinline__ void red_row(float* dst, const float* v) {
  if constexpr (F == 2) {
    asm volatile("red.relaxed.gpu.global.add.v2.f32 [%0], {%1, %2};" ::"l"(dst), "f"(v[0]), "f"(v[1]) : "memory");
  } else if constexpr (F % 4 == 0) {
#pragma unroll
    for (int f = 0; f < F; f += 4)
      asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst + f), "f"(v[f]),
                   "f"(v[f + 1]), "f"(v[f + 2]), "f"(v[f + 3])
                   : "memory");
  } else {
#pragma unroll
    for (int f = 0; f < F; ++f) atomicAdd(dst + f, v[f]);
  }
}

template <int F>
__global__ void __launch_bounds__(kTgThreads) k_table_grad(const __grid_constant__ Enc e,
                                                           const __grid_constant__ TgPlan p, const float* __restrict__ dX,
                                                           long long sl, int si, int W, int H, int n0, int count,
                                                           float* dtable) {
  extern __shared__ float box[];
  const int b = blockIdx.x;
  int l = 0;
  while (l + 1 < p.L && b >= p.pre[l + 1]) ++l;
  const int t = b - p.pre[l];
  const int n = e.res[l];
  const int x0 = (t % p.tiles_x) * kTgThreads;
  const int y0 = p.y_first + (t / p.tiles_x) * p.ty[l], y1 = min(y0 + p.ty[l], p.y_first + p.nrows);
  float r;
  const int bx0 = lattice_cell(x0, W, n, r), by0 = lattice_cell(y0, H, n, r);
  const int bxn = lattice_cell(min(x0 + kTgThreads - 1, W - 1), W, n, r) + 2 - bx0;
  const int byn = lattice_cell(y1 - 1, H, n, r) + 2 - by0;
  const int nbox = bxn * byn * F;
  const bool direct = p.direct[l] || nbox > kTgSmem;   // block-uniform
  float* tl = dtable + ((size_t)l << e.logT) * F;
  if (!direct) {
    for (int i = threadIdx.x; i < nbox; i += blockDim.x) box[i] = 0.0f;
    __syncthreads();
  }
  const int x = x0 + threadIdx.x;
  if (x < W) {
    float rx;
    const int cx = lattice_cell(x, W, n, rx);
    const float wx[2] = {1.0f - rx, rx};
    float acc[2][F];
    int cur = -1;
    // the four corners of cell row `cur` from the column's sums
    auto flush = [&]() {
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          if (wx[dx] == 0.0f) continue;
          float v[F];
          bool any = false;
#pragma unroll
          for (int f = 0; f < F; ++f) {
            v[f] = wx[dx] * acc[dy][f];
            any = any || v[f] != 0.0f;
          }
          if (!any) continue;
          const int vx = cx + dx, vy = cur + dy;
          if (direct) {
            red_row<F>(tl + (size_t)table_row(e, l, (uint32_t)vx, (uint32_t)vy) * F, v);
          } else {
            float* q = box + ((vy - by0) * bxn + (vx - bx0)) * F;
#pragma unroll
            for (int f = 0; f < F; ++f) atomicAdd(q + f, v[f]);
          }
        }
    };
    for (int y = y0; y < y1; ++y) {
      const long long nn = (long long)y * W + x;
      if (nn < n0 || nn >= (long long)n0 + count) continue;   // outside this chunk
      float ry;
      const int cy = lattice_cell(y, H, n, ry);
      if (cy != cur) {
        if (cur >= 0) flush();
        cur = cy;
#pragma unroll
        for (int f = 0; f < F; ++f) acc[0][f] = acc[1][f] = 0.0f;
      }
      const float* d = dX + l * sl + (nn - n0) * si;
#pragma unroll
      for (int f = 0; f < F; ++f) {
        const float v = __ldg(d + f);
        acc[0][f] += (1.0f - ry) * v;
        acc[1][f] += ry * v;
      }
    }
    if (cur >= 0) flush();
  }
  if (!direct) {
    __syncthreads();
    for (int i = threadIdx.x; i < bxn * byn; i += blockDim.x) {
      float v[F];
      bool any = false;
#pragma unroll
      for (int f = 0; f < F; ++f) {
        v[f] = box[i * F + f];
        any = any || v[f] != 0.0f;
      }
      if (!any) continue;
      const int vy = by0 + i / bxn, vx = bx0 + i % bxn;
      red_row<F>(tl + (size_t)table_row(e, l, (uint32_t)vx, (uint32_t)vy) * F, v);
    }
  }
}

// dZ = dH * (H > 0) for H the ReLU output (in place on dH).
__global__ void __launch_bounds__(kThreads) k_relu_bwd(float* dH, const float* H, long long n) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id < n && !(H[id] > 0.0f)) dH[id] = 0.0f;
}

// db[j] += sum_r dZ[r, j] -- one thread per column strip, atomics per block.
__global__ void __launch_bounds__(kThreads) k_colsum(const float* dZ, int rows, int cols, float* db) {
  const int j = blockIdx.y;
  float s = 0.0f;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) s += dZ[(size_t)r * cols + j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ float part[kThreads / 32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < kThreads / 32; ++w) t += part[w];
    atomicAdd(db + j, t);
  }
}

// db[j] += sum_r dZ[r, j] with dZ = dH * (H > 0) written back in place
// (H = null: dZ = dH, no write).  Row-major and coalesced: thread t of a
// block owns column t % cols of rows t / cols + RS k, RS = 256 / cols rows
// per step (cols <= 256); the block adds its per-column partials once.
__global__ void __launch_bounds__(kThreads) k_relu_colsum(float* dH, const float* H, int rows, int cols, float* db) {
  __shared__ float part[kThreads];
  const int RS = kThreads / cols;
  const int t = threadIdx.x;
  float s = 0.0f;
  if (t < RS * cols) {
    const int j = t % cols;
    for (long long r = (long long)blockIdx.x * RS + t / cols; r < rows; r += (long long)gridDim.x * RS) {
      const size_t o = (size_t)r * cols + j;
      float v = dH[o];
      if (H && !(H[o] > 0.0f)) {
        v = 0.0f;
        dH[o] = 0.0f;
      }
      s += v;
    }
  }
  part[t] = s;
  __syncthreads();
  if (t < cols) {
    float u = 0.0f;
    for (int k = 0; k < RS; ++k) u += part[t + k * cols];
    atomicAdd(db + t, u);
  }
}

// Texel values: channels [ch0, ch0 + C) of texel n0 + i from Y[i, :].
__global__ void __launch_bounds__(kThreads) k_write_texels(const float* Y, int C, int n0, int count, void* texels,
                                                            int dtype, int pitch, int ch0) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)count * C) return;
  const int i = (int)(id / C), c = (int)(id - (long long)i * C);
  const size_t off = (size_t)(n0 + i) * pitch + ch0 + c;
  if (dtype == 1) reinterpret_cast<__half*>(texels)[off] = __float2half_rn(Y[id]);
  else reinterpret_cast<float*>(texels)[off] = Y[id];
}

__global__ void __launch_bounds__(kThreads) k_gather_grad(const float* G, int C, int n0, int count, int pitch, int ch0,
                                                           float* dY) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)count * C) return;
  const int i = (int)(id / C), c = (int)(id - (long long)i * C);
  dY[id] = __ldg(G + (size_t)(n0 + i) * pitch + ch0 + c);
}

// Adam (Kingma & Ba) with bias correction.
__global__ void __launch_bounds__(kThreads) k_adam(float* p, const float* g, float* m, float* v, long long n, float lr,
                                                    float b1, float b2, float eps, float c1, float c2) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n) return;
  const float gi = g[id];
  const float mi = b1 * m[id] + (1.0f - b1) * gi;
  const float vi = b2 * v[id] + (1.0f - b2) * gi * gi;
  m[id] = mi;
  v[id] = vi;
  p[id] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ----------------------------------------------------------------------------
// GEMMs of the layers (FP32 pipes).  Row-major throughout; "rows" are texels.
// ----------------------------------------------------------------------------
// Epilogues of Y = A B^T: store, + bias, + bias and ReLU, or (adjoint) the
// ReLU mask of the forward activation H applied and the masked column sums
// added into db (the bias gradient).
enum { EPI_NONE = 0, EPI_BIAS = 1, EPI_BIAS_RELU = 2, EPI_MASK_COLSUM = 3 };

constexpr int kGM = 128, kGN = 64, kGK = 16;   // block tile of k_gemm_abt

// Y[r, n] = sum_k A[r, k] B[n, k] (A rows x K, B N x K) with epilogue EPI.
// 256 threads, each 8 rows x 4 columns of the 128 x 64 tile; k in slices of
// 16 staged through shared memory (A and B transposed there, so the inner
// loop reads broadcast float4s).  FMAs in k order: exact FP32 products and
// sums, no reduced-precision path.
template <int EPI>
__global__ void __launch_bounds__(kThreads) k_gemm_abt(const float* __restrict__ A, const float* __restrict__ B,
                                                        float* __restrict__ Y, int rows, int N, int K,
                                                        const float* __restrict__ bias, const float* __restrict__ H,
                                                        float* __restrict__ db) {
  __shared__ __align__(16) float As[kGK][kGM];
  __shared__ __align__(16) float Bs[kGK][kGN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;          // 4 columns tx * 4.., 8 rows ty * 8..
  const long long r0 = (long long)blockIdx.x * kGM;
  const int n0 = blockIdx.y * kGN;
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
  for (int k0 = 0; k0 < K; k0 += kGK) {
    // A tile: 128 rows x 16 k, 8 values per thread (k fastest: coalesced)
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + q * kThreads, rr = e >> 4, kk = e & 15;
      const long long r = r0 + rr;
      As[kk][rr] = (r < rows && k0 + kk < K) ? __ldg(A + r * K + k0 + kk) : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + q * kThreads, nn = e >> 4, kk = e & 15;
      Bs[kk][nn] = (n0 + nn < N && k0 + kk < K) ? __ldg(B + (size_t)(n0 + nn) * K + k0 + kk) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][ty * 8 + 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
  float csum[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const long long r = r0 + ty * 8 + i;
    if (r >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      float v = acc[i][j];
      if constexpr (EPI == EPI_BIAS || EPI == EPI_BIAS_RELU) v += __ldg(bias + n);
      if constexpr (EPI == EPI_BIAS_RELU) v = fmaxf(v, 0.0f);
      if constexpr (EPI == EPI_MASK_COLSUM) {
        if (!(__ldg(H + r * N + n) > 0.0f)) v = 0.0f;
        csum[j] += v;
      }
      Y[r * N + n] = v;
    }
  }
  if constexpr (EPI == EPI_MASK_COLSUM) {
    // column sums over the block's 128 rows: 16 row groups per column
    __syncthreads();
    float* part = &As[0][0];   // 16 x 64 floats
#pragma unroll
    for (int j = 0; j < 4; ++j) part[ty * kGN + tx * 4 + j] = csum[j];
    __syncthreads();
    if (tid < kGN && n0 + tid < N) {
      float t = 0.0f;
      for (int g = 0; g < 16; ++g) t += part[g * kGN + tid];
      atomicAdd(db + n0 + tid, t);
    }
  }
}

}  // namespace vsn

#include "vs_ntex_tc.cuh"

namespace vsn {

constexpr int kWN = 64, kWK = 64, kWR = 16;   // output tile and row slice of k_gemm_atb
constexpr int kWRows = 1024;                  // rows per block (split of the reduction)

// dW[n, k] += sum_r D[r, n] A[r, k] (D rows x N, A rows x K): the weight
// gradient, a reduction over the texels.  Block = one 64 x 64 tile of dW
// over kWRows rows, 4 x 4 outputs per thread; the partial tile is added
// into dW with one atomic per value.
__global__ void __launch_bounds__(kThreads) k_gemm_atb(const float* __restrict__ D, const float* __restrict__ A,
                                                        float* __restrict__ dW, int rows, int N, int K) {
  __shared__ __align__(16) float Ds[kWR][kWN];
  __shared__ __align__(16) float Xs[kWR][kWK];
  const int tid = threadIdx.x;
  const int tn = tid >> 4, tk = tid & 15;          // 4 n (tn * 4..), 4 k (tk * 4..)
  const int tiles_k = (K + kWK - 1) / kWK;
  const int n0 = (blockIdx.x / tiles_k) * kWN, k0 = (blockIdx.x % tiles_k) * kWK;
  const long long rb = (long long)blockIdx.y * kWRows;
  const long long re = rb + kWRows < rows ? rb + kWRows : rows;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
  for (long long s0 = rb; s0 < re; s0 += kWR) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + q * kThreads, rr = e >> 6, cc = e & 63;
      const long long r = s0 + rr;
      Ds[rr][cc] = (r < re && n0 + cc < N) ? __ldg(D + r * N + n0 + cc) : 0.0f;
      Xs[rr][cc] = (r < re && k0 + cc < K) ? __ldg(A + r * K + k0 + cc) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < kWR; ++rr) {
      const float4 d = *reinterpret_cast<const float4*>(&Ds[rr][tn * 4]);
      const float4 x = *reinterpret_cast<const float4*>(&Xs[rr][tk * 4]);
      const float dv[4] = {d.x, d.y, d.z, d.w}, xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(dv[i], xv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int n = n0 + tn * 4 + i;
    if (n >= N) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = k0 + tk * 4 + j;
      if (k < K && acc[i][j] != 0.0f) atomicAdd(dW + (size_t)n * K + k, acc[i][j]);
    }
  }
}

// Wt[k, n] = W[n, k] (W N x K): the adjoint's B operands.
__global__ void __launch_bounds__(kThreads) k_transpose(const float* __restrict__ W, float* __restrict__ Wt, int N,
                                                         int K) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)N * K) return;
  const int n = (int)(id / K), k = (int)(id - (long long)n * K);
  Wt[(size_t)k * N + n] = W[id];
}

unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// db += column sums of dZ, dZ = dH * (H > 0) in place (H may be null).
void relu_colsum(float* dH, const float* H, int rows, int cols, float* db, cudaStream_t st) {
  if (cols <= kThreads) {
    const long long steps = (rows + kThreads / cols - 1) / (kThreads / cols);
    const unsigned grid = (unsigned)(steps < 1216 ? steps : 1216);
    k_relu_colsum<<<grid, kThreads, 0, st>>>(dH, H, rows, cols, db);
  } else {
    if (H) k_relu_bwd<<<blocks_for((long long)rows * cols), kThreads, 0, st>>>(dH, H, (long long)rows * cols);
    k_colsum<<<dim3(64, cols), kThreads, 0, st>>>(dH, rows, cols, db);
  }
}

}  // namespace vsn

// ----------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------
namespace vsntex {

using namespace vsn;

struct Views {
  const float *table, *W0, *b0, *W1, *b1, *W2, *b2;
};

template <class P>
void views(const vs_ntex_config& c, P* base, P* out[7]) {
  const long long L = c.levels, T = 1ll << c.log2_table, F = c.features, H = c.hidden, C = c.out_ch;
  const long long sz[7] = {L * T * F, H * L * F, H, H * H, H, C * H, C};
  long long off = 0;
  for (int i = 0; i < 7; ++i) {
    out[i] = base + off;
    off += sz[i];
  }
}

// Workspace carve for a chunk of `rows` texels, plus the transposed weights
// of the adjoint; the first 256 bytes hold the status word (0, or
// kNtexTimeout when a tensor-core wait ran out).
struct Ws {
  int* status;
  float *X, *H1, *H2, *Y, *dY, *dH2, *dH1, *dX, *W2t, *W1t, *W0t;
};

Ws carve(const vs_ntex_config& c, int rows, void* ws) {
  const size_t LF = (size_t)c.levels * c.features, H = c.hidden, C = c.out_ch;
  float* p = static_cast<float*>(ws);
  Ws w;
  w.status = reinterpret_cast<int*>(p);
  p += 64;
  auto take = [&](size_t n) {
    float* q = p;
    p += (n + 63) & ~(size_t)63;   // 256-byte steps
    return q;
  };
  w.X = take(rows * LF);
  w.H1 = take(rows * H);
  w.H2 = take(rows * H);
  w.Y = take(rows * C);
  w.dY = take(rows * C);
  w.dH2 = take(rows * H);
  w.dH1 = take(rows * H);
  w.dX = take(rows * LF);
  w.W2t = take(H * C);
  w.W1t = take(H * H);
  w.W0t = take(H * LF);
  return w;
}

size_t ws_floats(const vs_ntex_config& c, int rows) {
  const size_t LF = (size_t)c.levels * c.features, H = c.hidden, C = c.out_ch;
  auto r = [](size_t n) { return (n + 63) & ~(size_t)63; };
  return 64 + 2 * r(rows * LF) + 4 * r(rows * H) + 2 * r(rows * C) + r(H * C) + r(H * H) + r(H * LF);
}

#define VS_TRY_CUDA(x)                          \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return (int)e_;      \
  } while (0)

// Dynamic shared memory of k_gemm_abt_tc for N x K operands, and the
// tensor-memory columns of its accumulator; the request also keeps the CTAs
// per SM within the 512 tensor-memory columns, so an allocation never waits.
struct TcShape {
  size_t smem;
  int cols;
};
TcShape tc_shape(int N, int K) {
  const int Kp = (K + 7) & ~7, Np = (N + 15) & ~15;
  int cols = 32;
  while (cols < Np) cols *= 2;
  size_t smem = sizeof(float) * (size_t)Kp * (kTcRows + Np) + 16;
  const size_t per_sm = 228 * 1024, floor_smem = per_sm / (512 / cols) + 1024;
  return {smem > floor_smem ? smem : floor_smem, cols};
}
constexpr size_t kTcMaxSmem = 200 * 1024;

template <int EPI>
int launch_tc(const float* A, const float* B, float* Y, int rows, int N, int K, const float* bias, const float* H,
              float* db, int* status, cudaStream_t st) {
  static bool configured = false;   // idempotent; a race only repeats the call
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_abt_tc<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTcMaxSmem);
    if (e != cudaSuccess) return (int)e;
    configured = true;
  }
  const TcShape s = tc_shape(N, K);
  k_gemm_abt_tc<EPI><<<(unsigned)((rows + kTcRows - 1) / kTcRows), kTcThreads, s.smem, st>>>(
      A, B, Y, rows, N, K, bias, H, db, status, s.cols, 1ll << 22);
  return (int)cudaGetLastError();
}

// Y = A B^T with epilogue epi (rows x N outputs, K inner): FP32 pipes, or
// the tensor cores in TF32 when tc and the operands fit (N <= 256).
int gemm_abt(bool tc, int epi, const float* A, const float* B, float* Y, int rows, int N, int K, const float* bias,
             const float* H, float* db, int* status, cudaStream_t st) {
  if (tc && N <= 256 && tc_shape(N, K).smem <= kTcMaxSmem) {
    switch (epi) {
      case EPI_BIAS: return launch_tc<EPI_BIAS>(A, B, Y, rows, N, K, bias, H, db, status, st);
      case EPI_BIAS_RELU: return launch_tc<EPI_BIAS_RELU>(A, B, Y, rows, N, K, bias, H, db, status, st);
      case EPI_MASK_COLSUM: return launch_tc<EPI_MASK_COLSUM>(A, B, Y, rows, N, K, bias, H, db, status, st);
      default: return launch_tc<EPI_NONE>(A, B, Y, rows, N, K, bias, H, db, status, st);
    }
  }
  const dim3 grid((unsigned)((rows + kGM - 1) / kGM), (unsigned)((N + kGN - 1) / kGN));
  switch (epi) {
    case EPI_BIAS: k_gemm_abt<EPI_BIAS><<<grid, kThreads, 0, st>>>(A, B, Y, rows, N, K, bias, H, db); break;
    case EPI_BIAS_RELU: k_gemm_abt<EPI_BIAS_RELU><<<grid, kThreads, 0, st>>>(A, B, Y, rows, N, K, bias, H, db); break;
    case EPI_MASK_COLSUM:
      k_gemm_abt<EPI_MASK_COLSUM><<<grid, kThreads, 0, st>>>(A, B, Y, rows, N, K, bias, H, db);
      break;
    default: k_gemm_abt<EPI_NONE><<<grid, kThreads, 0, st>>>(A, B, Y, rows, N, K, bias, H, db);
  }
  return (int)cudaGetLastError();
}

// dW += D^T A over `rows` texels.
int gemm_atb(const float* D, const float* A, float* dW, int rows, int N, int K, cudaStream_t st) {
  const dim3 grid((unsigned)(((N + kWN - 1) / kWN) * ((K + kWK - 1) / kWK)), (unsigned)((rows + kWRows - 1) / kWRows));
  k_gemm_atb<<<grid, kThreads, 0, st>>>(D, A, dW, rows, N, K);
  return (int)cudaGetLastError();
}

#define VS_TRY(x)            \
  do {                       \
    int r_ = (x);            \
    if (r_) return r_;       \
  } while (0)

// Forward of one chunk: activations X, H1, H2, Y in the workspace.
// Tile plan of k_table_grad for texels n0 .. n0 + count of a W x H texture.
// Per level: the tallest power-of-two tile (at most 128 rows) whose vertex
// box fits the shared buffer, and the route with fewer atomics -- the box
// (every box vertex once per tile) or direct (the four corners of every run
// of texels down a column inside one cell row).
TgPlan tg_plan(const Enc& e, int W, int H, int n0, int count) {
  TgPlan p{};
  p.L = e.L;
  p.tiles_x = (W + kTgThreads - 1) / kTgThreads;
  p.y_first = n0 / W;
  p.nrows = (int)(((long long)n0 + count - 1) / W) - p.y_first + 1;
  const long long cols = W < kTgThreads ? W : kTgThreads;
  p.pre[0] = 0;
  for (int l = 0; l < e.L; ++l) {
    const long long n = e.res[l];
    const long long bx = ((cols - 1) * n + W - 1) / W + 3;   // box width bound (vertices)
    auto by = [&](long long ty) { return ((ty - 1) * n + H - 1) / H + 3; };
    int ty = 0;
    for (int c = 128; c >= 1 && ty == 0; c >>= 1)
      if (bx * by(c) * e.F <= kTgSmem) ty = c;
    bool direct = ty == 0;
    if (!direct) {
      const long long tiles = (long long)p.tiles_x * ((p.nrows + ty - 1) / ty);
      const long long runs = (long long)count * (n < H ? n : H) / H + W;
      direct = 4 * runs < tiles * bx * by(ty);
    }
    if (direct) ty = 16;
    p.ty[l] = ty;
    p.direct[l] = direct ? 1 : 0;
    p.pre[l + 1] = p.pre[l] + p.tiles_x * ((p.nrows + ty - 1) / ty);
  }
  return p;
}

// dtable += the encoding's adjoint of dX (element (l, i, f) at
// dX[l sl + i si + f]) for texels n0 .. n0 + count.
int table_grad(const Enc& e, const float* dX, long long sl, int si, int W, int H, int n0, int count, float* dtable,
               cudaStream_t st) {
  if (count <= 0) return 0;
  const TgPlan p = tg_plan(e, W, H, n0, count);
  const unsigned grid = (unsigned)p.pre[e.L];
  const size_t smem = kTgSmem * sizeof(float);
  switch (e.F) {
    case 1: k_table_grad<1><<<grid, kTgThreads, smem, st>>>(e, p, dX, sl, si, W, H, n0, count, dtable); break;
    case 2: k_table_grad<2><<<grid, kTgThreads, smem, st>>>(e, p, dX, sl, si, W, H, n0, count, dtable); break;
    case 3: k_table_grad<3><<<grid, kTgThreads, smem, st>>>(e, p, dX, sl, si, W, H, n0, count, dtable); break;
    case 4: k_table_grad<4><<<grid, kTgThreads, smem, st>>>(e, p, dX, sl, si, W, H, n0, count, dtable); break;
    case 5: k_table_grad<5><<<grid, kTgThreads, smem, st>>>(e, p, dX, sl, si, W, H, n0, count, dtable); break;
    case 6: k_table_grad<6><<<grid, kTgThreads, smem, st>>>(e, p, dX, sl, si, W, H, n0, count, dtable); break;
    case 7: k_table_grad<7><<<grid, kTgThreads, smem, st>>>(e, p, dX, sl, si, W, H, n0, count, dtable); break;
    default: k_table_grad<8><<<grid, kTgThreads, smem, st>>>(e, p, dX, sl, si, W, H, n0, count, dtable); break;
  }
  return (int)cudaGetLastError();
}

int chunk_forward(const vs_ntex_config& c, const Enc& e, const Views& P, int W, int H, int n0, int rows, const Ws& w,
                  cudaStream_t st) {
  const int LF = c.levels * c.features, Hd = c.hidden, C = c.out_ch;
  const bool tc = c.tensor_cores != 0;
  k_encode<<<blocks_for((long long)rows * c.levels), kThreads, 0, st>>>(e, P.table, W, H, n0, rows, w.X);
  VS_TRY_CUDA(cudaGetLastError());
  VS_TRY(gemm_abt(tc, EPI_BIAS_RELU, w.X, P.W0, w.H1, rows, Hd, LF, P.b0, nullptr, nullptr, w.status, st));
  VS_TRY(gemm_abt(tc, EPI_BIAS_RELU, w.H1, P.W1, w.H2, rows, Hd, Hd, P.b1, nullptr, nullptr, w.status, st));
  VS_TRY(gemm_abt(tc, EPI_BIAS, w.H2, P.W2, w.Y, rows, C, Hd, P.b2, nullptr, nullptr, w.status, st));
  return 0;
}

// The fused tensor-core forward (TF32 mode) for networks of 64-wide hidden
// layers with at most 64 encoding values and outputs; one persistent launch
// over the whole texture.  Returns -1 when the shape is not covered.
int fused_forward_tc(const vs_ntex_config& c, const Views& P, const Enc& e, int W, int H, void* texels, int dtype,
                     int pitch, int ch0, int* status, cudaStream_t st) {
  const int LF = c.levels * c.features;
  if (!c.tensor_cores || c.hidden != kMlpH || LF > 64 || c.out_ch > 64) return -1;
  const int smem = mlp_fwd_smem(LF, c.out_ch);
  static bool configured = false;
  if (!configured) {
    cudaError_t err = cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (err != cudaSuccess) return (int)err;
    configured = true;
  }
  int dev = 0, sms = 0;
  VS_TRY_CUDA(cudaGetDevice(&dev));
  VS_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // two CTAs per SM at most: 2 x 256 tensor-memory columns, and the shared
  // memory of a third would not fit
  const int per_sm = 2 * (smem + 1024) <= 228 * 1024 ? 2 : 1;
  MlpFwdArgs a{P.table, P.W0, P.b0, P.W1, P.b1, P.W2, P.b2, texels, W, H, W * H, c.out_ch, LF, dtype, pitch, ch0,
               status, 1ll << 22};
  k_mlp_fwd_tc<<<sms * per_sm, kFwdThreads, smem, st>>>(a, e);
  return (int)cudaGetLastError();
}

int forward(const vs_ntex_config& c, const float* params, int W, int H, void* texels, int dtype, int pitch, int ch0,
            void* ws, cudaStream_t st) {
  const float* v[7];
  views(c, params, v);
  const Views P{v[0], v[1], v[2], v[3], v[4], v[5], v[6]};
  const Enc e = make_enc(c);
  const int N = W * H;
  {
    const int r = fused_forward_tc(c, P, e, W, H, texels, dtype, pitch, ch0, carve(c, 1, ws).status, st);
    if (r >= 0) return r;
  }
  const int chunk = N < kNtexChunk ? N : kNtexChunk;
  const Ws w = carve(c, chunk, ws);
  for (int n0 = 0; n0 < N; n0 += chunk) {
    const int rows = N - n0 < chunk ? N - n0 : chunk;
    VS_TRY(chunk_forward(c, e, P, W, H, n0, rows, w, st));
    k_write_texels<<<blocks_for((long long)rows * c.out_ch), kThreads, 0, st>>>(w.Y, c.out_ch, n0, rows, texels, dtype,
                                                                                 pitch, ch0);
    VS_TRY_CUDA(cudaGetLastError());
  }
  return 0;
}

// The fused tensor-core adjoint (TF32 mode) for 64-wide hidden layers, at
// most 32 encoding values with F dividing 16, and at most 32 outputs; one
// persistent launch over the whole texture.  -1 when not covered.
int fused_backward_tc(const vs_ntex_config& c, const Views& P, float* const g[7], const Enc& e, int W, int H,
                      const float* grad, int pitch, int ch0, void* ws, cudaStream_t st) {
  const int LF = c.levels * c.features;
  if (!c.tensor_cores || c.hidden != kMlpH || LF > 32 || c.out_ch > 32 || 16 % c.features != 0) return -1;
  const int smem = mlp_bwd_smem(LF, c.out_ch);
  if (smem > 227 * 1024) return -1;
  static bool configured = false;
  if (!configured) {
    cudaError_t err = cudaFuncSetAttribute(k_mlp_bwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (err != cudaSuccess) return (int)err;
    configured = true;
  }
  int dev = 0, sms = 0;
  VS_TRY_CUDA(cudaGetDevice(&dev));
  VS_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // chunks of texels whose level-major dX fits the workspace (sized for
  // kNtexChunk texels of every activation: at least four times this)
  const int N = W * H;
  const int rows_ws = N < kNtexChunk ? N : kNtexChunk;
  const int chunk = N < 4 * rows_ws ? N : 4 * rows_ws;
  const Ws w = carve(c, 1, ws);
  float* dX = reinterpret_cast<float*>(ws) + 64;
  for (int n0 = 0; n0 < N; n0 += chunk) {
    const int count = N - n0 < chunk ? N - n0 : chunk;
    MlpBwdArgs a{P.table, P.W0, P.b0, P.W1, P.b1, P.W2, grad, g[1], g[2], g[3], g[4], g[5], g[6], dX,
                 W, H, n0, count, c.out_ch, LF, c.features, pitch, ch0, w.status, 1ll << 22};
    k_mlp_bwd_tc<<<sms, kBwdThreads, smem, st>>>(a, e);   // one CTA per SM (shared memory)
    VS_TRY_CUDA(cudaGetLastError());
    VS_TRY(table_grad(e, dX, (long long)count * c.features, c.features, W, H, n0, count, g[0], st));
  }
  return 0;
}

int backward(const vs_ntex_config& c, const float* params, int W, int H, const float* grad_texels, int pitch, int ch0,
             float* grads, void* ws, cudaStream_t st) {
  const float* v[7];
  views(c, params, v);
  const Views P{v[0], v[1], v[2], v[3], v[4], v[5], v[6]};
  float* g[7];
  views(c, grads, g);
  const Enc e = make_enc(c);
  {
    const int r = fused_backward_tc(c, P, g, e, W, H, grad_texels, pitch, ch0, ws, st);
    if (r >= 0) return r;
  }
  const int N = W * H;
  const int LF = c.levels * c.features, Hd = c.hidden, C = c.out_ch;
  const bool tc = c.tensor_cores != 0;
  const int chunk = N < kNtexChunk ? N : kNtexChunk;
  const Ws w = carve(c, chunk, ws);
  // the adjoint's B operands: W2^T, W1^T, W0^T
  k_transpose<<<blocks_for((long long)C * Hd), kThreads, 0, st>>>(P.W2, w.W2t, C, Hd);
  k_transpose<<<blocks_for((long long)Hd * Hd), kThreads, 0, st>>>(P.W1, w.W1t, Hd, Hd);
  k_transpose<<<blocks_for((long long)Hd * LF), kThreads, 0, st>>>(P.W0, w.W0t, Hd, LF);
  VS_TRY_CUDA(cudaGetLastError());
  for (int n0 = 0; n0 < N; n0 += chunk) {
    const int rows = N - n0 < chunk ? N - n0 : chunk;
    VS_TRY(chunk_forward(c, e, P, W, H, n0, rows, w, st));   // recompute the activations
    k_gather_grad<<<blocks_for((long long)rows * C), kThreads, 0, st>>>(grad_texels, C, n0, rows, pitch, ch0, w.dY);
    VS_TRY_CUDA(cudaGetLastError());
    // output layer: dW2 += dY^T H2, db2 += column sums of dY, dH2 = (dY W2) * (H2 > 0), db1 += its sums
    VS_TRY(gemm_atb(w.dY, w.H2, g[5], rows, C, Hd, st));
    relu_colsum(w.dY, nullptr, rows, C, g[6], st);
    VS_TRY(gemm_abt(tc, EPI_MASK_COLSUM, w.dY, w.W2t, w.dH2, rows, Hd, C, nullptr, w.H2, g[4], w.status, st));
    // second hidden layer: dW1 += dH2^T H1, dH1 = (dH2 W1) * (H1 > 0), db0 += its sums
    VS_TRY(gemm_atb(w.dH2, w.H1, g[3], rows, Hd, Hd, st));
    VS_TRY(gemm_abt(tc, EPI_MASK_COLSUM, w.dH2, w.W1t, w.dH1, rows, Hd, Hd, nullptr, w.H1, g[2], w.status, st));
    // first layer and the encoding: dW0 += dH1^T X, dX = dH1 W0
    VS_TRY(gemm_atb(w.dH1, w.X, g[1], rows, Hd, LF, st));
    VS_TRY(gemm_abt(tc, EPI_NONE, w.dH1, w.W0t, w.dX, rows, LF, Hd, nullptr, nullptr, nullptr, w.status, st));
    VS_TRY(table_grad(e, w.dX, c.features, (int)LF, W, H, n0, rows, g[0], st));
  }
  return 0;
}

int adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2, float eps, int step,
         cudaStream_t st) {
  const float c1 = (float)(1.0 - std::pow((double)b1, step)), c2 = (float)(1.0 - std::pow((double)b2, step));
  k_adam<<<blocks_for(n), kThreads, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
  return (int)cudaGetLastError();
}

}  // namespace vsntex
