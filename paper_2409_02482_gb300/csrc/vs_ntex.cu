// Neural texture (Sec. 3 "Texturing Meshes"; the supplement's neural texture
// architecture): a 2D multiresolution hash encoding (the trainable
// positional encoding of Mueller et al. 2022) and an MLP of two ReLU hidden
// layers with a linear output, evaluated at the texel centres of the target
// resolution, so that the texture the renderer samples IS the network's
// prediction there ("grounded").  The adjoint takes the renderer's texel
// gradients (vs_render_backward / the fused batch) back to the hash tables
// and MLP parameters; vs_adam_step updates them.
//
// GB300 mapping: the encoding (a 4-corner gather per level) and its adjoint
// (a scatter with float atomics) are hand-written kernels, one thread per
// (texel, level); the three layers are dense contractions over the texels
// -- plain FP32 GEMMs through cuBLAS -- with bias/ReLU, texel writes and
// gradient gathers as small elementwise kernels.  Texels run in chunks of
// kChunk so that the activations fit a bounded workspace.

#include <cublas_v2.h>
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

// Corner c (dx = c & 1, dy = c >> 1) of level l at texel n: table row and weight.
__device__ __forceinline__ void corner(const Enc& e, int l, int tx, int ty, int W, int H, int c, uint32_t& row,
                                       float& w) {
  const int n = e.res[l];
  const float px = (tx + 0.5f) / (float)W * (float)n, py = (ty + 0.5f) / (float)H * (float)n;
  const float fx = floorf(px), fy = floorf(py);
  const float rx = px - fx, ry = py - fy;
  const int dx = c & 1, dy = c >> 1;
  const uint32_t c0 = (uint32_t)((int)fx + dx), c1 = (uint32_t)((int)fy + dy);
  const uint32_t T = 1u << e.logT;
  if ((uint64_t)(n + 1) * (uint64_t)(n + 1) <= T) row = c0 + c1 * (uint32_t)(n + 1);
  else row = (c0 ^ (c1 * kPrime)) & (T - 1u);
  w = (dx ? rx : 1.0f - rx) * (dy ? ry : 1.0f - ry);
}

// X[i, l F + f] = sum_corners w table[l, row, f] for texels n0 + i.
__global__ void __launch_bounds__(kThreads) k_encode(Enc e, const float* table, int W, int H, int n0, int count,
                                                      float* X) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)count * e.L) return;
  const int i = (int)(id / e.L), l = (int)(id - (long long)i * e.L);
  const int n = n0 + i, tx = n % W, ty = n / W;
  const size_t lt = (size_t)l << e.logT;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int c = 0; c < 4; ++c) {
    uint32_t row;
    float w;
    corner(e, l, tx, ty, W, H, c, row, w);
    const float* t = table + (lt + row) * e.F;
    for (int f = 0; f < e.F; ++f) acc[f] = fmaf(w, __ldg(t + f), acc[f]);
  }
  float* x = X + (size_t)i * e.L * e.F + l * e.F;
  for (int f = 0; f < e.F; ++f) x[f] = acc[f];
}

// dtable[l, row, f] += w dX[i, l F + f]  (the encoding's adjoint), level
// blockIdx.y.  Texels are row-major, so a segment of kSeg consecutive texels
// touches only a band of two or three vertex rows of a dense level: the
// block accumulates the segment's contributions to that band in shared
// memory and adds the band to the table once (a coarse level would
// otherwise receive millions of float atomics on a few hundred rows).
// Hashed levels (and bands too large for the buffer) scatter straight to
// the table, where rows are spread out.
constexpr int kSmemAcc = 12288;   // floats of band buffer (48 KB)
constexpr int kSeg = 4096;        // texels per segment

__device__ __forceinline__ int cell_row(const Enc& e, int l, int ty, int H) {
  return (int)floorf((ty + 0.5f) / (float)H * (float)e.res[l]);
}

// Run of consecutive lanes holding the same key: `start` = lane of the run's
// first member, `tail` = this lane ends the run.  The sentinel 0xffffffff
// (idle lanes) never matches a table row.
__device__ __forceinline__ void lane_run(uint32_t key, int lane, int& start, bool& tail) {
  const uint32_t prev = __shfl_up_sync(0xffffffffu, key, 1), next = __shfl_down_sync(0xffffffffu, key, 1);
  const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != key);
  start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
  tail = lane == 31 || next != key;
}
// Sum of v over the lanes [start, lane] (inclusive segmented scan).
__device__ __forceinline__ float run_scan(float v, int lane, int start) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane - o >= start) v += u;
  }
  return v;
}

__global__ void __launch_bounds__(kThreads) k_encode_bwd(Enc e, const float* dX, int W, int H, int n0, int count,
                                                          float* dtable) {
  extern __shared__ float acc[];
  const int l = blockIdx.y;
  const int n = e.res[l];
  const int lane = threadIdx.x & 31;
  // neighbouring texels share a cell (two or more texels per cell): a warp's
  // contributions to one row are added up across its lanes first, so that a
  // row takes one atomic per run instead of one per texel
  const bool runs = 2 * n <= W;                              // block-uniform
  const bool dense = (long long)(n + 1) * (n + 1) <= (1ll << e.logT);
  const size_t lt = (size_t)l << e.logT;
  const int nseg = (count + kSeg - 1) / kSeg;
  for (int seg = blockIdx.x; seg < nseg; seg += gridDim.x) {
    const int i0 = seg * kSeg, i1 = min(count, i0 + kSeg);
    int vb = 0, band = 0;
    if (dense) {
      const int cy0 = cell_row(e, l, (n0 + i0) / W, H), cy1 = cell_row(e, l, (n0 + i1 - 1) / W, H);
      vb = cy0 * (n + 1);
      band = (cy1 - cy0 + 2) * (n + 1);
    }
    const bool local = dense && band * e.F <= kSmemAcc;   // block-uniform
    if (local) {
      for (int r = threadIdx.x; r < band * e.F; r += blockDim.x) acc[r] = 0.0f;
      __syncthreads();
    }
    if (runs) {
      // whole warps step together (shuffles); idle lanes carry the sentinel
      for (int ib = i0 + (threadIdx.x & ~31); ib < i1; ib += blockDim.x) {
        const int i = ib + lane;
        const bool ok = i < i1;
        const int t = n0 + (ok ? i : i0), tx = t % W, ty = t / W;
        const float* d = dX + (size_t)(ok ? i : i0) * e.L * e.F + l * e.F;
        for (int c = 0; c < 4; ++c) {
          uint32_t row;
          float w;
          corner(e, l, tx, ty, W, H, c, row, w);
          int start;
          bool tail;
          lane_run(ok ? row : 0xffffffffu, lane, start, tail);
          for (int f = 0; f < e.F; ++f) {
            const float v = run_scan(ok ? w * d[f] : 0.0f, lane, start);
            if (ok && tail) {
              if (local) atomicAdd(acc + ((int)row - vb) * e.F + f, v);
              else atomicAdd(dtable + (lt + row) * e.F + f, v);
            }
          }
        }
      }
    } else {
      for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int t = n0 + i, tx = t % W, ty = t / W;
        const float* d = dX + (size_t)i * e.L * e.F + l * e.F;
        for (int c = 0; c < 4; ++c) {
          uint32_t row;
          float w;
          corner(e, l, tx, ty, W, H, c, row, w);
          for (int f = 0; f < e.F; ++f) {
            if (local) atomicAdd(acc + ((int)row - vb) * e.F + f, w * d[f]);
            else atomicAdd(dtable + (lt + row) * e.F + f, w * d[f]);
          }
        }
      }
    }
    if (local) {
      __syncthreads();
      float* t = dtable + (lt + vb) * e.F;
      for (int r = threadIdx.x; r < band * e.F; r += blockDim.x)
        if (acc[r] != 0.0f) atomicAdd(t + r, acc[r]);
      __syncthreads();   // the buffer is reused by the next segment
    }
  }
}

// Z[r, j] = act(Z[r, j] + b[j]); act = ReLU or identity.
__global__ void __launch_bounds__(kThreads) k_bias_act(float* Z, const float* b, int rows, int cols, int relu) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)rows * cols) return;
  const int j = (int)(id % cols);
  const float v = Z[id] + __ldg(b + j);
  Z[id] = relu ? fmaxf(v, 0.0f) : v;
}
// The same four values at a time (cols a multiple of 4; Z and b 16-byte aligned).
__global__ void __launch_bounds__(kThreads) k_bias_act4(float4* Z, const float* b, long long n4, int cols, int relu) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n4) return;
  const int j = (int)((4 * id) % cols);
  const float4 bb = __ldg(reinterpret_cast<const float4*>(b + j));
  float4 v = Z[id];
  v.x += bb.x;
  v.y += bb.y;
  v.z += bb.z;
  v.w += bb.w;
  if (relu) {
    v.x = fmaxf(v.x, 0.0f);
    v.y = fmaxf(v.y, 0.0f);
    v.z = fmaxf(v.z, 0.0f);
    v.w = fmaxf(v.w, 0.0f);
  }
  Z[id] = v;
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

unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

void bias_act(float* Z, const float* b, int rows, int cols, int relu, cudaStream_t st) {
  if (cols % 4 == 0 && ((uintptr_t)Z | (uintptr_t)b) % 16 == 0) {
    const long long n4 = (long long)rows * cols / 4;
    k_bias_act4<<<blocks_for(n4), kThreads, 0, st>>>(reinterpret_cast<float4*>(Z), b, n4, cols, relu);
  } else {
    k_bias_act<<<blocks_for((long long)rows * cols), kThreads, 0, st>>>(Z, b, rows, cols, relu);
  }
}

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

// Workspace carve for a chunk of `rows` texels.
struct Ws {
  float *X, *H1, *H2, *Y, *dY, *dH2, *dH1, *dX;
};

Ws carve(const vs_ntex_config& c, int rows, void* ws) {
  const size_t LF = (size_t)c.levels * c.features, H = c.hidden, C = c.out_ch;
  float* p = static_cast<float*>(ws);
  Ws w;
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
  return w;
}

size_t ws_floats(const vs_ntex_config& c, int rows) {
  const size_t LF = (size_t)c.levels * c.features, H = c.hidden, C = c.out_ch;
  auto r = [](size_t n) { return (n + 63) & ~(size_t)63; };
  return 2 * r(rows * LF) + 4 * r(rows * H) + 2 * r(rows * C);
}

// Row-major Y[rows, m] = A[rows, k] B[m, k]^T (+ beta Y), as column-major
// Y^T = B A^T.
cublasStatus_t gemm_abt(cublasHandle_t h, int rows, int m, int k, const float* A, const float* B, float* Y,
                        float beta) {
  const float one = 1.0f;
  return cublasSgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, m, rows, k, &one, B, k, A, k, &beta, Y, m);
}

// Row-major Y[rows, k] = A[rows, m] B[m, k], as column-major Y^T = B^T A^T.
cublasStatus_t gemm_ab(cublasHandle_t h, int rows, int k, int m, const float* A, const float* B, float* Y) {
  const float one = 1.0f, zero = 0.0f;
  return cublasSgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, k, rows, m, &one, B, k, A, m, &zero, Y, k);
}

// Row-major dW[m, k] += D[rows, m]^T A[rows, k], as column-major dW^T += A^T D.
cublasStatus_t gemm_atb_acc(cublasHandle_t h, int rows, int m, int k, const float* D, const float* A, float* dW) {
  const float one = 1.0f;
  return cublasSgemm(h, CUBLAS_OP_N, CUBLAS_OP_T, k, m, rows, &one, A, k, D, m, &one, dW, k);
}

#define VS_TRY_CUDA(x)                          \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return (int)e_;      \
  } while (0)
#define VS_TRY_BLAS(x)                                   \
  do {                                                   \
    if ((x) != CUBLAS_STATUS_SUCCESS) return -1000;      \
  } while (0)

// Forward of one chunk: activations X, H1, H2, Y in the workspace.
int chunk_forward(cublasHandle_t h, const vs_ntex_config& c, const Enc& e, const Views& P, int W, int H, int n0,
                  int rows, const Ws& w, cudaStream_t st) {
  const int LF = c.levels * c.features, Hd = c.hidden, C = c.out_ch;
  k_encode<<<blocks_for((long long)rows * c.levels), kThreads, 0, st>>>(e, P.table, W, H, n0, rows, w.X);
  VS_TRY_CUDA(cudaGetLastError());
  VS_TRY_BLAS(gemm_abt(h, rows, Hd, LF, w.X, P.W0, w.H1, 0.0f));
  bias_act(w.H1, P.b0, rows, Hd, 1, st);
  VS_TRY_BLAS(gemm_abt(h, rows, Hd, Hd, w.H1, P.W1, w.H2, 0.0f));
  bias_act(w.H2, P.b1, rows, Hd, 1, st);
  VS_TRY_BLAS(gemm_abt(h, rows, C, Hd, w.H2, P.W2, w.Y, 0.0f));
  bias_act(w.Y, P.b2, rows, C, 0, st);
  VS_TRY_CUDA(cudaGetLastError());
  return 0;
}

int forward(cublasHandle_t h, const vs_ntex_config& c, const float* params, int W, int H, void* texels, int dtype,
            int pitch, int ch0, void* ws, cudaStream_t st) {
  const float* v[7];
  views(c, params, v);
  const Views P{v[0], v[1], v[2], v[3], v[4], v[5], v[6]};
  const Enc e = make_enc(c);
  const int N = W * H;
  const int chunk = N < kNtexChunk ? N : kNtexChunk;
  const Ws w = carve(c, chunk, ws);
  for (int n0 = 0; n0 < N; n0 += chunk) {
    const int rows = N - n0 < chunk ? N - n0 : chunk;
    int r = chunk_forward(h, c, e, P, W, H, n0, rows, w, st);
    if (r) return r;
    k_write_texels<<<blocks_for((long long)rows * c.out_ch), kThreads, 0, st>>>(w.Y, c.out_ch, n0, rows, texels, dtype,
                                                                                 pitch, ch0);
    VS_TRY_CUDA(cudaGetLastError());
  }
  return 0;
}

int backward(cublasHandle_t h, const vs_ntex_config& c, const float* params, int W, int H, const float* grad_texels,
             int pitch, int ch0, float* grads, void* ws, cudaStream_t st) {
  const float* v[7];
  views(c, params, v);
  const Views P{v[0], v[1], v[2], v[3], v[4], v[5], v[6]};
  float* g[7];
  views(c, grads, g);
  const Enc e = make_enc(c);
  const int N = W * H;
  const int LF = c.levels * c.features, Hd = c.hidden, C = c.out_ch;
  const int chunk = N < kNtexChunk ? N : kNtexChunk;
  const Ws w = carve(c, chunk, ws);
  for (int n0 = 0; n0 < N; n0 += chunk) {
    const int rows = N - n0 < chunk ? N - n0 : chunk;
    int r = chunk_forward(h, c, e, P, W, H, n0, rows, w, st);   // recompute the activations
    if (r) return r;
    k_gather_grad<<<blocks_for((long long)rows * C), kThreads, 0, st>>>(grad_texels, C, n0, rows, pitch, ch0, w.dY);
    VS_TRY_CUDA(cudaGetLastError());
    // output layer
    VS_TRY_BLAS(gemm_atb_acc(h, rows, C, Hd, w.dY, w.H2, g[5]));
    relu_colsum(w.dY, nullptr, rows, C, g[6], st);
    VS_TRY_BLAS(gemm_ab(h, rows, Hd, C, w.dY, P.W2, w.dH2));
    relu_colsum(w.dH2, w.H2, rows, Hd, g[4], st);
    // second hidden layer
    VS_TRY_BLAS(gemm_atb_acc(h, rows, Hd, Hd, w.dH2, w.H1, g[3]));
    VS_TRY_BLAS(gemm_ab(h, rows, Hd, Hd, w.dH2, P.W1, w.dH1));
    relu_colsum(w.dH1, w.H1, rows, Hd, g[2], st);
    // first hidden layer and the encoding
    VS_TRY_BLAS(gemm_atb_acc(h, rows, Hd, LF, w.dH1, w.X, g[1]));
    VS_TRY_BLAS(gemm_ab(h, rows, LF, Hd, w.dH1, P.W0, w.dX));
    {
      const unsigned nseg = (unsigned)((rows + kSeg - 1) / kSeg);
      const unsigned gx = nseg < 256u ? nseg : 256u;
      k_encode_bwd<<<dim3(gx, c.levels), kThreads, kSmemAcc * sizeof(float), st>>>(e, w.dX, W, H, n0, rows, g[0]);
    }
    VS_TRY_CUDA(cudaGetLastError());
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
