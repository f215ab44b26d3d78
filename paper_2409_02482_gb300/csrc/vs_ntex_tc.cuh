// Tensor-core GEMM of the neural texture's layers (sm_103a, tcgen05): the
// TF32 mode of Y = A B^T with the same epilogues as the FP32 kernel.
//
// One CTA (4 warps) per 128 rows (texels).  The tile's rows of A [128 x K]
// and all of B [N x K] are staged in shared memory in the canonical K-major
// layout without swizzle -- 8-row x 16-byte core matrices, core matrices
// along K 128 bytes apart (LBO), 8-row groups K/4 * 128 bytes apart (SBO) --
// rounded to TF32 (cvt.rna).  One elected thread issues K/8
// tcgen05.mma.kind::tf32 (M = 128, N = N padded to 16, K = 8 each) into an
// FP32 accumulator in tensor memory and commits them to an mbarrier; every
// warp then reads its 32 rows of the accumulator (tcgen05.ld, lane = row)
// and applies the epilogue.  Waits are bounded: on expiry the CTA records
// VS_NTEX_TIMEOUT in the status word, waits (bounded) once more for its MMAs,
// frees its tensor memory and returns.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vsn {

constexpr int kTcThreads = 128;
constexpr int kTcRows = 128;
constexpr int kNtexTimeout = 1;   // status word value of a wait that ran out

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05): start address, LBO and SBO in
// 16-byte units, version 1, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of tcgen05
  return d;                 // base offset 0, relative LBO, layout type 0 (no swizzle)
}

// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major,
// M = 128, N (multiple of 16).
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4)            // D format: F32
         | (2u << 7)          // A format: TF32
         | (2u << 10)         // B format: TF32
         | ((uint32_t)(n >> 3) << 17)
         | ((uint32_t)(kTcRows >> 4) << 24);
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Bounded wait for phase `parity` of the mbarrier; false when it ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  const uint32_t a = smem_u32(bar);
  for (long long i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    __nanosleep(64);
  }
  return false;
}

// Y[r, n] = sum_k tf32(A[r, k]) tf32(B[n, k]) (FP32 accumulation) with
// epilogue EPI (as k_gemm_abt).  N <= 256, and shared memory for 128 rows
// and N rows of K (padded to 8) TF32 values; dynamic smem carries both
// operand tiles plus the mbarrier and the tensor-memory address.
template <int EPI>
__global__ void __launch_bounds__(kTcThreads) k_gemm_abt_tc(const float* __restrict__ A, const float* __restrict__ B,
                                                             float* __restrict__ Y, int rows, int N, int K,
                                                             const float* __restrict__ bias,
                                                             const float* __restrict__ H, float* __restrict__ db,
                                                             int* status, int tmem_cols, long long spin_limit) {
  extern __shared__ __align__(128) char tsm[];
  const int Kp = (K + 7) & ~7, Np = (N + 15) & ~15;
  const uint32_t sbo = (uint32_t)(Kp / 4) * 128u;   // between 8-row groups
  float* As = reinterpret_cast<float*>(tsm);                          // 128 rows
  float* Bs = As + (size_t)kTcRows * Kp;                              // Np rows
  uint64_t* bar = reinterpret_cast<uint64_t*>(Bs + (size_t)Np * Kp);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
  __shared__ float csum[4][256];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long r0 = (long long)blockIdx.x * kTcRows;

  // tensor memory (whole warp 0) and the mbarrier
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // operands, canonical K-major layout: element (m, k) at
  // (m / 8) sbo + (k / 4) 128 + (m % 8) 16 + (k % 4) 4 bytes
  for (int q = tid; q < kTcRows * (Kp / 4); q += kTcThreads) {
    const int m = q % kTcRows, c = q / kTcRows;
    const long long r = r0 + m;
    float v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k = 4 * c + e;
      v[e] = (r < rows && k < K) ? tf32_rna(__ldg(A + r * K + k)) : 0.0f;
    }
    *reinterpret_cast<float4*>(reinterpret_cast<char*>(As) + (m >> 3) * sbo + c * 128 + (m & 7) * 16) =
        make_float4(v[0], v[1], v[2], v[3]);
  }
  for (int q = tid; q < Np * (Kp / 4); q += kTcThreads) {
    const int n = q % Np, c = q / Np;
    float v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k = 4 * c + e;
      v[e] = (n < N && k < K) ? tf32_rna(__ldg(B + (size_t)n * K + k)) : 0.0f;
    }
    *reinterpret_cast<float4*>(reinterpret_cast<char*>(Bs) + (n >> 3) * sbo + c * 128 + (n & 7) * 16) =
        make_float4(v[0], v[1], v[2], v[3]);
  }
  // the operands are read by the tensor cores (async proxy)
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (tid == 0) {
    const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
    const uint32_t id = idesc_tf32(Np);
    for (int s = 0; s < Kp / 8; ++s) {   // K = 8 per instruction: two core matrices along K
      const uint64_t da = sdesc(a0 + s * 256u, 128u, sbo), dbd = sdesc(b0 + s * 256u, 128u, sbo);
      const uint32_t acc = s > 0 ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
          "l"(da), "l"(dbd), "r"(id), "r"(acc)
          : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
  }
  bool ok = mbar_wait(bar, 0, spin_limit);
  if (!ok) {
    if (tid == 0) atomicExch(status, kNtexTimeout);
    ok = mbar_wait(bar, 0, spin_limit);   // the MMAs must be done before the memory is freed
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // epilogue: warp w owns rows (lanes) 32 w .. 32 w + 31, 16 columns at a time
  const long long r = r0 + warp * 32 + lane;
  float cs[16];
  for (int n0 = 0; n0 < Np; n0 += 16) {
    uint32_t u[16];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)n0;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
          "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int n = n0 + j;
      float v = ok ? __uint_as_float(u[j]) : 0.0f;
      cs[j] = 0.0f;
      if (r < rows && n < N) {
        if constexpr (EPI == EPI_BIAS || EPI == EPI_BIAS_RELU) v += __ldg(bias + n);
        if constexpr (EPI == EPI_BIAS_RELU) v = fmaxf(v, 0.0f);
        if constexpr (EPI == EPI_MASK_COLSUM) {
          if (!(__ldg(H + r * N + n) > 0.0f)) v = 0.0f;
          cs[j] = v;
        }
        Y[r * N + n] = v;
      }
    }
    if constexpr (EPI == EPI_MASK_COLSUM) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        float t = cs[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) csum[warp][(n0 + j) & 255] = t;
      }
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if constexpr (EPI == EPI_MASK_COLSUM) {
    for (int n = tid; n < N; n += kTcThreads)
      atomicAdd(db + n, csum[0][n] + csum[1][n] + csum[2][n] + csum[3][n]);
  }
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

}  // namespace vsn

namespace vsn {

// ----------------------------------------------------------------------------
// Fused forward of the network on the tensor cores (TF32 mode): encoding ->
// layer 0 -> ReLU -> layer 1 -> ReLU -> output layer -> texels, for tiles
// of 128 texels, with the activations kept on chip (shared memory for the
// MMA operands, tensor memory for the accumulators).  Persistent: each CTA
// stages the three weight matrices once and loops over tiles.  Shapes: the
// encoding LF <= 64 values, hidden H = 64, outputs C <= 64.
// ----------------------------------------------------------------------------
constexpr int kMlpH = 64;

struct MlpFwdArgs {
  const float *table, *W0, *b0, *W1, *b1, *W2, *b2;
  void* texels;
  int W, H, N, C, LF, dtype, pitch, ch0;
  int* status;
  long long spin_limit;
};

// Bytes of a [rows x K] operand in the canonical layout (K padded to 8).
__host__ __device__ constexpr int op_bytes(int rows, int K) { return rows * ((K + 7) & ~7) * 4; }

// Element (m, k) of a canonical K-major operand with Kp (padded) columns.
__device__ __forceinline__ float* op_at(float* base, int m, int k, int Kp) {
  return reinterpret_cast<float*>(reinterpret_cast<char*>(base) + (m >> 3) * (Kp / 4) * 128 + (k >> 2) * 128 +
                                  (m & 7) * 16 + (k & 3) * 4);
}

// n_rows x K row-major global matrix -> canonical operand (TF32), rows
// beyond n_rows and columns beyond K zero, rows padded to rows_p.
__device__ __forceinline__ void stage_op(float* dst, const float* src, int n_rows, int rows_p, int K) {
  const int Kp = (K + 7) & ~7;
  for (int i = threadIdx.x; i < rows_p * Kp; i += blockDim.x) {
    const int m = i / Kp, k = i - m * Kp;
    *op_at(dst, m, k, Kp) = (m < n_rows && k < K) ? tf32_rna(__ldg(src + (size_t)m * K + k)) : 0.0f;
  }
}

// Encoding of texel (tx, ty), levels [l0, l1), into row m of the canonical
// operand X (TF32).  With two features per level the levels go four at a
// time, all sixteen corner rows (8 bytes each) loaded before any is used;
// the sums run in the same order as the generic loop.
__device__ __forceinline__ void encode_row(const Enc& e, const float* table, int tx, int ty, int W, int H, int l0,
                                           int l1, float* X, int m, int Kp) {
  if (e.F == 2) {
    const float2* t2 = reinterpret_cast<const float2*>(table);
    for (int lb = l0; lb < l1; lb += 4) {
      float2 v[4][4];
      float w[4][4];
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        const int l = lb + d < l1 ? lb + d : lb;
        const size_t lt = (size_t)l << e.logT;
        uint32_t row[4];
        corners4(e, l, tx, ty, W, H, row, w[d]);
#pragma unroll
        for (int c = 0; c < 4; ++c) v[d][c] = __ldg(t2 + lt + row[c]);
      }
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        if (lb + d < l1) {
          float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            a0 = fmaf(w[d][c], v[d][c].x, a0);
            a1 = fmaf(w[d][c], v[d][c].y, a1);
          }
          *op_at(X, m, 2 * (lb + d), Kp) = tf32_rna(a0);
          *op_at(X, m, 2 * (lb + d) + 1, Kp) = tf32_rna(a1);
        }
      }
    }
    return;
  }
  for (int l = l0; l < l1; ++l) {
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const size_t lt = (size_t)l << e.logT;
    uint32_t row[4];
    float w[4];
    corners4(e, l, tx, ty, W, H, row, w);
    for (int c = 0; c < 4; ++c) {
      const float* t = table + (lt + row[c]) * e.F;
      for (int f = 0; f < e.F; ++f) acc[f] = fmaf(w[c], __ldg(t + f), acc[f]);
    }
    for (int f = 0; f < e.F; ++f) *op_at(X, m, l * e.F + f, Kp) = tf32_rna(acc[f]);
  }
}

// Issues the MMAs of D[128 x Np] = A[128 x Kp] B[Np x Kp]^T (one thread)
// and, with commit, commits every MMA this thread issued so far to the
// mbarrier (one phase).
__device__ __forceinline__ void mma_tile(uint32_t d_tmem, const float* A, const float* B, int Kp, int Np,
                                         uint64_t* bar, bool commit = true) {
  const uint32_t a0 = smem_u32(A), b0 = smem_u32(B), sbo = (uint32_t)(Kp / 4) * 128u;
  const uint32_t id = idesc_tf32(Np);
  for (int s = 0; s < Kp / 8; ++s) {
    const uint64_t da = sdesc(a0 + s * 256u, 128u, sbo), dbd = sdesc(b0 + s * 256u, 128u, sbo);
    const uint32_t acc = s > 0 ? 1u : 0u;
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(da), "l"(dbd), "r"(id), "r"(acc)
        : "memory");
  }
  if (commit)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t u[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]),
        "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(u[j]);
}

// One commit's completion: bounded wait on the barrier's current phase;
// a wait that runs out records the status and is retried once (the tensor
// memory must not be freed under running MMAs); returns whether the
// results are valid.
__device__ __forceinline__ bool wait_mma(uint64_t* bar, uint32_t& phase, int* status, long long limit) {
  bool ok = mbar_wait(bar, phase, limit);
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(status, kNtexTimeout);
    ok = mbar_wait(bar, phase, limit);
  }
  phase ^= 1u;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return ok;
}

constexpr int kMlpTmemCols = 256;   // D0 [0, 64), D1 [64, 128), D2 [128, 128 + Cp)

// Four consecutive values k .. k + 3 (k % 4 == 0) of row m: one 16-byte
// access (a warp's 32 rows then cover 512 contiguous-in-groups bytes:
// 4 wavefronts, the least for 16-byte accesses).
__device__ __forceinline__ void st4(float* base, int m, int k, int Kp, float4 v) {
  *reinterpret_cast<float4*>(op_at(base, m, k, Kp)) = v;
}
// TF32(max(v + b, 0)) of four values (live: else zeros).
__device__ __forceinline__ float4 relu_tf32(const float* v, const float* b, bool live) {
  if (!live) return make_float4(0.f, 0.f, 0.f, 0.f);
  return make_float4(tf32_rna(fmaxf(v[0] + __ldg(b), 0.0f)), tf32_rna(fmaxf(v[1] + __ldg(b + 1), 0.0f)),
                     tf32_rna(fmaxf(v[2] + __ldg(b + 2), 0.0f)), tf32_rna(fmaxf(v[3] + __ldg(b + 3), 0.0f)));
}

// Dynamic shared memory of k_mlp_fwd_tc for LF inputs and C outputs.
__host__ __device__ constexpr int mlp_fwd_smem(int LF, int C) {
  return op_bytes(kMlpH, LF) + op_bytes(kMlpH, kMlpH) + op_bytes((C + 15) & ~15, kMlpH) + op_bytes(128, LF) +
         2 * op_bytes(128, kMlpH) + 256;
}

// 8 warps per CTA, as in the adjoint: warps w and w + 4 share a tensor-memory
// lane quarter (texel rows) and split the columns and the encoding's levels.
constexpr int kFwdThreads = 256;

__global__ void __launch_bounds__(kFwdThreads, 2) k_mlp_fwd_tc(const MlpFwdArgs a, const __grid_constant__ Enc e) {
  extern __shared__ __align__(128) char msm[];
  const int LFp = (a.LF + 7) & ~7, Cp = (a.C + 15) & ~15;
  float* W0s = reinterpret_cast<float*>(msm);
  float* W1s = W0s + kMlpH * LFp;
  float* W2s = W1s + kMlpH * kMlpH;
  float* Xs = W2s + Cp * kMlpH;
  float* H1s = Xs + 128 * LFp;
  float* H2s = H1s + 128 * kMlpH;
  uint64_t* bar = reinterpret_cast<uint64_t*>(H2s + 128 * kMlpH);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int half = tid >> 7, r = tid & 127;        // column half, texel row of the tile
  const int l_lo = half ? (e.L + 1) / 2 : 0, l_hi = half ? e.L : (e.L + 1) / 2;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kMlpTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  stage_op(W0s, a.W0, kMlpH, kMlpH, a.LF);
  stage_op(W1s, a.W1, kMlpH, kMlpH, kMlpH);
  stage_op(W2s, a.W2, a.C, Cp, kMlpH);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  uint32_t phase = 0;
  bool ok = true;
  const int tiles = (a.N + 127) / 128;
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    // encoding of texel n = 128 tile + r into row r of X (this half's levels)
    const int n = tile * 128 + r;
    if (n < a.N) encode_row(e, a.table, n % a.W, n / a.W, a.W, a.H, l_lo, l_hi, Xs, r, LFp);
    else
      for (int k = l_lo * e.F; k < l_hi * e.F; ++k) *op_at(Xs, r, k, LFp) = 0.0f;
    if (half == 0)
      for (int k = a.LF; k < LFp; ++k) *op_at(Xs, r, k, LFp) = 0.0f;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // layer 0
    if (tid == 0) mma_tile(tmem, Xs, W0s, LFp, kMlpH, bar);
    ok = wait_mma(bar, phase, a.status, a.spin_limit) && ok;
    for (int c0 = 32 * half; c0 < 32 * half + 32; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + lane_base + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 16; j += 4)
        st4(H1s, r, c0 + j, kMlpH, relu_tf32(v + j, a.b0 + c0 + j, true));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // layer 1
    if (tid == 0) mma_tile(tmem + 64u, H1s, W1s, kMlpH, kMlpH, bar);
    ok = wait_mma(bar, phase, a.status, a.spin_limit) && ok;
    for (int c0 = 32 * half; c0 < 32 * half + 32; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + lane_base + 64u + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 16; j += 4)
        st4(H2s, r, c0 + j, kMlpH, relu_tf32(v + j, a.b1 + c0 + j, true));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // output layer -> texels
    if (tid == 0) mma_tile(tmem + 128u, H2s, W2s, kMlpH, Cp, bar);
    ok = wait_mma(bar, phase, a.status, a.spin_limit) && ok;
    for (int c0 = 16 * half; c0 < Cp; c0 += 32) {
      float v[16];
      tmem_ld16(tmem + lane_base + 128u + (uint32_t)c0, v);
      if (n < a.N) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = c0 + j;
          if (c >= a.C) break;
          const float y = ok ? v[j] + __ldg(a.b2 + c) : 0.0f;
          const size_t off = (size_t)n * a.pitch + a.ch0 + c;
          if (a.dtype == 1) reinterpret_cast<__half*>(a.texels)[off] = __float2half_rn(y);
          else reinterpret_cast<float*>(a.texels)[off] = y;
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();   // X, H1, H2 and the accumulators are reused by the next tile
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMlpTmemCols) : "memory");
}

}  // namespace vsn

namespace vsn {

// ----------------------------------------------------------------------------
// Fused adjoint of the network on the tensor cores (TF32 mode), for tiles of
// 128 texels: the forward's hidden layers again (encoding, layer 0, layer 1),
// then dH2 = (dY W2) * (H2 > 0), dH1 = (dH2 W1) * (H1 > 0), dX = dH1 W0 on
// the tensor cores (the transposed weights staged once per CTA, K-major),
// dX written level-major for the encoding's adjoint (k_table_grad), and the
// weight and bias gradients accumulated in registers over the CTA's tiles
// (FP32 FMAs on the staged tiles, overlapping the tensor-core products) and
// added into the gradient vector once at the end.  Shapes: LF <= 32
// encoding values, hidden 64, C <= 32 outputs.
// ----------------------------------------------------------------------------
struct MlpBwdArgs {
  const float *table, *W0, *b0, *W1, *b1, *W2;
  const float* grad;   // dL/d(texels) [N, pitch], channels ch0 .. ch0 + C
  float *dW0, *db0, *dW1, *db1, *dW2, *db2;
  float* dX;           // dL/d(encoding) of texels n0 .. n0 + count, level-major [L][count][F]
  int W, H, n0, count, C, LF, F, pitch, ch0;
  int* status;
  long long spin_limit;
};

// dst (m, k) = src[k * src_cols + m]: the transpose of a row-major matrix as
// a canonical operand (TF32), zero outside rows x K.
__device__ __forceinline__ void stage_op_tr(float* dst, const float* src, int rows, int rows_p, int K, int src_cols) {
  const int Kp = (K + 7) & ~7;
  for (int i = threadIdx.x; i < rows_p * Kp; i += blockDim.x) {
    const int m = i / Kp, k = i - m * Kp;
    *op_at(dst, m, k, Kp) = (m < rows && k < K) ? tf32_rna(__ldg(src + (size_t)k * src_cols + m)) : 0.0f;
  }
}

__host__ __device__ constexpr int mlp_bwd_smem(int LF, int C) {
  return op_bytes(kMlpH, LF) + op_bytes(kMlpH, kMlpH) + op_bytes(kMlpH, C) + op_bytes(kMlpH, kMlpH) +
         op_bytes((LF + 15) & ~15, kMlpH) + op_bytes(128, LF) + 2 * op_bytes(128, kMlpH) + op_bytes(128, C) +
         2 * op_bytes(128, kMlpH) + 256;
}

__device__ __forceinline__ float4 ld4(const float* base, int m, int k, int Kp) {
  return *reinterpret_cast<const float4*>(op_at(const_cast<float*>(base), m, k, Kp));
}

// Writes the block barrier sequence around a phase whose shared-memory
// results feed the tensor cores.
__device__ __forceinline__ void sync_for_mma() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// kBwdWarps warps per CTA: warps w, w + 4, ... share the tensor-memory lane
// quarter (texel rows 32 (w % 4) ..) and split the columns (and the
// encoding's levels) between them; the weight gradients of a tile are summed
// by warp-level MMAs while the tensor cores run the next product.  16 warps
// (125 registers) hide more of the gathers' and products' latency than 8.
#ifndef VS_NTEX_BWD_WARPS
#define VS_NTEX_BWD_WARPS 16
#endif
constexpr int kBwdWarps = VS_NTEX_BWD_WARPS;   // 8 or 16: 2 or 4 warps per tensor-memory lane quarter
constexpr int kBwdThreads = 32 * kBwdWarps;
static_assert(kBwdWarps == 8 || kBwdWarps == 16, "column groups of 32 or 16 hidden units");

// Element (m, k) of a canonical operand tile as raw bits (an MMA fragment).
__device__ __forceinline__ uint32_t lds_u(const float* base, int m, int k, int Kp) {
  return __float_as_uint(*op_at(const_cast<float*>(base), m, k, Kp));
}
// D[16 x 8] += A[16 x 8] B[8 x 8], TF32 inputs, FP32 accumulators (one warp).
__device__ __forceinline__ void mma_tf32(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(kBwdThreads, 1) k_mlp_bwd_tc(const MlpBwdArgs a, const __grid_constant__ Enc e) {
  extern __shared__ __align__(128) char msm[];
  const int LF = a.LF, LFp = (LF + 7) & ~7, LF16 = (LF + 15) & ~15, Cp = (a.C + 7) & ~7;
  float* W0s = reinterpret_cast<float*>(msm);      // [64 x LF]   layer 0 B
  float* W1s = W0s + kMlpH * LFp;                  // [64 x 64]   layer 1 B
  float* W2Ts = W1s + kMlpH * kMlpH;               // [64 x C]    W2^T: B of dH2
  float* W1Ts = W2Ts + kMlpH * Cp;                 // [64 x 64]   W1^T: B of dH1
  float* W0Ts = W1Ts + kMlpH * kMlpH;              // [LF16 x 64] W0^T: B of dX
  float* Xs = W0Ts + LF16 * kMlpH;                 // [128 x LF]
  float* H1s = Xs + 128 * LFp;                     // [128 x 64]
  float* H2s = H1s + 128 * kMlpH;
  float* dYs = H2s + 128 * kMlpH;                  // [128 x C]
  float* dH2s = dYs + 128 * Cp;                    // [128 x 64]
  float* dH1s = dH2s + 128 * kMlpH;
  uint64_t* bar = reinterpret_cast<uint64_t*>(dH1s + 128 * kMlpH);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quad = tid >> 7, r = tid & 127;        // column group, texel row of the tile
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kMlpTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  stage_op(W0s, a.W0, kMlpH, kMlpH, LF);
  stage_op(W1s, a.W1, kMlpH, kMlpH, kMlpH);
  stage_op_tr(W2Ts, a.W2, kMlpH, kMlpH, a.C, kMlpH);
  stage_op_tr(W1Ts, a.W1, kMlpH, kMlpH, kMlpH, kMlpH);
  stage_op_tr(W0Ts, a.W0, LF, LF16, kMlpH, LF);
  sync_for_mma();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  uint32_t phase = 0;
  bool ok = true;

  // Weight and bias gradients of the tile, summed over its 128 texels with
  // warp-level TF32 MMAs (mma.sync m16n8k8) whose fragments are read
  // straight from the texel-major tiles: as a product over texels they want
  // texel-contiguous (transposed) operands, which tcgen05's TF32 K-major
  // descriptors would need as extra copies that do not fit shared memory.
  // FP32 accumulators in registers over the CTA's tiles.  Warp w:
  //   dW1 = dH2^T H1: rows 16 (w & 3) .. +15, J1 n8-tiles of columns from 8 J1 (w >> 2)
  //   dW2 = dY^T H2:  rows 16 (w & 1) .. +15, J2 n8-tiles from 8 J2 (w >> 1)
  //   dW0 = dH1^T X:  rows 16 (w & 3) .. +15, J0 n8-tiles from 8 J0 (w >> 2)
  //   db1, db0 (warps 0-3): the same A fragments times a matrix of ones
  //   db2: FP32 sums of dY per thread (kept exact: a plain sum)
  constexpr int J1 = 32 / kBwdWarps, J2 = 16 / kBwdWarps, J0 = 16 / kBwdWarps, NG = kBwdWarps / 4;
  constexpr int kDy = 32 / NG;                      // dY columns per thread at most (Cp <= 32)
  const int g = lane >> 2, tig = lane & 3;
  const int m1 = 16 * (warp & 3), n1 = 8 * J1 * (warp >> 2);
  const int m2 = 16 * (warp & 1), n2 = 8 * J2 * (warp >> 1);
  const int n0c = 8 * J0 * (warp >> 2);
  const bool do_w2 = m2 < Cp, bias = warp < 4;
  float acc1[J1][4], acc2[J2][4], acc0[J0][4], accb1[4], accb0[4], gb2[kDy];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    accb1[q] = accb0[q] = 0.0f;
#pragma unroll
    for (int j = 0; j < J1; ++j) acc1[j][q] = 0.0f;
#pragma unroll
    for (int j = 0; j < J2; ++j) acc2[j][q] = 0.0f;
#pragma unroll
    for (int j = 0; j < J0; ++j) acc0[j][q] = 0.0f;
  }
#pragma unroll
  for (int q = 0; q < kDy; ++q) gb2[q] = 0.0f;
  const uint32_t one = __float_as_uint(1.0f);
  const int l_lo = quad * e.L / NG, l_hi = (quad + 1) * e.L / NG;   // this group's levels
  const int cw = kMlpH / NG;                                        // hidden columns per group

  const int tiles = (a.count + 127) / 128;
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int i = tile * 128 + r, n = a.n0 + i;
    const bool live = i < a.count;
    const int tx = live ? n % a.W : 0, ty = live ? n / a.W : 0;
    // encoding of row r (this group's levels) and the output gradient (this
    // group's columns)
    if (live) encode_row(e, a.table, tx, ty, a.W, a.H, l_lo, l_hi, Xs, r, LFp);
    else
      for (int k = l_lo * e.F; k < l_hi * e.F; ++k) *op_at(Xs, r, k, LFp) = 0.0f;
    if (quad == 0)
      for (int k = LF; k < LFp; ++k) *op_at(Xs, r, k, LFp) = 0.0f;
    // dY kept in FP32 (the tensor cores read its TF32 part; the bias and
    // weight gradients of the output layer use all of it)
#pragma unroll
    for (int q = 0; q < kDy; ++q) {
      const int c = quad * (Cp / NG) + q;
      if (q < Cp / NG) {
        const float v = (live && c < a.C) ? __ldg(a.grad + (size_t)n * a.pitch + a.ch0 + c) : 0.0f;
        *op_at(dYs, r, c, Cp) = v;
        gb2[q] += v;
      }
    }
    sync_for_mma();
    // layer 0 -> H1
    if (tid == 0) mma_tile(tmem, Xs, W0s, LFp, kMlpH, bar);
    ok = wait_mma(bar, phase, a.status, a.spin_limit) && ok;
    for (int c0 = cw * quad; c0 < cw * quad + cw; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + lane_base + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 16; j += 4) st4(H1s, r, c0 + j, kMlpH, relu_tf32(v + j, a.b0 + c0 + j, live));
    }
    sync_for_mma();
    // layer 1 -> H2; dH2 = dY W2 (independent: issued together, one commit)
    if (tid == 0) {
      mma_tile(tmem + 64u, H1s, W1s, kMlpH, kMlpH, bar, false);
      mma_tile(tmem + 128u, dYs, W2Ts, Cp, kMlpH, bar);
    }
    ok = wait_mma(bar, phase, a.status, a.spin_limit) && ok;
    for (int c0 = cw * quad; c0 < cw * quad + cw; c0 += 16) {
      float v[16], u[16];
      tmem_ld16(tmem + lane_base + 64u + (uint32_t)c0, v);
      tmem_ld16(tmem + lane_base + 128u + (uint32_t)c0, u);
#pragma unroll
      for (int j = 0; j < 16; j += 4) {
        const float4 h2 = relu_tf32(v + j, a.b1 + c0 + j, live);
        st4(H2s, r, c0 + j, kMlpH, h2);
        st4(dH2s, r, c0 + j, kMlpH,
            make_float4(h2.x > 0.0f ? tf32_rna(u[j]) : 0.0f, h2.y > 0.0f ? tf32_rna(u[j + 1]) : 0.0f,
                        h2.z > 0.0f ? tf32_rna(u[j + 2]) : 0.0f, h2.w > 0.0f ? tf32_rna(u[j + 3]) : 0.0f));
      }
    }
    sync_for_mma();
    // dH1 = (dH2 W1) * (H1 > 0) on the tensor cores; meanwhile dW1 += dH2^T H1
    // (and db1) and dW2 += dY^T H2
    if (tid == 0) mma_tile(tmem, dH2s, W1Ts, kMlpH, kMlpH, bar);
    for (int k0 = 0; k0 < 128; k0 += 8) {
      const int ka = k0 + tig, kb = ka + 4;
      const uint32_t A[4] = {lds_u(dH2s, ka, m1 + g, kMlpH), lds_u(dH2s, ka, m1 + g + 8, kMlpH),
                             lds_u(dH2s, kb, m1 + g, kMlpH), lds_u(dH2s, kb, m1 + g + 8, kMlpH)};
#pragma unroll
      for (int j = 0; j < J1; ++j)
        mma_tf32(acc1[j], A, lds_u(H1s, ka, n1 + 8 * j + g, kMlpH), lds_u(H1s, kb, n1 + 8 * j + g, kMlpH));
      if (bias) mma_tf32(accb1, A, one, one);
      if (do_w2) {
        // dY holds FP32 values: rounded to TF32 here (rows beyond Cp are zero)
        auto dy = [&](int t, int c) { return c < Cp ? __float_as_uint(tf32_rna(*op_at(dYs, t, c, Cp))) : 0u; };
        const uint32_t A2[4] = {dy(ka, m2 + g), dy(ka, m2 + g + 8), dy(kb, m2 + g), dy(kb, m2 + g + 8)};
#pragma unroll
        for (int j = 0; j < J2; ++j)
          mma_tf32(acc2[j], A2, lds_u(H2s, ka, n2 + 8 * j + g, kMlpH), lds_u(H2s, kb, n2 + 8 * j + g, kMlpH));
      }
    }
    ok = wait_mma(bar, phase, a.status, a.spin_limit) && ok;
    for (int c0 = cw * quad; c0 < cw * quad + cw; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + lane_base + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 16; j += 4) {
        const float4 h1 = ld4(H1s, r, c0 + j, kMlpH);
        st4(dH1s, r, c0 + j, kMlpH,
            make_float4(h1.x > 0.0f ? tf32_rna(v[j]) : 0.0f, h1.y > 0.0f ? tf32_rna(v[j + 1]) : 0.0f,
                        h1.z > 0.0f ? tf32_rna(v[j + 2]) : 0.0f, h1.w > 0.0f ? tf32_rna(v[j + 3]) : 0.0f));
      }
    }
    sync_for_mma();
    // dX = dH1 W0 on the tensor cores; meanwhile dW0 += dH1^T X (and db0)
    if (tid == 0) mma_tile(tmem + 64u, dH1s, W0Ts, kMlpH, LF16, bar);
    for (int k0 = 0; k0 < 128; k0 += 8) {
      const int ka = k0 + tig, kb = ka + 4;
      const uint32_t A[4] = {lds_u(dH1s, ka, m1 + g, kMlpH), lds_u(dH1s, ka, m1 + g + 8, kMlpH),
                             lds_u(dH1s, kb, m1 + g, kMlpH), lds_u(dH1s, kb, m1 + g + 8, kMlpH)};
#pragma unroll
      for (int j = 0; j < J0; ++j)
        if (n0c + 8 * j < LFp)
          mma_tf32(acc0[j], A, lds_u(Xs, ka, n0c + 8 * j + g, LFp), lds_u(Xs, kb, n0c + 8 * j + g, LFp));
      if (bias) mma_tf32(accb0, A, one, one);
    }
    ok = wait_mma(bar, phase, a.status, a.spin_limit) && ok;
    // dX stored level-major for the encoding's adjoint (a separate tiled
    // kernel: k_table_grad)
    for (int c0 = 16 * quad; c0 < LF16; c0 += 16 * NG) {
      float v[16];
      tmem_ld16(tmem + lane_base + 64u + (uint32_t)c0, v);
      if (live) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          if (c0 + j < LF) {
            const int l = (c0 + j) / a.F, f = (c0 + j) - l * a.F;
            a.dX[((size_t)l * a.count + i) * a.F + f] = ok ? v[j] : 0.0f;
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();   // the tiles and accumulators are reused
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  // the CTA's gradient sums into the gradient vector (accumulator fragment
  // q of an m16n8 tile: row g + 8 (q >> 1), column 2 tig + (q & 1))
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int row = g + 8 * (q >> 1), col = 2 * tig + (q & 1);
#pragma unroll
    for (int j = 0; j < J1; ++j) atomicAdd(a.dW1 + (m1 + row) * kMlpH + n1 + 8 * j + col, acc1[j][q]);
#pragma unroll
    for (int j = 0; j < J2; ++j)
      if (do_w2 && m2 + row < a.C) atomicAdd(a.dW2 + (m2 + row) * kMlpH + n2 + 8 * j + col, acc2[j][q]);
#pragma unroll
    for (int j = 0; j < J0; ++j)
      if (n0c + 8 * j + col < LF) atomicAdd(a.dW0 + (m1 + row) * LF + n0c + 8 * j + col, acc0[j][q]);
    if (bias && tig == 0 && (q & 1) == 0) {   // every column of a bias tile holds the same sums
      atomicAdd(a.db1 + m1 + row, accb1[q]);
      atomicAdd(a.db0 + m1 + row, accb0[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < kDy; ++q) {
    float v = gb2[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int c = quad * (Cp / NG) + q;
    if (lane == 0 && q < Cp / NG && c < a.C) atomicAdd(a.db2 + c, v);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMlpTmemCols) : "memory");
}

}  // namespace vsn
