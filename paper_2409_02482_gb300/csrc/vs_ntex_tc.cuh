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

// Issues the MMAs of D[128 x Np] = A[128 x Kp] B[Np x Kp]^T (one thread) and
// commits them to the mbarrier.
__device__ __forceinline__ void mma_tile(uint32_t d_tmem, const float* A, const float* B, int Kp, int Np,
                                         uint64_t* bar) {
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

// Dynamic shared memory of k_mlp_fwd_tc for LF inputs and C outputs.
__host__ __device__ constexpr int mlp_fwd_smem(int LF, int C) {
  return op_bytes(kMlpH, LF) + op_bytes(kMlpH, kMlpH) + op_bytes((C + 15) & ~15, kMlpH) + op_bytes(128, LF) +
         2 * op_bytes(128, kMlpH) + 256;
}

__global__ void __launch_bounds__(kTcThreads, 1) k_mlp_fwd_tc(const MlpFwdArgs a, const Enc e) {
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
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  uint32_t phase = 0;
  bool ok = true;
  const int tiles = (a.N + 127) / 128;
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    // encoding of texel n = 128 tile + tid into row tid of X
    const int n = tile * 128 + tid;
    if (n < a.N) {
      const int tx = n % a.W, ty = n / a.W;
      for (int l = 0; l < e.L; ++l) {
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const size_t lt = (size_t)l << e.logT;
        for (int c = 0; c < 4; ++c) {
          uint32_t row;
          float w;
          corner(e, l, tx, ty, a.W, a.H, c, row, w);
          const float* t = a.table + (lt + row) * e.F;
          for (int f = 0; f < e.F; ++f) acc[f] = fmaf(w, __ldg(t + f), acc[f]);
        }
        for (int f = 0; f < e.F; ++f) *op_at(Xs, tid, l * e.F + f, LFp) = tf32_rna(acc[f]);
      }
      for (int k = a.LF; k < LFp; ++k) *op_at(Xs, tid, k, LFp) = 0.0f;
    } else {
      for (int k = 0; k < LFp; ++k) *op_at(Xs, tid, k, LFp) = 0.0f;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // layer 0
    if (tid == 0) mma_tile(tmem, Xs, W0s, LFp, kMlpH, bar);
    ok = wait_mma(bar, phase, a.status, a.spin_limit) && ok;
    for (int c0 = 0; c0 < kMlpH; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + lane_base + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) *op_at(H1s, tid, c0 + j, kMlpH) = tf32_rna(fmaxf(v[j] + __ldg(a.b0 + c0 + j), 0.0f));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // layer 1
    if (tid == 0) mma_tile(tmem + 64u, H1s, W1s, kMlpH, kMlpH, bar);
    ok = wait_mma(bar, phase, a.status, a.spin_limit) && ok;
    for (int c0 = 0; c0 < kMlpH; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + lane_base + 64u + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) *op_at(H2s, tid, c0 + j, kMlpH) = tf32_rna(fmaxf(v[j] + __ldg(a.b1 + c0 + j), 0.0f));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // output layer -> texels
    if (tid == 0) mma_tile(tmem + 128u, H2s, W2s, kMlpH, Cp, bar);
    ok = wait_mma(bar, phase, a.status, a.spin_limit) && ok;
    for (int c0 = 0; c0 < Cp; c0 += 16) {
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
