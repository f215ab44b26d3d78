// Kernels without a texel class (table upload, vertex setup, raster) and the
// host-side launchers, which dispatch the shading kernels to the
// translation unit of the batch's texel class.

#include "vs_kernels.cuh"

namespace vsd {

__global__ void __launch_bounds__(kThreads) k_upload(char* ws, const __grid_constant__ UploadChunk c) {
  uint4* dst = reinterpret_cast<uint4*>(ws + c.dst_off);
  for (uint32_t i = threadIdx.x; i < c.nbytes / 16; i += blockDim.x) dst[i] = c.data[i];
  if (c.reset && threadIdx.x == 0) {
    WsHeader* h = reinterpret_cast<WsHeader*>(ws);
    h->next_unit = 0;
    h->abort = 0;
    h->launches += (unsigned long long)c.launches;
    h->kernel_class = c.kernel_class;
  }
}

// Plain per-phase kernels.  Setup: each warp runs one unit (8 per block).
// Raster and shade: block b runs unit b, its warp w runs round w of it --
// the same arithmetic as the persistent kernel, spread over more warps.
__global__ void __launch_bounds__(kThreads) k_setup(TableRef tb, int item) {
  const DItem& it = tb.items[item];
  const int u = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (u < it.units[PH_SETUP]) unit_setup(it, tb.shells + it.shell0, u);
}

template <bool FULL>
__global__ void __launch_bounds__(kThreads) k_raster(TableRef tb, int item) {
  const DItem& it = tb.items[item];
  const int w = threadIdx.x >> 5;
  unit_raster<FULL>(it, tb.shells + it.shell0, blockIdx.x, tb.hdr, vs_smem + w * kRasterWarpBytes, w, w + 1);
}

}  // namespace vsd

// ----------------------------------------------------------------------------
// host-side launchers (C++ linkage, used by vs_api.cu)
// ----------------------------------------------------------------------------
namespace vsk {

const TcOps& tc_ops(int tc) {
  switch (tc) {
    case vsd::TC_RGBA: return kTcRgba;
    case vsd::TC_SH0: return kTcSh0;
    case vsd::TC_SH0 + 1: return kTcSh1;
    case vsd::TC_SH0 + 2: return kTcSh2;
    case vsd::TC_SH0 + 3: return kTcSh3;
    case vsd::TC_U80: return kTcU80;
    case vsd::TC_U80 + 1: return kTcU81;
    case vsd::TC_U80 + 2: return kTcU82;
    case vsd::TC_U80 + 3: return kTcU83;
    default: return kTcAny;
  }
}

cudaError_t upload(char* ws, const UploadChunk& c, cudaStream_t st) {
  vsd::k_upload<<<1, vsd::kThreads, 0, st>>>(ws, c);
  return cudaGetLastError();
}

int plain_forward_launches(const int units[4]) { return (units[0] > 0) + (units[1] > 0) + (units[2] > 0); }
int plain_backward_launches(const int units[4]) { return (units[0] > 0) + (units[2] > 0); }

cudaError_t plain_forward(const TableRef& tb, const int units[4], int tc, bool full, cudaStream_t st) {
  const int W = vsd::kWarps;
  if (units[0]) vsd::k_setup<<<(units[0] + W - 1) / W, vsd::kThreads, 0, st>>>(tb, 0);
  if (units[1]) {
    if (full) vsd::k_raster<true><<<units[1], vsd::kThreads, vsd::kRasterWarpBytes * W, st>>>(tb, 0);
    else vsd::k_raster<false><<<units[1], vsd::kThreads, vsd::kRasterWarpBytes * W, st>>>(tb, 0);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !units[2]) return e;
  return tc_ops(tc).shade(tb, false, full, units[2], vsd::block_smem_bytes(tb.kmax, false, tc), st);
}

cudaError_t plain_backward(const TableRef& tb, const int units[4], int tc, bool full, cudaStream_t st) {
  const int W = vsd::kWarps;
  if (units[0]) vsd::k_setup<<<(units[0] + W - 1) / W, vsd::kThreads, 0, st>>>(tb, 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !units[2]) return e;
  return tc_ops(tc).shade(tb, true, full, units[2], vsd::block_smem_bytes(tb.kmax, true, tc), st);
}

cudaError_t persistent(const TableRef& tb, bool bwd, int tc, bool full, int grid, long long spin_limit,
                       cudaStream_t st) {
  return tc_ops(tc).persistent(tb, bwd, full, grid, spin_limit, vsd::pers_smem_bytes(tb.kmax, bwd, tc), st);
}

cudaError_t persistent_occupancy(bool bwd, int tc, bool full, int kmax, int* blocks_per_sm) {
  return tc_ops(tc).occupancy(bwd, full, vsd::pers_smem_bytes(kmax, bwd, tc), blocks_per_sm);
}

cudaError_t configure_kernels() {
  for (int tc = 0; tc < vsd::kNumTc; ++tc) {
    const int most_f = (int)std::max(vsd::block_smem_bytes(vsd::kMaxShells, false, tc),
                                     vsd::pers_smem_bytes(vsd::kMaxShells, false, tc));
    const int most_b = (int)std::max(vsd::block_smem_bytes(vsd::kMaxShells, true, tc),
                                     vsd::pers_smem_bytes(vsd::kMaxShells, true, tc));
    cudaError_t e = tc_ops(tc).configure(most_f, most_b);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace vsk
