// Shading and persistent kernels of one texel class, instantiated in the
// translation unit that includes this file with VS_TC (the class) and
// VS_TC_OPS (the name of its launcher table) defined.

#include "vs_kernels.cuh"

#if !defined(VS_TC) || !defined(VS_TC_OPS)
#error "define VS_TC and VS_TC_OPS before including vs_tc_impl.cuh"
#endif

namespace {

cudaError_t tc_persistent(const TableRef& tb, bool bwd, int grid, long long spin_limit, size_t smem,
                          cudaStream_t st) {
  if (bwd) vsd::k_persistent<true, VS_TC><<<grid, vsd::kThreads, smem, st>>>(tb, spin_limit);
  else vsd::k_persistent<false, VS_TC><<<grid, vsd::kThreads, smem, st>>>(tb, spin_limit);
  return cudaGetLastError();
}

// Plain shading launch: forward from the visibility words, or the
// standalone adjoint from the caller's hit buffer.
cudaError_t tc_shade(const TableRef& tb, bool bwd, int blocks, size_t smem, cudaStream_t st) {
  if (bwd) vsd::k_shade<true, true, VS_TC><<<blocks, vsd::kThreads, smem, st>>>(tb, 0);
  else vsd::k_shade<false, false, VS_TC><<<blocks, vsd::kThreads, smem, st>>>(tb, 0);
  return cudaGetLastError();
}

cudaError_t tc_occupancy(bool bwd, size_t smem, int* blocks_per_sm) {
  if (bwd)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, vsd::k_persistent<true, VS_TC>, vsd::kThreads,
                                                         smem);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, vsd::k_persistent<false, VS_TC>, vsd::kThreads,
                                                       smem);
}

cudaError_t tc_configure(int most_f, int most_b) {
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(vsd::k_shade<false, false, VS_TC>, A, most_f)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(vsd::k_shade<true, true, VS_TC>, A, most_b)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(vsd::k_persistent<false, VS_TC>, A, most_f)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(vsd::k_persistent<true, VS_TC>, A, most_b);
}

}  // namespace

namespace vsk {
extern const TcOps VS_TC_OPS = {tc_persistent, tc_shade, tc_occupancy, tc_configure};
}  // namespace vsk
