// Shading and persistent kernels of one texel class, instantiated in the
// translation unit that includes this file with VS_TC (the class) and
// VS_TC_OPS (the name of its launcher table) defined.

#include "vs_kernels.cuh"

#if !defined(VS_TC) || !defined(VS_TC_OPS)
#error "define VS_TC and VS_TC_OPS before including vs_tc_impl.cuh"
#endif

namespace {

// Only the generic class carries the full variants (near-plane clipping,
// per-layer buffers).
constexpr bool kHasFull = (VS_TC) == vsd::TC_ANY;

template <bool BWD, bool FULL>
cudaError_t launch_persistent(const TableRef& tb, int grid, long long spin_limit, size_t smem, cudaStream_t st) {
  vsd::k_persistent<BWD, VS_TC, FULL><<<grid, vsd::pers_threads(BWD), smem, st>>>(tb, spin_limit);
  return cudaGetLastError();
}

cudaError_t tc_persistent(const TableRef& tb, bool bwd, bool full, int grid, long long spin_limit, size_t smem,
                          cudaStream_t st) {
  if (full) {
    if constexpr (kHasFull) {
      return bwd ? launch_persistent<true, true>(tb, grid, spin_limit, smem, st)
                 : launch_persistent<false, true>(tb, grid, spin_limit, smem, st);
    }
    return cudaErrorInvalidValue;
  }
  return bwd ? launch_persistent<true, false>(tb, grid, spin_limit, smem, st)
             : launch_persistent<false, false>(tb, grid, spin_limit, smem, st);
}

// Plain shading launch: forward from the visibility words, or the
// standalone adjoint from the caller's hit buffer.
template <bool BWD, bool FULL>
cudaError_t launch_shade(const TableRef& tb, int blocks, size_t smem, cudaStream_t st) {
  vsd::k_shade<BWD, BWD, VS_TC, FULL><<<blocks, vsd::kThreads, smem, st>>>(tb, 0);
  return cudaGetLastError();
}

cudaError_t tc_shade(const TableRef& tb, bool bwd, bool full, int blocks, size_t smem, cudaStream_t st) {
  if (full) {
    if constexpr (kHasFull) {
      return bwd ? launch_shade<true, true>(tb, blocks, smem, st) : launch_shade<false, true>(tb, blocks, smem, st);
    }
    return cudaErrorInvalidValue;
  }
  return bwd ? launch_shade<true, false>(tb, blocks, smem, st) : launch_shade<false, false>(tb, blocks, smem, st);
}

template <bool BWD, bool FULL>
cudaError_t occupancy_of(size_t smem, int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, vsd::k_persistent<BWD, VS_TC, FULL>,
                                                       vsd::pers_threads(BWD), smem);
}

cudaError_t tc_occupancy(bool bwd, bool full, size_t smem, int* blocks_per_sm) {
  if (full) {
    if constexpr (kHasFull) return bwd ? occupancy_of<true, true>(smem, blocks_per_sm) : occupancy_of<false, true>(smem, blocks_per_sm);
    *blocks_per_sm = 0;
    return cudaSuccess;
  }
  return bwd ? occupancy_of<true, false>(smem, blocks_per_sm) : occupancy_of<false, false>(smem, blocks_per_sm);
}

template <bool FULL>
cudaError_t configure_one(int most_f, int most_b) {
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(vsd::k_shade<false, false, VS_TC, FULL>, A, most_f)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(vsd::k_shade<true, true, VS_TC, FULL>, A, most_b)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(vsd::k_persistent<false, VS_TC, FULL>, A, most_f)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(vsd::k_persistent<true, VS_TC, FULL>, A, most_b);
}

cudaError_t tc_configure(int most_f, int most_b) {
  cudaError_t e = configure_one<false>(most_f, most_b);
  if constexpr (kHasFull) {
    if (e == cudaSuccess) e = configure_one<true>(most_f, most_b);
  }
  return e;
}

}  // namespace

namespace vsk {
extern const TcOps VS_TC_OPS = {tc_persistent, tc_shade, tc_occupancy, tc_configure};
}  // namespace vsk
