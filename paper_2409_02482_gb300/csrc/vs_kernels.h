// Interface between the host API (vs_api.cu) and the kernels (vs_kernels.cu,
// vs_tc_*.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vsd {
struct DItem;
struct DShell;
struct WsHeader;
}  // namespace vsd

// Device view of the item table uploaded into the workspace.
struct TableRef {
  vsd::WsHeader* hdr;
  vsd::DItem* items;        // [n]
  vsd::DShell* shells;      // [sum of k]
  int* done;                // [n * 3] completed units per (item, phase)
  const int* stage_pre;     // [n + 3] first global unit of each stage (+ total)
  int n;
  int total;                // all units
  int kmax;                 // most shells of any item (sizes shared memory)
};

// A slice of the host-built table carried to the device in kernel
// parameters (so the copy is captured by value in a CUDA graph).
constexpr int kUploadBytes = 24576;
struct UploadChunk {
  uint32_t dst_off;
  uint32_t nbytes;          // multiple of 16
  int32_t reset;            // first chunk: reset next_unit / abort, count launches
  int32_t launches;         // kernels this call enqueues (added to the header)
  int32_t kernel_class;     // first chunk: the call's shading kernels (vs_stats::kernel_class)
  int32_t pad[3];
  uint4 data[kUploadBytes / 16];
};

namespace vsk {
// Launchers of the kernels compiled for one texel class (vsd::TC_*), one
// table per translation unit vs_tc_*.cu.
struct TcOps {
  cudaError_t (*persistent)(const TableRef& tb, bool bwd, bool full, int grid, long long spin_limit, size_t smem,
                            cudaStream_t st);
  cudaError_t (*shade)(const TableRef& tb, bool bwd, bool full, int blocks, size_t smem, cudaStream_t st);
  cudaError_t (*occupancy)(bool bwd, bool full, size_t smem, int* blocks_per_sm);
  cudaError_t (*configure)(int most_smem_fwd, int most_smem_bwd);
};
// full = the variant with the rare features -- near-plane clipping and the
// per-layer buffers -- compiled for the generic class only; the host asks for
// it when a shell may reach nearer than znear or layers are requested
extern const TcOps kTcAny, kTcRgba, kTcSh0, kTcSh1, kTcSh2, kTcSh3, kTcU80, kTcU81, kTcU82, kTcU83;

cudaError_t upload(char* ws, const UploadChunk& c, cudaStream_t st);
int plain_forward_launches(const int units[4]);
int plain_backward_launches(const int units[4]);
cudaError_t plain_forward(const TableRef& tb, const int units[4], int tc, bool full, cudaStream_t st);
cudaError_t plain_backward(const TableRef& tb, const int units[4], int tc, bool full, cudaStream_t st);
cudaError_t persistent(const TableRef& tb, bool bwd, int tc, bool full, int grid, long long spin_limit,
                       cudaStream_t st);
cudaError_t persistent_occupancy(bool bwd, int tc, bool full, int kmax, int* blocks_per_sm);
cudaError_t configure_kernels();
}  // namespace vsk
