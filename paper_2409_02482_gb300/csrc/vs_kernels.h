// Interface between the host API (vs_api.cu) and the kernels (vs_kernels.cu).
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
  int* done;                // [n * 4] completed units per (item, phase)
  const int* unit_pre;      // [4][n + 1] unit prefix per phase
  int n;
  int total;                // all units
  int phase_start[4];       // first global unit of each phase
};

// A slice of the host-built table carried to the device in kernel
// parameters (so the copy is captured by value in a CUDA graph).
constexpr int kUploadBytes = 24576;
struct UploadChunk {
  uint32_t dst_off;
  uint32_t nbytes;          // multiple of 16
  int32_t reset;            // reset next_unit / abort in the header
  int32_t pad;
  uint4 data[kUploadBytes / 16];
};

namespace vsk {
cudaError_t upload(char* ws, const UploadChunk& c, cudaStream_t st);
cudaError_t plain_forward(const TableRef& tb, const int units[4], cudaStream_t st);
cudaError_t plain_backward(const TableRef& tb, const int units[4], cudaStream_t st);
cudaError_t persistent(const TableRef& tb, int grid, long long spin_limit, cudaStream_t st);
cudaError_t persistent_occupancy(int* blocks_per_sm);
}  // namespace vsk
