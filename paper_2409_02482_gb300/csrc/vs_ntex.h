// Interface between the host API (vs_api.cu) and the neural-texture kernels
// (vs_ntex.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "vs.h"

namespace vsntex {
constexpr int kNtexChunk = 1 << 18;   // texels per chunk of activations

// Floats of workspace for chunks of `rows` texels.
size_t ws_floats(const vs_ntex_config& c, int rows);
// 0 on success, else a cudaError_t value.
int forward(const vs_ntex_config& c, const float* params, int W, int H, void* texels, int dtype, int pitch, int ch0,
            void* ws, cudaStream_t st);
int backward(const vs_ntex_config& c, const float* params, int W, int H, const float* grad_texels, int pitch, int ch0,
             float* grads, void* ws, cudaStream_t st);
int adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2, float eps, int step,
         cudaStream_t st);
}  // namespace vsntex
