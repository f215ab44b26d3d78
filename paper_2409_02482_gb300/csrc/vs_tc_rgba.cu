// Shading kernels for batches whose shells all hold RGBA FP32 texels, 16-byte loads and reductions.
#define VS_TC (vsd::TC_RGBA)
#define VS_TC_OPS kTcRgba
#include "vs_tc_impl.cuh"
