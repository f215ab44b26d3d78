// Shading kernels for batches whose shells all hold SH degree 0 FP16 texels (16-byte aligned: 128-bit loads).
#define VS_TC (vsd::TC_SH0)
#define VS_TC_OPS kTcSh0
#include "vs_tc_impl.cuh"
