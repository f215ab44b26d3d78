// Shading kernels for batches whose shells all hold SH degree 1 FP16 texels (32-byte aligned: 256-bit loads).
#define VS_TC (vsd::TC_SH0 + 1)
#define VS_TC_OPS kTcSh1
#include "vs_tc_impl.cuh"
