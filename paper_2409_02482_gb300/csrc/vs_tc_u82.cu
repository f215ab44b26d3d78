// Shading kernels for batches whose shells all hold baked SH degree 2 bytes.
#define VS_TC (vsd::TC_U80 + 2)
#define VS_TC_OPS kTcU82
#include "vs_tc_impl.cuh"
