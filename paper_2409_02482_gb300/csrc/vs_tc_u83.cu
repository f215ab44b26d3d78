// Shading kernels for batches whose shells all hold baked SH degree 3 bytes.
#define VS_TC (vsd::TC_U80 + 3)
#define VS_TC_OPS kTcU83
#include "vs_tc_impl.cuh"
