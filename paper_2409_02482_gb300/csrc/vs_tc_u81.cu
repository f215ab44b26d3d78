// Shading kernels for batches whose shells all hold baked SH degree 1 bytes.
#define VS_TC (vsd::TC_U80 + 1)
#define VS_TC_OPS kTcU81
#include "vs_tc_impl.cuh"
