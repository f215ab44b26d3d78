// Shading kernels for batches whose shells all hold baked SH degree 0 bytes.
#define VS_TC (vsd::TC_U80 + 0)
#define VS_TC_OPS kTcU80
#include "vs_tc_impl.cuh"
