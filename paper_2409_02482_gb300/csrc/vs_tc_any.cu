// Shading kernels for batches whose shells all hold any mix of formats (decided per shell).
#define VS_TC (vsd::TC_ANY)
#define VS_TC_OPS kTcAny
#include "vs_tc_impl.cuh"
