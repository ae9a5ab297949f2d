// FP32 instantiation of the WCNS-FE kernels (bulk arithmetic in single precision;
// the reductions accumulate in FP64).
#include "wcns_launch.cuh"
WCNS_INSTANTIATE(float)
