// FP64 instantiation of the WCNS-FE kernels.
#include "wcns_launch.cuh"
WCNS_INSTANTIATE(double)
