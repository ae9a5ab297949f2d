// F32 instantiation: CFL step, reductions, weight statistics and the kernel configuration.
#include "wcns_launch.cuh"
WCNS_INSTANTIATE_MISC(float)
