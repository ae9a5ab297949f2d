// F64 instantiation: adjoint sweeps of one RK step.
#include "wcns_launch.cuh"
WCNS_INSTANTIATE_ADJ(double)
