// F64 instantiation: x sweeps of the 1D Euler (interface fluxes along rows, Eq. 3
// difference, RK stage).
#include "wcns_launch.cuh"
WCNS_INSTANTIATE_X(double, 3)
