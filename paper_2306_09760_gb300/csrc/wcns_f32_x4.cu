// F32 instantiation: x sweeps of the 2D Euler (interface fluxes along rows, Eq. 3
// difference, RK stage).
#include "wcns_launch.cuh"
WCNS_INSTANTIATE_X(float, 4)
