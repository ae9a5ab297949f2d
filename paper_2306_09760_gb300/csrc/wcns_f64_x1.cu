// F64 instantiation: x sweeps of the one-variable systems (scalar advection) (interface fluxes along rows, Eq. 3
// difference, RK stage).
#include "wcns_launch.cuh"
WCNS_INSTANTIATE_X(double, 1)
