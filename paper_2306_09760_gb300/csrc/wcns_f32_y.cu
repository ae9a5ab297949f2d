// F32 instantiation: y sweeps (interface fluxes along columns, stage completion).
#include "wcns_launch.cuh"
WCNS_INSTANTIATE_Y(float)
