// F64 instantiation: the banded 2D stage (x and y sweeps of a stage in one persistent launch).
#include "wcns_launch.cuh"
WCNS_INSTANTIATE_BAND(double)
