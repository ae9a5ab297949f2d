// F32 instantiation: the banded 2D stage (x and y sweeps of a stage in one persistent launch).
#include "wcns_launch.cuh"
WCNS_INSTANTIATE_BAND(float)

namespace wcns {
static_assert(kBandCounters == kBandCounterWords, "counter words of the banded stage");
size_t band_ring_bytes_of(const GridInfo& g, size_t elem) { return band_ring_bytes(g, elem); }
}  // namespace wcns
