// F64 instantiation: the banded 2D stage (x and y sweeps of a stage in one persistent launch).
#include "wcns_launch.cuh"
WCNS_INSTANTIATE_BAND(double)

namespace wcns {
// Self-test of the two bounded waits: one thread waits on a counter that nothing
// increments (band_wait) and on an mbarrier armed for 16 bytes that no copy delivers
// (mbar_wait).  Both must give up; gave_up[0..1] receive 1 when they did, and each sets
// bit 1 of *err as the kernels do.
__global__ void bounded_wait_selftest_kernel(const unsigned* never, int* err, int* gave_up) {
  __shared__ unsigned long long bar;
  if (threadIdx.x != 0) return;
  const bool a = band_wait(never, 1u);
  if (!a) atomicOr(err, 2);
  mbar_init(&bar, 1);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" : : "r"(smem_u32(&bar)), "r"(16u) : "memory");
  const bool b = mbar_wait(&bar, 0);
  if (!b) atomicOr(err, 2);
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" : : "r"(smem_u32(&bar)) : "memory");
  gave_up[0] = a ? 0 : 1;
  gave_up[1] = b ? 0 : 1;
}

cudaError_t launch_wait_selftest(const unsigned* never, int* err, int* gave_up, cudaStream_t st) {
  bounded_wait_selftest_kernel<<<1, 32, 0, st>>>(never, err, gave_up);
  return cudaGetLastError();
}
}  // namespace wcns
