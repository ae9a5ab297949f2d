// wcns_reduce_noalloc: the FP64 norm reduction of wcns_reduce for callers that cannot
// allocate device memory.
//
// Some callers must not call cudaMalloc at the point where they need a sum or a norm:
// a host loop that reserved all of its device memory up front and must not stall
// (cudaMalloc can synchronise the device), or code embedded in a framework whose own
// allocator owns the device memory.  Such callers also cannot create a wcns_ctx,
// because wcns_init allocates the context's scratch.  This entry point needs neither:
// the per-block partial results and the completion tickets live in one file-scope
// device array of fixed size that every GPU loading the library holds until exit.
//
// The array is shared by every call and keeps the last call's contents.  The tickets
// must start at zero, so each call clears them on its stream before its kernel; the
// partials are always written before they are read.  Two calls that overlap on the
// GPU (different streams, no ordering between them) race on the array.
#include <cstdint>
#include <cstring>

#include "../../include/wcns.h"
#include "wcns_kernels.cuh"

namespace {

// Scratch layout: kNoAllocVars ticket counters, then kNoAllocVars x kNoAllocBlocks
// FP64 partials.  64 KiB in total.
constexpr int kNoAllocVars = 4;
constexpr int kNoAllocBlocks = 2040;
constexpr size_t kTicketBytes = 256;
constexpr size_t kScratchBytes = kTicketBytes + sizeof(double) * kNoAllocVars * kNoAllocBlocks;
static_assert(kScratchBytes <= 64 * 1024, "the static scratch stays at 64 KiB");

static __device__ __align__(256) unsigned char g_reduce_scratch[kScratchBytes];

// Device address of g_reduce_scratch, resolved once per device.
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};

cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_reduce_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" wcns_status wcns_reduce_noalloc(const wcns_grid* grid, const void* a, const void* b, int32_t what,
                                           void* stream, double* out) {
  if (!grid || !a || !out) return WCNS_ERR_ARG;
  const wcns_grid& g = *grid;
  if (g.dtype != WCNS_F64 && g.dtype != WCNS_F32) return WCNS_ERR_ARG;
  if (g.ndim != 1 && g.ndim != 2) return WCNS_ERR_ARG;
  if (g.nx < 1 || g.ny < 1 || g.pitch < g.nx || g.pitch % 32 != 0) return WCNS_ERR_ARG;
  if (g.ndim == 1 && g.ny != 1) return WCNS_ERR_ARG;
  // one ticket counter and one row of partials per variable: more variables than the
  // array holds are rejected
  if (g.nvar < 1 || g.nvar > kNoAllocVars) return WCNS_ERR_ARG;
  if (what != WCNS_REDUCE_SUM && what != WCNS_REDUCE_L1 && what != WCNS_REDUCE_LINF) return WCNS_ERR_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(a) & 15u) || (b && (reinterpret_cast<uintptr_t>(b) & 15u)) ||
      (reinterpret_cast<uintptr_t>(out) & 7u))
    return WCNS_ERR_ARG;
  void* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return WCNS_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  e = cudaMemsetAsync(scratch, 0, kTicketBytes, st);  // tickets start at zero
  if (e != cudaSuccess) return WCNS_ERR_CUDA;
  wcns::ReduceArgs A{};
  A.a = a;
  A.b = b;
  A.nx = g.nx;
  A.ny = g.ny;
  A.pitch = g.pitch;
  A.fstride = g.ny * g.pitch;
  A.what = what;
  A.counters = static_cast<unsigned int*>(scratch);
  A.partials = reinterpret_cast<double*>(static_cast<unsigned char*>(scratch) + kTicketBytes);
  A.out = out;
  const int64_t ncell = g.nx * g.ny;
  int64_t want = (ncell + wcns::kRedThreads * 4 - 1) / (wcns::kRedThreads * 4);
  const int blocks = (int)(want < 1 ? 1 : (want > kNoAllocBlocks ? kNoAllocBlocks : want));
  dim3 grd(blocks, g.nvar);
  if (g.dtype == WCNS_F64) wcns::reduce_kernel<double><<<grd, wcns::kRedThreads, 0, st>>>(A);
  else wcns::reduce_kernel<float><<<grd, wcns::kRedThreads, 0, st>>>(A);
  return cudaGetLastError() == cudaSuccess ? WCNS_OK : WCNS_ERR_CUDA;
}
