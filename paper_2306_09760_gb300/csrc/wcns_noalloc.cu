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
#include <mutex>

#include <cuda.h>

#include "../../include/wcns.h"
#include "wcns_grid_check.h"
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

// Device address of g_reduce_scratch.  The address belongs to the CUDA context that
// loaded the library's device code, so it is cached per context, keyed by the context's
// process-unique ID (cuCtxGetId): a device reset, or another context made current on
// the same device, gets its own lookup instead of a stale address.  The two driver
// queries are fetched through the runtime, so the library needs no link to libcuda.
// A mutex guards the cache: host threads may call this concurrently.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

struct ScratchCache {
  std::mutex mu;
  bool resolved = false;  // driver entry points looked up (successfully or not)
  CtxGetCurrentFn get_current = nullptr;
  CtxGetIdFn get_id = nullptr;
  static constexpr int kSlots = 64;
  unsigned long long ctx_id[kSlots] = {};
  void* addr[kSlots] = {};
  int used = 0, next = 0;  // filled slots; slot replaced next once all are filled
};
ScratchCache g_cache;

// ID of the current context, or 0 when none is current or the driver cannot say.
unsigned long long current_context_id(ScratchCache& c) {
  if (!c.resolved) {
    c.resolved = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      c.get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      c.get_id = reinterpret_cast<CtxGetIdFn>(f);
  }
  if (!c.get_current || !c.get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (c.get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (c.get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

cudaError_t scratch_address(void** out) {
  std::lock_guard<std::mutex> lock(g_cache.mu);
  unsigned long long id = current_context_id(g_cache);
  if (id != 0) {
    for (int k = 0; k < g_cache.used; ++k)
      if (g_cache.ctx_id[k] == id) {
        *out = g_cache.addr[k];
        return cudaSuccess;
      }
  }
  // first call in this context: resolve the address with the device current (this
  // also creates the device's primary context if the runtime has not made it yet)
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_reduce_scratch);
  if (e != cudaSuccess) return e;
  if (id == 0) id = current_context_id(g_cache);
  if (id != 0) {
    const int k = g_cache.used < ScratchCache::kSlots ? g_cache.used++ : g_cache.next;
    if (g_cache.used == ScratchCache::kSlots) g_cache.next = (k + 1) % ScratchCache::kSlots;
    g_cache.ctx_id[k] = id;
    g_cache.addr[k] = p;
  }
  *out = p;
  return cudaSuccess;
}

}  // namespace

extern "C" wcns_status wcns_reduce_noalloc(const wcns_grid* grid, const void* a, const void* b, int32_t what,
                                           void* stream, double* out) {
  if (!grid || !a || !out) return WCNS_ERR_ARG;
  const wcns_grid& g = *grid;
  // the layout rules of wcns_init (ndim = 1 with ny > 1: independent lines, reduced
  // like any grid); lo, hi and bc are not read
  if (wcns::check_grid_layout(g) != WCNS_OK) return WCNS_ERR_ARG;
  // one ticket counter and one row of partials per variable: more variables than the
  // array holds are rejected
  if (g.nvar > kNoAllocVars) return WCNS_ERR_ARG;
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
