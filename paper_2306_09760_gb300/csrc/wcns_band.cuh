// Banded RK stage of a 2D grid in one persistent launch.
//
// A 2D stage is an x sweep, which writes the partial stage R = a u^n + b (u + dt L_x),
// and a y sweep, which completes it with b dt L_y.  Run as two launches over the whole
// grid, R is a full state-sized array: at 2048^2 it is written to and read back from
// DRAM, and the y sweep reads the state u a second time after the x sweep's pass over
// the grid has pushed it out of L2.
//
// Here the rows are grouped into bands of whole y tiles, and the x tiles of a band and
// then its y tiles form one work list.  A cooperative launch keeps every block resident;
// block k takes items k, k + G, k + 2G, ... (G blocks) in list order.  The y tiles of
// band b are listed after the x tiles of band b + kBandLead, so the x tiles they need
// have normally finished when a block reaches them; the block still waits (bounded) on
// the band's completion counter.  R lives in a ring of kBandRing band-sized slots: band
// b writes slot b mod kBandRing, and the x tiles of band b wait until the y tiles of band
// b - kBandRing have consumed that slot.  The ring (a few tens of MB) stays in L2, and the
// y tiles find the rows of u that the x tiles of the same band read shortly before, so
// the stage's DRAM traffic is about reading u (and u^n) once and writing the new stage
// once.
//
// Progress: an item waits only on items listed before it (the x tiles of its band, or
// the y tiles of the band kBandRing back, listed before the x tiles of band
// b - kBandRing + kBandLead + 1 <= b).  Each block publishes an item's completion before
// it waits for anything its next item needs, and every block is resident, so the
// earliest unfinished item never waits and the launch always completes.  Each wait still
// gives up after kBandSpin polls, sets bit 1 of the sticky error word (WCNS_ERR_TIMEOUT
// at the next status query) and skips its item.
//
// Measured on GB300 (2048^2 FP32): the stage moves 116 MB (first stage) and 199 MB
// (later stages) of DRAM traffic against 259 and 340 MB for the two launches, but takes
// 0.32 ms against 0.24 ms: the sweeps are bound by instruction issue, and the block-wide
// synchronisation at every tile boundary of the persistent loop costs more than the
// traffic saves.  It is therefore an option (wcns_set_stage_form), not the default.
#pragma once

#include <algorithm>

#include "wcns_kernels.cuh"

namespace wcns {

constexpr int kBandMax = 64;                // bands per grid at most
constexpr int kBandLead = 2;                // y tiles of band b follow the x tiles of band b + kBandLead
constexpr int kBandRing = kBandLead + 2;    // partial-stage slots (at least kBandLead + 1)
constexpr int kBandSpin = 1 << 22;          // polls (about 0.1 us each) before a wait gives up
constexpr int kBandCounters = 2 + 2 * kBandMax;  // word 0 unused, blocks done, x and y items done per band

// The work list of one banded stage (host-built, passed by value).
struct BandPlan {
  int nband, nseg;
  int seg_start[2 * kBandMax + 1];          // first item of segment j; seg_start[nseg] = items
  unsigned char seg_kind[2 * kBandMax];     // 0: x tiles of a band, 1: y tiles of a band
  unsigned char seg_band[2 * kBandMax];
  int row0[kBandMax + 1];                   // first row of band b; row0[nband] = ny
  unsigned x_items[kBandMax], y_items[kBandMax];
  int xfull, xtiles;                        // full x tiles per row, x tiles per row
  int ycols, ytiles_per_band;               // y column blocks, y tile rows per band
  int64_t slot_elems, slot_vstride;         // elements per ring slot, per variable of a slot
};

// Decodes work item `item`: kind 0 (x tile of row p0, tile p1 of the row) or kind 1 (y
// tile of column block p0, row block p1), and its band b.  Full x tiles of a band come
// first, the ragged last tile of each of its rows after them.
WCNS_HD void band_decode(const BandPlan& L, int item, int& kind, int& b, int64_t& p0, int64_t& p1) {
  int lo = 0, hi = L.nseg - 1;  // the segment holding the item
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.seg_start[mid] <= item) lo = mid;
    else hi = mid - 1;
  }
  kind = L.seg_kind[lo];
  b = L.seg_band[lo];
  const int l = item - L.seg_start[lo];
  if (kind == 0) {
    const int nf = (L.row0[b + 1] - L.row0[b]) * L.xfull;
    if (l < nf) {
      p0 = L.row0[b] + l / L.xfull;
      p1 = l % L.xfull;
    } else {
      p0 = L.row0[b] + (l - nf);
      p1 = L.xfull;
    }
  } else {
    p0 = l % L.ycols;
    p1 = (int64_t)b * L.ytiles_per_band + l / L.ycols;
  }
}

template <typename T>
struct BandArgs {
  SweepArgs<T> X;  // the stage's x sweep (writes the ring, not X.out)
  SweepArgs<T> Y;  // the stage's y sweep (reads the ring, not Y.R)
  BandPlan plan;
  T* ring;
  unsigned* ctr;   // kBandCounters, zero at launch; the last block to leave zeroes them again
  int* err;
};

// Polls *p (acquire, device scope) until it reaches target; false after kBandSpin polls.
__device__ __forceinline__ bool band_wait(const unsigned* p, unsigned target) {
  for (int it = 0; it < kBandSpin; ++it) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    if (v >= target) return true;
    __nanosleep(64);
  }
  return false;
}

// Adds 1 to *p with release semantics at device scope: the item's stores (made by the
// whole block, ordered before this by the preceding barrier) become visible to a block
// that reads the count with acquire semantics.
__device__ __forceinline__ void band_done(unsigned* p) {
  asm volatile("red.release.gpu.global.add.u32 [%0], 1;" : : "l"(p) : "memory");
}

// Thread 0 prepares item `item` for the block: decodes it into s_job and waits (bounded)
// for what it depends on.  s_job = {kind, band, p0, p1, ok}; kind < 0 ends the loop.
template <typename T>
__device__ __forceinline__ void band_prepare(const BandArgs<T>& B, int item, int (&s_job)[5]) {
  const BandPlan& L = B.plan;
  if (item >= L.seg_start[L.nseg]) {
    s_job[0] = -1;
    return;
  }
  int kind, b;
  int64_t p0, p1;
  band_decode(L, item, kind, b, p0, p1);
  bool ok = true;
  if (kind == 0) {
    if (b >= kBandRing) ok = band_wait(&B.ctr[2 + kBandMax + b - kBandRing], L.y_items[b - kBandRing]);
  } else {
    ok = band_wait(&B.ctr[2 + b], L.x_items[b]);
  }
  if (!ok) atomicOr(B.err, 2);
  s_job[0] = kind;
  s_job[1] = b;
  s_job[2] = (int)p0;
  s_job[3] = (int)p1;
  s_job[4] = ok ? 1 : 0;
}

// The loop of one block: items blockIdx.x, blockIdx.x + gridDim.x, ... of the work list,
// in list order.  The launch is cooperative (every block resident at once), so the
// block that holds an item an earlier item waits on is running, and the earliest
// unfinished item never waits (each block publishes an item's completion before it
// waits for anything its next item needs).  Thread 0 publishes, decodes the next item
// and waits for what it depends on while the block is at a barrier.
template <typename T, int FIX, int P>
__global__ void __launch_bounds__(kXThreads, sweep_min_blocks<T>()) stage_band_kernel(const __grid_constant__ BandArgs<T> B) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int s_job[5];
  const BandPlan& L = B.plan;
  if (B.X.dt && B.X.dt->zero) return;  // the run has reached t_end: every block leaves untouched
  const bool lead = threadIdx.x == 0;
  int item = blockIdx.x;
  if (lead) band_prepare<T>(B, item, s_job);
  __syncthreads();
  for (;;) {
    const int kind = s_job[0];
    if (kind < 0) break;
    const int b = s_job[1];
    T* slot = B.ring + (int64_t)(b % kBandRing) * L.slot_elems;
    if (s_job[4]) {
      if (kind == 0)
        sweep_x_body<T, 4, kStage, FIX, P>(B.X, s_job[2], s_job[3], slot, L.slot_vstride, L.row0[b], smem_raw);
      else
        sweep_y_body<T, 4, kStage, FIX>(B.Y, s_job[2], s_job[3], slot, L.slot_vstride, L.row0[b],
                                        (unsigned)(s_job[2] + s_job[3] * L.ycols), smem_raw);
    }
    __syncthreads();  // every store of the item precedes its count; s_job may be rewritten
    if (lead) {
      // published before the next item's wait: that item may depend on this one
      band_done(&B.ctr[2 + kind * kBandMax + b]);
      item += gridDim.x;
      band_prepare<T>(B, item, s_job);
    }
    __syncthreads();
  }
  // the last block to leave zeroes the counters for the next launch
  if (lead) {
    __threadfence();
    if (atomicAdd(&B.ctr[1], 1u) == gridDim.x - 1) {
      for (int k = 0; k < kBandCounters; ++k) B.ctr[k] = 0u;
      __threadfence();
    }
  }
}

template <typename T, int P>
constexpr size_t stage_band_smem() {
  return sweep_x_smem<T, 4, P>() > sweep_y_smem<T, 4>() ? sweep_x_smem<T, 4, P>() : sweep_y_smem<T, 4>();
}

// Rows per band: whole y tiles, at least two, so that at most kBandMax bands cover ny.
inline int64_t band_rows(int64_t ny) {
  const int64_t nty = (ny + kYTile - 1) / kYTile;
  int64_t k = (nty + kBandMax - 1) / kBandMax;
  if (k < 2) k = 2;
  return k * kYTile;
}

// The work list for a 2D grid whose x tiles hold `xtile` cells.
inline BandPlan make_band_plan(const GridInfo& g, int xtile) {
  BandPlan L{};
  const int64_t rows = band_rows(g.ny);
  L.nband = (int)((g.ny + rows - 1) / rows);
  L.ytiles_per_band = (int)(rows / kYTile);
  L.xfull = (int)(g.nx / xtile);
  L.xtiles = (int)((g.nx + xtile - 1) / xtile);
  L.ycols = (int)((g.nx + kYCols - 1) / kYCols);
  L.slot_vstride = rows * g.pitch;
  L.slot_elems = 4 * L.slot_vstride;
  for (int b = 0; b <= L.nband; ++b) L.row0[b] = (int)std::min<int64_t>((int64_t)b * rows, g.ny);
  for (int b = 0; b < L.nband; ++b) {
    const int64_t nrow = L.row0[b + 1] - L.row0[b];
    const int64_t ntr = (nrow + kYTile - 1) / kYTile;
    L.x_items[b] = (unsigned)(nrow * L.xtiles);
    L.y_items[b] = (unsigned)(ntr * L.ycols);
  }
  int64_t at = 0;
  int j = 0;
  auto push = [&](int kind, int b) {
    L.seg_start[j] = (int)at;
    L.seg_kind[j] = (unsigned char)kind;
    L.seg_band[j] = (unsigned char)b;
    at += kind == 0 ? L.x_items[b] : L.y_items[b];
    ++j;
  };
  for (int b = 0; b < std::min(kBandLead, L.nband); ++b) push(0, b);
  for (int b = 0; b < L.nband; ++b) {
    if (b + kBandLead < L.nband) push(0, b + kBandLead);
    push(1, b);
  }
  L.nseg = j;
  L.seg_start[j] = (int)at;
  return L;
}

// Bytes of the partial-stage ring for a 2D grid of element size `elem`.
inline size_t band_ring_bytes(const GridInfo& g, size_t elem) {
  return (size_t)kBandRing * 4 * (size_t)band_rows(g.ny) * (size_t)g.pitch * elem;
}

}  // namespace wcns
