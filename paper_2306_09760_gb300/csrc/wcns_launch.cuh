// Launchers for one element type T; included by the per-type, per-family units wcns_f32*.cu / wcns_f64*.cu.
#pragma once

#include <algorithm>
#include <atomic>

#include "wcns_internal.h"
#include "wcns_kernels.cuh"
#include "wcns_adjoint_kernels.cuh"
#include "wcns_stats.cuh"
#include "wcns_band.cuh"

namespace wcns {

// FIX = 1 (compile-time default configuration) applies to the Euler systems only.
template <int NV>
static bool use_fixed(const Scheme& s) {
  return NV > 1 && fixed_config(s);
}

template <typename T, int NV, int MODE, int P, int TH = kXThreads>
static cudaError_t run_sweep_x_per(const GridInfo& g, const SweepArgs<T>& A0, bool fixed, cudaStream_t st) {
  const size_t smem = sweep_x_smem<T, NV, P, TH>();
  const int64_t tiles = (g.nx + sweep_x_tile<P, TH>() - 1) / sweep_x_tile<P, TH>();
  // Blocks run in order of blockIdx.x first: with rows along x every row's first tiles are
  // scheduled before any ragged last tile, so the short blocks of the ragged tiles come
  // last and fill the grid's final partial wave (grid y is limited to 65535).
  SweepArgs<T> A = A0;
  A.row_major = tiles <= 65535 ? 1 : 0;
  dim3 grid = A.row_major ? dim3((unsigned)g.ny, (unsigned)tiles) : dim3((unsigned)tiles, (unsigned)g.ny);
  if (fixed) sweep_x_kernel<T, NV, MODE, (NV > 1 ? 1 : 0), P, TH><<<grid, TH, smem, st>>>(A);
  else sweep_x_kernel<T, NV, MODE, 0, P, TH><<<grid, TH, smem, st>>>(A);
  return cudaGetLastError();
}

// SM count of the current device, written by configure_kernels (before any launch or
// capture).  Contexts may be created and used on several host threads, so the value and
// the occupancy figures below are atomics.
inline std::atomic<int>& sweep_sm_count() {
  static std::atomic<int> nsm{0};
  return nsm;
}
inline int sm_count_or_one() {
  const int n = sweep_sm_count().load(std::memory_order_relaxed);
  return n > 0 ? n : 1;
}

// Four interfaces per thread (single-precision Euler systems) when the grid gives at
// least two full waves of such blocks (four per SM), else one.
inline bool sweep_x_wide(const GridInfo& g) {
  const int nsm = sm_count_or_one();
  const int64_t blocks = g.ny * ((g.nx + sweep_x_tile<4>() - 1) / sweep_x_tile<4>());
  return blocks >= 2 * 4 * (int64_t)nsm;
}

// Narrow (kXNarrow-thread) blocks for the one-variable and 1D Euler systems when
// 256-thread tiles would give fewer blocks than SMs: a line of 4096 cells then spreads
// over 152 blocks of 27 cells instead of 17 blocks of 251, at 5/27 redundant interfaces.
inline bool sweep_x_narrow(const GridInfo& g) {
  const int nsm = sm_count_or_one();
  const int64_t blocks = g.ny * ((g.nx + sweep_x_tile<1>() - 1) / sweep_x_tile<1>());
  return blocks < (int64_t)nsm;
}

template <typename T, int NV, int MODE>
static cudaError_t run_sweep_x(const GridInfo& g, const SweepArgs<T>& A, bool fixed, cudaStream_t st) {
  if constexpr (sizeof(T) == 4 && NV > 1) {
    if (sweep_x_wide(g)) return run_sweep_x_per<T, NV, MODE, 4>(g, A, fixed, st);
  }
  if constexpr (NV < 4) {
    if (sweep_x_narrow(g)) return run_sweep_x_per<T, NV, MODE, 1, kXNarrow>(g, A, fixed, st);
  }
  return run_sweep_x_per<T, NV, MODE, 1>(g, A, fixed, st);
}

// One variable count's x sweeps, instantiated in a unit of its own (wcns_<type>_x<NV>.cu).
template <typename T, int NV>
cudaError_t sweep_x_nv(const GridInfo& g, const SweepArgs<T>& A, bool stage, bool fixed, cudaStream_t st) {
  return stage ? run_sweep_x<T, NV, kStage>(g, A, fixed, st) : run_sweep_x<T, NV, kWriteL>(g, A, fixed, st);
}

template <typename T, int NV, int MODE>
static cudaError_t run_sweep_y(const GridInfo& g, const SweepArgs<T>& A, bool fixed, cudaStream_t st) {
  const size_t smem = sweep_y_smem<T, NV>();
  dim3 grid((unsigned)((g.nx + kYCols - 1) / kYCols), (unsigned)((g.ny + kYTile - 1) / kYTile));
  dim3 block(kYCols, kYRowsT);
  if (fixed) sweep_y_kernel<T, NV, MODE, (NV > 1 ? 1 : 0)><<<grid, block, smem, st>>>(A);
  else sweep_y_kernel<T, NV, MODE, 0><<<grid, block, smem, st>>>(A);
  return cudaGetLastError();
}

template <typename T>
static SweepArgs<T> make_args(const GridInfo& g, const Scheme& s, int dir, const SweepCall<T>& c) {
  SweepArgs<T> A{};
  A.nx = g.nx; A.ny = g.ny; A.pitch = g.pitch; A.fstride = g.ny * g.pitch;
  A.bc = g.bc[dir];
  A.inv_h = T(1.0 / g.h[dir]);
  A.s = scheme_as<T>(s);
  A.fallbacks = c.fallbacks;
  A.u = c.u; A.un = c.un; A.R = c.R; A.out = c.out; A.dt = c.dt;
  A.a = T(c.a); A.b = T(c.b);
  A.general = c.general ? 1 : 0;
  A.e = T(c.e); A.c1 = T(c.c1); A.c2 = T(c.c2);
  A.X1 = c.X1; A.X2 = c.X2;
  if (c.faces) A.f = faces_as<T>(*c.faces);
  A.cstage = c.cstage;
  A.tnow = c.tnow;
  A.wave = c.wave;
  A.err = c.err;
  A.status = c.status;
  return A;
}

// The tensor map of state buffer u as a (x, y, variable) tensor with the y sweep's
// kYCols x kYCells x nvar box (columns beyond nx read as zeros); false when the driver
// entry point is missing or refuses the layout (the sweep then stages with loads).  The
// entry point is fetched through the runtime, so the library needs no link to libcuda.
template <typename T>
static bool encode_y_map(const GridInfo& g, const T* u, CUtensorMap* map) {
  using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static const EncodeFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeFn) nullptr;
    return reinterpret_cast<EncodeFn>(f);
  }();
  if (!fn || !u || (reinterpret_cast<uintptr_t>(u) & 15u)) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nvar};
  const cuuint64_t strides[2] = {(cuuint64_t)g.pitch * sizeof(T), (cuuint64_t)g.ny * (cuuint64_t)g.pitch * sizeof(T)};
  const cuuint32_t box[3] = {(cuuint32_t)kYCols, (cuuint32_t)kYCells, (cuuint32_t)g.nvar};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
            const_cast<T*>(u), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T, int NV, int FIX, int P, int TH = kXThreads>
static cudaError_t configure_x() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(sweep_x_kernel<T, NV, kWriteL, FIX, P, TH>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sweep_x_smem<T, NV, P, TH>())) != cudaSuccess) return e;
  return cudaFuncSetAttribute(sweep_x_kernel<T, NV, kStage, FIX, P, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sweep_x_smem<T, NV, P, TH>());
}

template <typename T, int NV, int FIX>
static cudaError_t configure_x_fix() {
  cudaError_t e;
  if ((e = configure_x<T, NV, FIX, 1>()) != cudaSuccess) return e;
  if constexpr (sizeof(T) == 4 && NV > 1) {
    if ((e = configure_x<T, NV, FIX, 4>()) != cudaSuccess) return e;
  }
  if constexpr (NV < 4) {
    if ((e = configure_x<T, NV, FIX, 1, kXNarrow>()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T, int NV, int FIX>
static cudaError_t configure_y_fix() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(sweep_y_kernel<T, NV, kWriteL, FIX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sweep_y_smem<T, NV>())) != cudaSuccess) return e;
  return cudaFuncSetAttribute(sweep_y_kernel<T, NV, kStage, FIX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sweep_y_smem<T, NV>());
}

template <typename T, int NV>
cudaError_t configure_x_nv() {
  cudaError_t e = configure_x_fix<T, NV, 0>();
  if constexpr (NV == 1) {
    return e;
  } else {
    if (e != cudaSuccess) return e;
    return configure_x_fix<T, NV, 1>();
  }
}

template <typename T, int NV>
static cudaError_t configure_y_nv() {
  cudaError_t e = configure_y_fix<T, NV, 0>();
  if constexpr (NV == 1) {
    return e;
  } else {
    if (e != cudaSuccess) return e;
    return configure_y_fix<T, NV, 1>();
  }
}

template <typename T, int NV>
static cudaError_t configure_adjoint() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(adjoint_x_kernel<T, NV, kAdjWrite>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)adj_x_smem<T, NV>())) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(adjoint_x_kernel<T, NV, kAdjCombine>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)adj_x_smem<T, NV>())) != cudaSuccess) return e;
  if constexpr (NV == 4) {
    return cudaFuncSetAttribute(adjoint_y_kernel<T, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)adj_y_smem<T, NV>());
  }
  return cudaSuccess;
}

// Resident blocks of the CFL kernel on the whole GPU (occupancy x SMs), read once.
template <typename T, int NV>
static int64_t dt_wave_blocks_nv() {
  static std::atomic<int64_t> cached{0};
  int64_t n = cached.load(std::memory_order_relaxed);
  if (n <= 0) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dt_kernel<T, NV>, kRedThreads, 0) != cudaSuccess ||
        occ <= 0)
      occ = 1;
    n = (int64_t)occ * sm_count_or_one();
    cached.store(n, std::memory_order_relaxed);
  }
  return n;
}
template <typename T>
static int64_t dt_wave_blocks(int nvar) {
  return nvar == 4 ? dt_wave_blocks_nv<T, 4>() : dt_wave_blocks_nv<T, 3>();
}

// Shared-memory attributes per kernel family; each family's part is instantiated in the
// translation unit that compiles that family's kernels (wcns_<type>_<family>.cu).
template <typename T>
cudaError_t configure_sweep_x(int nvar) {
  switch (nvar) {
    case 1: return configure_x_nv<T, 1>();
    case 3: return configure_x_nv<T, 3>();
    case 4: return configure_x_nv<T, 4>();
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t configure_sweep_y(int nvar) {
  switch (nvar) {
    case 1: return configure_y_nv<T, 1>();
    case 3: return cudaSuccess;  // no y sweep in 1D Euler
    case 4: return configure_y_nv<T, 4>();
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t configure_adjoints(int nvar) {
  switch (nvar) {
    case 1: return cudaSuccess;
    case 3: return configure_adjoint<T, 3>();
    case 4: return configure_adjoint<T, 4>();
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t configure_band();

template <typename T>
cudaError_t configure_kernels(int nvar) {
  cudaError_t e;
  int dev = 0, nsm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  sweep_sm_count().store(nsm, std::memory_order_relaxed);
  if (nvar != 1 && nvar != 3 && nvar != 4) return cudaErrorInvalidValue;
  if (nvar > 1) (void)dt_wave_blocks<T>(nvar);  // occupancy query before any stream capture
  if ((e = configure_sweep_x<T>(nvar)) != cudaSuccess) return e;
  if ((e = configure_sweep_y<T>(nvar)) != cudaSuccess) return e;
  if (nvar == 4 && (e = configure_band<T>()) != cudaSuccess) return e;
  return configure_adjoints<T>(nvar);
}

template <typename T>
static AdjArgs<T> make_adj_args(const GridInfo& g, const Scheme& s, int dir, const AdjCall<T>& c) {
  AdjArgs<T> A{};
  A.u = c.u; A.mu = c.mu; A.R = c.R; A.X1 = c.X1; A.X2 = c.X2; A.out = c.out;
  A.c1 = T(c.c1); A.c2 = T(c.c2); A.b = T(c.b); A.dt = T(c.dt);
  A.nx = g.nx; A.ny = g.ny; A.pitch = g.pitch; A.fstride = g.ny * g.pitch;
  A.bc = g.bc[dir];
  A.inv_h = T(1.0 / g.h[dir]);
  A.s = scheme_as<T>(s);
  return A;
}

template <typename T>
cudaError_t launch_adjoint_x(const GridInfo& g, const Scheme& s, const AdjCall<T>& c, cudaStream_t st) {
  AdjArgs<T> A = make_adj_args<T>(g, s, 0, c);
  dim3 grid((unsigned)((g.nx + kXTile - 1) / kXTile), (unsigned)g.ny);
  switch (g.nvar) {
    case 3:
      if (c.combine) adjoint_x_kernel<T, 3, kAdjCombine><<<grid, kAXThreads, adj_x_smem<T, 3>(), st>>>(A);
      else adjoint_x_kernel<T, 3, kAdjWrite><<<grid, kAXThreads, adj_x_smem<T, 3>(), st>>>(A);
      break;
    case 4:
      if (c.combine) adjoint_x_kernel<T, 4, kAdjCombine><<<grid, kAXThreads, adj_x_smem<T, 4>(), st>>>(A);
      else adjoint_x_kernel<T, 4, kAdjWrite><<<grid, kAXThreads, adj_x_smem<T, 4>(), st>>>(A);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adjoint_y(const GridInfo& g, const Scheme& s, const AdjCall<T>& c, cudaStream_t st) {
  if (g.nvar != 4) return cudaErrorInvalidValue;
  AdjArgs<T> A = make_adj_args<T>(g, s, 1, c);
  dim3 grid((unsigned)((g.nx + kAYCols - 1) / kAYCols), (unsigned)((g.ny + kAYTile - 1) / kAYTile));
  dim3 block(kAYCols, kAYRowsT);
  adjoint_y_kernel<T, 4><<<grid, block, adj_y_smem<T, 4>(), st>>>(A);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sweep_x(const GridInfo& g, const Scheme& s, const SweepCall<T>& c, cudaStream_t st) {
  SweepArgs<T> A = make_args<T>(g, s, 0, c);
  // the 2D stage writes the partial stage from the x sweep (same kernel body as kStage)
  switch (g.nvar) {
    case 1: return sweep_x_nv<T, 1>(g, A, c.stage, false, st);
    case 3: return sweep_x_nv<T, 3>(g, A, c.stage, use_fixed<3>(s), st);
    case 4: return sweep_x_nv<T, 4>(g, A, c.stage, use_fixed<4>(s), st);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_sweep_y(const GridInfo& g, const Scheme& s, const SweepCall<T>& c, cudaStream_t st) {
  SweepArgs<T> A = make_args<T>(g, s, 1, c);
  A.ytma = encode_y_map<T>(g, A.u, &A.ymap) ? 1 : 0;
  switch (g.nvar) {
    case 1: return c.stage ? run_sweep_y<T, 1, kStage>(g, A, false, st) : run_sweep_y<T, 1, kWriteL>(g, A, false, st);
    case 4: {
      const bool f = use_fixed<4>(s);
      return c.stage ? run_sweep_y<T, 4, kStage>(g, A, f, st) : run_sweep_y<T, 4, kWriteL>(g, A, f, st);
    }
  }
  return cudaErrorInvalidValue;
}

// Resident blocks of one banded-stage kernel on the whole GPU (occupancy x SMs), read
// at configuration time (before any stream capture).
template <typename T, int FIX, int P>
static std::atomic<int>& band_blocks_nv() {
  static std::atomic<int> n{0};
  return n;
}

template <typename T, int FIX, int P>
static cudaError_t configure_band_one() {
  cudaError_t e = cudaFuncSetAttribute(stage_band_kernel<T, FIX, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)stage_band_smem<T, P>());
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, stage_band_kernel<T, FIX, P>, kXThreads,
                                                    stage_band_smem<T, P>());
  if (e != cudaSuccess) return e;
  band_blocks_nv<T, FIX, P>().store((occ > 0 ? occ : 1) * sm_count_or_one(), std::memory_order_relaxed);
  return cudaSuccess;
}

// x tiles per thread of the banded stage: four in single precision, one in double.
template <typename T>
constexpr int band_p() { return sizeof(T) == 4 ? 4 : 1; }

// The banded stage is compiled for the default scheme configuration only (the FIX = 1
// kernels), which keeps its build unit small.
template <typename T>
cudaError_t configure_band() {
  return configure_band_one<T, 1, band_p<T>()>();
}

// The banded stage applies to 2D Euler stages of the default scheme configuration on
// grids with enough bands to fill the ring; single precision also needs the grid to take
// the wide (four-interface) x tiles.
template <typename T>
bool band_applies(const GridInfo& g, const Scheme& s) {
  if (g.ndim != 2 || g.nvar != 4 || !use_fixed<4>(s)) return false;
  if (sizeof(T) == 4 && !sweep_x_wide(g)) return false;
  // work items are counted in int
  const int64_t xt = (g.nx + sweep_x_tile<band_p<T>()>() - 1) / sweep_x_tile<band_p<T>()>();
  const int64_t items = g.ny * xt + ((g.nx + kYCols - 1) / kYCols) * ((g.ny + kYTile - 1) / kYTile);
  if (items >= ((int64_t)1 << 31)) return false;
  return (g.ny + band_rows(g.ny) - 1) / band_rows(g.ny) > kBandRing;
}

// One 2D stage (x then y sweep of the same stage arguments as launch_sweep_x/_y) as a
// banded persistent launch.  ring: band_ring_bytes(g, sizeof(T)); ctr: kBandCounters
// zeroed words (left zeroed by the launch).
template <typename T>
cudaError_t launch_stage_band(const GridInfo& g, const Scheme& s, const SweepCall<T>& x, const SweepCall<T>& y,
                              T* ring, unsigned* ctr, int* err, cudaStream_t st) {
  constexpr int P = band_p<T>();
  BandArgs<T> B{};
  B.X = make_args<T>(g, s, 0, x);
  B.Y = make_args<T>(g, s, 1, y);
  B.Y.ytma = encode_y_map<T>(g, B.Y.u, &B.Y.ymap) ? 1 : 0;
  B.plan = make_band_plan(g, sweep_x_tile<P>());
  B.ring = ring;
  B.ctr = ctr;
  B.err = err;
  if (!band_applies<T>(g, s)) return cudaErrorInvalidValue;
  const int nitems = B.plan.seg_start[B.plan.nseg];
  const int resident = band_blocks_nv<T, 1, P>().load(std::memory_order_relaxed);
  if (resident <= 0) return cudaErrorInitializationError;
  // a cooperative launch: every block is resident at once (the kernel's progress needs it)
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)std::min(nitems, resident));
  cfg.blockDim = dim3(kXThreads);
  cfg.dynamicSmemBytes = stage_band_smem<T, P>();
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, stage_band_kernel<T, 1, P>, B);
}

template <typename T>
cudaError_t launch_dt(const GridInfo& g, const DtLaunch& d, cudaStream_t st) {
  DtArgs A{};
  A.u = d.u; A.copy = g.nvar > 1 ? d.copy : nullptr; A.nx = g.nx; A.ny = g.ny; A.pitch = g.pitch; A.fstride = g.ny * g.pitch;
  A.nvar = g.nvar; A.ndim = g.ndim; A.use_cfl = d.use_cfl;
  A.gamma = d.gamma; A.cfl = d.cfl; A.hx = g.h[0]; A.hy = g.h[1];
  A.fixed_dt = d.fixed_dt; A.t_end = d.t_end;
  A.adv_wave[0] = d.adv_wave[0]; A.adv_wave[1] = d.adv_wave[1];
  A.partials = d.partials; A.counter = d.counter; A.dt_out = d.dt_out; A.step = d.step; A.t = d.t;
  A.steps = d.steps; A.err = d.err; A.wave = d.wave;
  int blocks = 1;
  A.bpr = 1;
  if (g.nvar > 1) {
    // whole rows per block when there are enough rows, else rows split in chunks; at
    // most one wave of resident blocks (a second, partial wave would double the time)
    const int64_t vw = 16 / (int64_t)sizeof(T);
    const int64_t nvec = (g.nx + vw - 1) / vw;
    const int64_t max_blocks = std::min<int64_t>(d.max_blocks, dt_wave_blocks<T>(g.nvar));
    if (g.ny * 2 >= max_blocks) {
      const int64_t rpb = (g.ny + max_blocks - 1) / max_blocks;
      blocks = (int)((g.ny + rpb - 1) / rpb);
    } else {
      int64_t bpr = max_blocks / g.ny;
      const int64_t useful = (nvec + kRedThreads - 1) / kRedThreads;
      bpr = bpr < 1 ? 1 : (bpr > useful ? useful : bpr);
      A.bpr = (int)bpr;
      blocks = (int)(g.ny * bpr);
    }
  }
  switch (g.nvar) {
    case 1: dt_kernel<T, 1><<<blocks, kRedThreads, 0, st>>>(A); break;
    case 3: dt_kernel<T, 3><<<blocks, kRedThreads, 0, st>>>(A); break;
    case 4: dt_kernel<T, 4><<<blocks, kRedThreads, 0, st>>>(A); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_step_from_maxima(const GridInfo& g, const DtLaunch& d, cudaStream_t st) {
  DtArgs A{};
  A.nvar = g.nvar; A.ndim = g.ndim; A.use_cfl = d.use_cfl;
  A.cfl = d.cfl; A.hx = g.h[0]; A.hy = g.h[1]; A.fixed_dt = d.fixed_dt; A.t_end = d.t_end;
  A.adv_wave[0] = d.adv_wave[0]; A.adv_wave[1] = d.adv_wave[1];
  A.step = d.step; A.t = d.t; A.steps = d.steps; A.err = d.err; A.wave = d.wave;
  if (!A.wave || !A.t) return cudaErrorInvalidValue;
  step_from_maxima_kernel<T><<<1, kWaveSlots, 0, st>>>(A);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_reduce(const GridInfo& g, const void* a, const void* b, int what, double* partials,
                          int max_blocks, unsigned int* counters, double* out, cudaStream_t st) {
  ReduceArgs A{};
  A.a = a; A.b = b; A.nx = g.nx; A.ny = g.ny; A.pitch = g.pitch; A.fstride = g.ny * g.pitch;
  A.what = what; A.partials = partials; A.counters = counters; A.out = out;
  const int64_t ncell = g.nx * g.ny;
  int64_t want = (ncell + kRedThreads * 4 - 1) / (kRedThreads * 4);
  int per_var = max_blocks / g.nvar;
  int blocks = (int)(want < 1 ? 1 : (want > per_var ? per_var : want));
  dim3 grid(blocks, g.nvar);
  reduce_kernel<T><<<grid, kRedThreads, 0, st>>>(A);
  return cudaGetLastError();
}

}  // namespace wcns

namespace wcns {

template <typename T>
cudaError_t launch_weight_hist(const GridInfo& g, const Scheme& s, const Faces<double>& f, const double* tnow,
                               const void* u, int nbins, unsigned long long* hist, cudaStream_t st) {
  for (int dir = 0; dir < g.ndim; ++dir) {
    HistArgs<T> A{};
    A.u = static_cast<const T*>(u);
    A.n = dir == 0 ? g.nx : g.ny;
    A.lines = dir == 0 ? g.ny : g.nx;
    A.pitch = g.pitch;
    A.fstride = g.ny * g.pitch;
    A.dir = dir;
    A.bc = g.bc[dir];
    A.kmin = s.family == 1 ? -1 : -3;
    A.nk = s.family == 1 ? A.n + 1 : A.n + 5;
    A.s = scheme_as<T>(s);
    A.rec.hist = hist;
    A.rec.nbins = nbins;
    A.f = faces_as<T>(f);
    A.tnow = tnow;
    const int64_t threads = A.lines * A.nk;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    switch (g.nvar) {
      case 1: weight_hist_kernel<T, 1><<<blocks, 256, 0, st>>>(A); break;
      case 3: weight_hist_kernel<T, 3><<<blocks, 256, 0, st>>>(A); break;
      case 4: weight_hist_kernel<T, 4><<<blocks, 256, 0, st>>>(A); break;
      default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace wcns

// Explicit instantiations per kernel family.  A unit that instantiates one family declares
// the others extern, so it compiles none of their kernels.
#define WCNS_EXTERN_FAMILIES(T)                                                                      \
  namespace wcns {                                                                                   \
  extern template cudaError_t configure_x_nv<T, 1>();                                                \
  extern template cudaError_t configure_x_nv<T, 3>();                                                \
  extern template cudaError_t configure_x_nv<T, 4>();                                                \
  extern template cudaError_t sweep_x_nv<T, 1>(const GridInfo&, const SweepArgs<T>&, bool, bool,    \
                                               cudaStream_t);                                        \
  extern template cudaError_t sweep_x_nv<T, 3>(const GridInfo&, const SweepArgs<T>&, bool, bool,    \
                                               cudaStream_t);                                        \
  extern template cudaError_t sweep_x_nv<T, 4>(const GridInfo&, const SweepArgs<T>&, bool, bool,    \
                                               cudaStream_t);                                        \
  extern template cudaError_t configure_sweep_y<T>(int);                                             \
  extern template cudaError_t configure_adjoints<T>(int);                                            \
  extern template cudaError_t configure_band<T>();                                                   \
  }

#define WCNS_INSTANTIATE_X(T, NV)                                                                    \
  namespace wcns {                                                                                   \
  template cudaError_t configure_x_nv<T, NV>();                                                      \
  template cudaError_t sweep_x_nv<T, NV>(const GridInfo&, const SweepArgs<T>&, bool, bool,          \
                                         cudaStream_t);                                              \
  }

#define WCNS_INSTANTIATE_Y(T)                                                                        \
  namespace wcns {                                                                                   \
  template cudaError_t configure_sweep_y<T>(int);                                                    \
  template cudaError_t launch_sweep_y<T>(const GridInfo&, const Scheme&, const SweepCall<T>&,       \
                                         cudaStream_t);                                              \
  }

#define WCNS_INSTANTIATE_BAND(T)                                                                     \
  namespace wcns {                                                                                   \
  template cudaError_t configure_band<T>();                                                          \
  template bool band_applies<T>(const GridInfo&, const Scheme&);                                     \
  template cudaError_t launch_stage_band<T>(const GridInfo&, const Scheme&, const SweepCall<T>&,    \
                                            const SweepCall<T>&, T*, unsigned*, int*, cudaStream_t); \
  }

#define WCNS_INSTANTIATE_ADJ(T)                                                                      \
  namespace wcns {                                                                                   \
  template cudaError_t configure_adjoints<T>(int);                                                   \
  template cudaError_t launch_adjoint_x<T>(const GridInfo&, const Scheme&, const AdjCall<T>&,       \
                                           cudaStream_t);                                            \
  template cudaError_t launch_adjoint_y<T>(const GridInfo&, const Scheme&, const AdjCall<T>&,       \
                                           cudaStream_t);                                            \
  }

#define WCNS_INSTANTIATE_MISC(T)                                                                     \
  WCNS_EXTERN_FAMILIES(T)                                                                            \
  namespace wcns {                                                                                   \
  template cudaError_t configure_kernels<T>(int);                                                    \
  template cudaError_t launch_sweep_x<T>(const GridInfo&, const Scheme&, const SweepCall<T>&,       \
                                         cudaStream_t);                                              \
  template cudaError_t launch_dt<T>(const GridInfo&, const DtLaunch&, cudaStream_t);                 \
  template cudaError_t launch_step_from_maxima<T>(const GridInfo&, const DtLaunch&, cudaStream_t);   \
  template cudaError_t launch_weight_hist<T>(const GridInfo&, const Scheme&, const Faces<double>&,  \
                                             const double*, const void*, int, unsigned long long*,   \
                                             cudaStream_t);                                          \
  template cudaError_t launch_reduce<T>(const GridInfo&, const void*, const void*, int, double*, int, \
                                        unsigned int*, double*, cudaStream_t);                       \
  }
