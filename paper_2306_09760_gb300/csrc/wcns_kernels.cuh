// Kernels of the WCNS-FE hot path: per-direction sweeps fused with the TVD-RK3 stage
// update, the CFL step reduction and the FP64 norm reductions.
//
// Sweep structure (per RK stage, Eq. 2-3 + steps (a)-(e)):
//   1D:  sweep_x computes L and the stage update in one kernel.
//   2D:  sweep_x writes the partial stage a*u^n + b*(u + dt*L_x) (L_x alone for an RHS
//        evaluation) into a scratch plane set; sweep_y computes L_y and completes the
//        stage as R + b*dt*L_y.  Splitting the sweeps keeps the redundant interface
//        work at the tile edges small (x: 5 interfaces per 251- or 1019-cell tile;
//        y: 80 interfaces for 75 rows), where a fused 2D tile of 32 x 32 cells
//        recomputes ~16% of its interfaces; the extra plane traffic (one write and one
//        read of R) is hidden under the arithmetic.  The banded form (wcns_band.cuh)
//        runs both sweeps of a stage in one persistent launch with R kept in L2.
//
// A tile of T output cells along a line needs the T + 5 interfaces
// F_{c0-5/2} .. F_{c0+T-1+5/2}, which need the T + 10 cells c0-5 .. c0+T+4.  Ghost
// cells are produced by index arithmetic while the tile is staged in shared memory.
#pragma once

#include <cuda.h>

#include "wcns_device.cuh"
#include "wcns_pair.cuh"

namespace wcns {

// Stage coefficients: out = a * un + b * (u + dt * L).
template <typename T>
struct SweepArgs {
  const T* u;          // state the RHS is evaluated on
  const T* un;         // u^n (read only when a != 0)
  const T* R;          // L_x planes (y sweep of a 2D grid)
  T* out;              // destination (L, L_x or the stage state)
  const StepDt* dt;    // device step (stage modes)
  T a, b;
  // General stage form (RK4, Eq. 16): out = a*un + b*u + e*dt*L + c1*X1 + c2*X2.
  // When `general` is 0 the TVD-RK3 form a*un + b*(u + dt*L) is used as written.
  int general;
  T e, c1, c2;
  const T* X1;
  const T* X2;
  int64_t nx, ny, pitch, fstride;  // fstride = ny * pitch (elements per variable plane)
  int bc;              // boundary of this sweep's direction
  T inv_h;
  SchemeT<T> s;
  unsigned long long* fallbacks;   // interfaces that fell back to first order
  // y sweep of a 2D stage that completes an RK step (or null): the CFL maxima of the
  // cells it writes, max |u| + c and max |v| + c, merged per warp with atomicMax into
  // kWaveSlots slot pairs (bit patterns of non-negative doubles, whose integer order is
  // their numeric order; spreading the warps over slots keeps the atomics uncontended);
  // a non-physical written cell sets bit 0 of *err
  unsigned long long* wave;
  int* err;
  Faces<T> f;                      // boundary faces beyond periodic / transmissive lines
  double cstage;                   // stage time t0 + cstage * dt of the state read (faces)
  const double* tnow;              // device time (faces, RHS without a step)
  int row_major;                   // x sweep: blockIdx.x = row, blockIdx.y = tile (else swapped)
  // y sweep: tensor map of u as a (x, y, variable) tensor with a kYCols x kYCells x nvar
  // box, used to stage the tiles whose rows all lie inside the grid (ytma = 1); else the
  // per-thread loads stage every tile
  int ytma;
  int* status;                     // sticky error word (bit 1: a bounded wait ran out)
  CUtensorMap ymap;
};

// ---------------------------------------------------------------------------
// Tensor-memory-access (TMA) staging: one thread issues a bulk tensor copy of a whole
// tile into shared memory, completed on an mbarrier that every thread of the block waits
// on (bounded).
// ---------------------------------------------------------------------------
constexpr int kTmaSpin = 1 << 20;         // polls of the mbarrier before a wait gives up
constexpr unsigned kTmaPollNs = 1000;     // suspend-time hint of one poll (ns): a wait lasts about a second at most

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" : : "r"(smem_u32(bar)), "r"(count) : "memory");
  // make the initialised barrier visible to the async proxy (the copy engine)
  asm volatile("fence.mbarrier_init.release.cluster;" : : : "memory");
  asm volatile("fence.proxy.async.shared::cta;" : : : "memory");
}

// Arms the barrier for `bytes` of transfer and issues the copy of the box at (x, y, z)
// of the tensor map into dst.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, unsigned long long* bar, int x,
                                            int y, int z, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" : : "r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];"
      :
      : "r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z),
        "r"(smem_u32(bar))
      : "memory");
}

// Waits until phase `parity` of the barrier has completed; false after kTmaSpin polls,
// each suspended for at most about kTmaPollNs.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  for (int it = 0; it < kTmaSpin; ++it) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kTmaPollNs)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Time of the state a sweep reads, for time-dependent boundary faces.
template <typename T>
__device__ __forceinline__ double sweep_time(const SweepArgs<T>& A) {
  if (!A.f.active) return 0.0;
  return A.dt ? A.dt->t0 + A.cstage * A.dt->dt : *A.tnow;
}

// kWriteL: out = L (or L_x).  kStage: out = a*un + b*(u + dt*L).  In a 2D stage the x
// sweep runs in kStage form with L_x and writes the partial stage into R; the y sweep
// then adds b*dt*L_y, so its epilogue reads one array instead of two.
enum SweepMode { kWriteL = 0, kStage = 1 };

// Adds the warp's count of true flags to *ctr (one atomic per warp, by its first flagged lane).
__device__ __forceinline__ void count_fallbacks(bool fb, unsigned long long* ctr) {
  unsigned m = __ballot_sync(0xffffffffu, fb);
  unsigned lane;
  asm("mov.u32 %0, %%laneid;" : "=r"(lane));
  if (m && lane == ((unsigned)__ffs(m) - 1)) atomicAdd(ctr, (unsigned long long)__popc(m));
}

// Signal speeds |u| + c and |v| + c of one cell (rho, rho u, rho v, E) in the state's own
// precision; false for a non-physical state (rho <= 0, p <= 0 or NaN).  The CFL kernel
// and the fused stage epilogue share it, so both reduce the same values.
template <typename T>
__device__ __forceinline__ bool cell_wave(T rho, T mu, T mv, T E, T g, T gm1, T& wx, T& wy) {
  const T inv = T(1) / rho;
  const T ux = mu * inv, vy = mv * inv;
  const T p = gm1 * (E - T(0.5) * rho * (ux * ux + vy * vy));
  if (!(rho > T(0)) || !(p > T(0))) return false;
  const T cs = Num<T>::sqrt_(g * p * inv);
  wx = Num<T>::abs_(ux) + cs;
  wy = Num<T>::abs_(vy) + cs;
  return true;
}

// Warp maxima of two non-negative values (every lane of the warp calls it; lanes with
// nothing to add pass 0) merged into one of kWaveSlots slot pairs of wave with
// atomicMax, and the warp's non-physical flag into *err.
template <typename T>
__device__ __forceinline__ void warp_wave(T mx, T my, bool bad, unsigned vblock, unsigned long long* wave,
                                          int* err) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    my = fmax(my, __shfl_xor_sync(0xffffffffu, my, o));
  }
  const bool anybad = __any_sync(0xffffffffu, bad);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if ((tid & 31) == 0) {
    const unsigned slot = (vblock * (blockDim.x * blockDim.y / 32) +
                           (unsigned)(tid >> 5)) % kWaveSlots;
    atomicMax(&wave[2 * slot], (unsigned long long)__double_as_longlong((double)mx));
    atomicMax(&wave[2 * slot + 1], (unsigned long long)__double_as_longlong((double)my));
    if (anybad) atomicOr(err, 1);
  }
}

// ---------------------------------------------------------------------------
// x sweep: one block per (row, tile of cells); 256 threads, P interfaces per thread
// (interfaces t, t + 256, ...), so a block covers 256 P interfaces and 256 P - 5 cells.
// kXThreads / kXTile / kXCells are the one-interface-per-thread tile of the adjoint.
// ---------------------------------------------------------------------------
constexpr int kXThreads = 256;
constexpr int kXTile = kXThreads - 5;      // output cells per block
constexpr int kXCells = kXThreads + 5;     // staged cells per block

// P interfaces per thread: four for single-precision grids large enough to fill the GPU
// with such blocks (2048^2 x sweep 0.176 ms at one, 0.174 at two, 0.167 at four), else
// one (more, shorter blocks for small grids and for double precision).  TH threads per
// block: 256, or kXNarrow for lines too short to give every SM a 256-thread block.
constexpr int kXNarrow = 32;
template <int P, int TH = kXThreads>
constexpr int sweep_x_ifc() { return TH * P; }   // interfaces per block
template <int P, int TH = kXThreads>
constexpr int sweep_x_tile() { return sweep_x_ifc<P, TH>() - 5; }          // output cells per block
template <int P, int TH = kXThreads>
constexpr int sweep_x_cells() { return sweep_x_ifc<P, TH>() + 5; }         // staged cells per block

// staged cells, interface fluxes and (P > 1) u^n of the tile's cells
template <typename T, int NV, int P, int TH = kXThreads>
constexpr size_t sweep_x_smem() {
  return sizeof(T) * NV * (sweep_x_cells<P, TH>() + sweep_x_ifc<P, TH>() + (P > 1 ? sweep_x_tile<P, TH>() : 0));
}

// Single-precision sweeps ask for four resident blocks (32 warps per SM, at most 64
// registers per thread); double precision keeps the compiler's choice.
template <typename T>
constexpr int sweep_min_blocks() { return sizeof(T) == 4 ? 4 : 1; }

// One x tile (row `row`, tile `tile` of the row) of the sweep; the block calls it
// together.  The result goes to out[k * ostride + (row - orow0) * pitch + c] (the grid's
// own layout when ostride = fstride and orow0 = 0; a band of rows of the partial-stage
// ring otherwise).
template <typename T, int NV, int MODE, int FIX, int P, int TH = kXThreads>
__device__ __forceinline__ void sweep_x_body(const SweepArgs<T>& A, int64_t row, int64_t tile, T* out,
                                             int64_t ostride, int64_t orow0, unsigned char* smem_raw) {
  constexpr int IFC = sweep_x_ifc<P, TH>(), TILE = sweep_x_tile<P, TH>(), CELLS = sweep_x_cells<P, TH>();
  T* su = reinterpret_cast<T*>(smem_raw);   // [NV][CELLS]
  T* sf = su + NV * CELLS;                  // [NV][IFC]
  T* sn = sf + NV * IFC;                    // [NV][TILE] u^n (P > 1)
  T dt = T(0);
  if (A.dt) {
    if (A.dt->zero) return;  // the run has reached t_end: the step changes nothing
    dt = (sizeof(T) == 4) ? T(A.dt->dt32) : T(A.dt->dt);
  }
  const int64_t c0 = tile * TILE;
  const int ntile = (int)min((int64_t)TILE, A.nx - c0);
  const T* base = A.u + row * A.pitch;
  const bool use_un = MODE == kStage && A.a != T(0);
  // u^n of the output cells, loaded now so the latency hides under the sweep: in
  // registers for one cell per thread, staged in shared memory otherwise
  T unv[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) unv[k] = T(0);
  if (P == 1 && use_un && (int)threadIdx.x < ntile) {
#pragma unroll
    for (int k = 0; k < NV; ++k) unv[k] = A.un[k * A.fstride + row * A.pitch + c0 + threadIdx.x];
  }
  if (P > 1 && use_un) {
    for (int s = threadIdx.x; s < ntile; s += TH)
#pragma unroll
      for (int v = 0; v < NV; ++v) sn[v * TILE + s] = A.un[v * A.fstride + row * A.pitch + c0 + s];
  }
  // stage cells c0-5 .. c0+ntile+4 (ntile + 10 <= CELLS), one cell index per thread
  // and pass, all variables of it
  if (!A.f.active) {
    for (int s = threadIdx.x; s < ntile + 10; s += TH) {
      const int64_t gi = ghost(c0 - 5 + s, A.nx, A.bc);
#pragma unroll
      for (int v = 0; v < NV; ++v) su[v * CELLS + s] = base[v * A.fstride + gi];
    }
  } else {
    const double tf = sweep_time(A);
    for (int s = threadIdx.x; s < ntile + 10; s += TH)
      for (int v = 0; v < NV; ++v)
        su[v * CELLS + s] = face_cell<T>(A.u, A.pitch, A.fstride, 0, row, c0 - 5 + s, A.nx, A.bc, v, A.f, tf);
  }
  __syncthreads();
#pragma unroll 1
  for (int q = 0; q < P; ++q) {
    const int t = threadIdx.x + TH * q;
    bool fb = false;
    if (t < ntile + 5) {
      T S[6][NV];
#pragma unroll
      for (int m = 0; m < 6; ++m)
#pragma unroll
        for (int k = 0; k < NV; ++k) S[m][k] = su[k * CELLS + t + m];
      T F[NV];
      if constexpr (sizeof(T) == 4 && NV > 1) {
        fb = pk::interface_flux_pair<NV, FIX>(S, A.s, 0, F);
      } else {
        fb = interface_flux<T, NV, FIX>(S, A.s, 0, F);
      }
#pragma unroll
      for (int k = 0; k < NV; ++k) sf[k * IFC + t] = F[k];
      // each interface of the line is counted by exactly one tile
      const bool owned = (c0 + TILE >= A.nx) ? true : (t < TILE);
      fb = fb && owned;
    }
    count_fallbacks(fb, A.fallbacks);
  }
  __syncthreads();
#pragma unroll 1
  for (int q = 0; q < P; ++q) {
    const int t = threadIdx.x + TH * q;
    if (t >= ntile) break;
    const int64_t off = row * A.pitch + c0 + t;
    T* ob = out + (row - orow0) * A.pitch + c0 + t;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const T* f = sf + k * IFC + t;
      T L = flux_difference_family<T>(WCNS_OPT(FIX, A.s, family), f[0], f[1], f[2], f[3], f[4], f[5], A.inv_h);
      if (MODE == kWriteL) {
        ob[k * ostride] = L;
      } else {
        const T cur = su[k * CELLS + t + 5];
        // u^n is staged only when it enters (a != 0); the general form multiplies by a
        const T unk = (P == 1) ? unv[k] : (use_un ? sn[k * TILE + t] : T(0));
        T v;
        if constexpr (sizeof(T) == 4) {
          if (!A.general) {
            v = smul<T>(A.b, sfma<T>(dt, L, cur));
            if (A.a != T(0)) v = sfma<T>(A.a, unk, v);
          } else {
            v = sfma<T>(smul<T>(A.e, dt), L, sfma<T>(A.a, unk, smul<T>(A.b, cur)));
            if (A.X1) v = sfma<T>(A.c1, A.X1[k * A.fstride + off], v);
            if (A.X2) v = sfma<T>(A.c2, A.X2[k * A.fstride + off], v);
          }
        } else {
          if (!A.general) {
            v = A.b * (cur + dt * L);
            if (A.a != T(0)) v = A.a * unk + v;
          } else {
            v = A.a * unk + A.b * cur + (A.e * dt) * L;
            if (A.X1) v = v + A.c1 * A.X1[k * A.fstride + off];
            if (A.X2) v = v + A.c2 * A.X2[k * A.fstride + off];
          }
        }
        ob[k * ostride] = v;
      }
    }
  }
}

template <typename T, int NV, int MODE, int FIX, int P, int TH = kXThreads>
__global__ void __launch_bounds__(TH, sweep_min_blocks<T>()) sweep_x_kernel(SweepArgs<T> A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int64_t row = A.row_major ? blockIdx.x : blockIdx.y;
  const int64_t tile = A.row_major ? blockIdx.y : blockIdx.x;
  sweep_x_body<T, NV, MODE, FIX, P, TH>(A, row, tile, A.out, A.fstride, 0, smem_raw);
}

// ---------------------------------------------------------------------------
// y sweep: one block per (kYCols columns, kYTile rows); kYCols x kYRowsT threads, each
// computing kYPer interfaces of its column.  Stage: out = R + b*dt*L_y with R the
// partial stage of the x sweep; RHS: out = R + L_y with R = L_x.
// ---------------------------------------------------------------------------
// 16 columns x 16 thread rows: a tall tile keeps the 5-row halo small (80 interfaces
// for 75 output rows) at the same 256 threads and 42 KB of FP32 staging per block;
// measured against 32 x 8 x 6, 16 x 16 x 6 and 8 x 32 x 6 at 2048^2.
constexpr int kYCols = 16;
constexpr int kYRowsT = 16;                // thread rows
constexpr int kYPer = 5;                   // interfaces per thread
constexpr int kYIfc = kYRowsT * kYPer;     // 80 interfaces per column
constexpr int kYTile = kYIfc - 5;          // 75 output rows per block
constexpr int kYCells = kYIfc + 5;         // 85 staged rows

template <typename T, int NV>
constexpr size_t sweep_y_smem() { return sizeof(T) * NV * (kYCells + kYIfc) * kYCols; }

// One y tile (column block bx, row block by) of the sweep; the block (kYCols x kYRowsT
// threads) calls it together.  R is read at R[k * rstride + (r - rrow0) * pitch + c], with
// loads that bypass L1 (R may have been written by other blocks of the same launch).
// vblock spreads the fused CFL maxima over the slots.
template <typename T, int NV, int MODE, int FIX>
__device__ __forceinline__ void sweep_y_body(const SweepArgs<T>& A, int64_t bx, int64_t by, const T* R,
                                             int64_t rstride, int64_t rrow0, unsigned vblock,
                                             unsigned char* smem_raw) {
  T* su = reinterpret_cast<T*>(smem_raw);   // [NV][kYCells][kYCols]
  T* sf = su + NV * kYCells * kYCols;       // [NV][kYIfc][kYCols]
  T dt = T(0);
  if (A.dt) {
    if (A.dt->zero) return;
    dt = (sizeof(T) == 4) ? T(A.dt->dt32) : T(A.dt->dt);
  }
  const int64_t c0 = bx * kYCols;
  const int64_t r0 = by * kYTile;
  const int ntile = (int)min((int64_t)kYTile, A.ny - r0);
  const int ncol = (int)min((int64_t)kYCols, A.nx - c0);
  // kYCols x kYRowsT threads, in a (kYCols, kYRowsT) block or a flat one of the same size
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int tx = tid % kYCols, ty = tid / kYCols;
  // stage rows r0-5 .. r0+ntile+4 (ntile + 10 <= kYCells) of the block's columns: one
  // bulk tensor copy of the kYCols x kYCells x NV box when every one of its rows lies in
  // the grid (columns beyond nx arrive as zeros and are not used), else one row index per
  // thread row and pass, all variables of it
  const bool tma = A.ytma && !A.f.active && r0 - 5 >= 0 && r0 - 5 + kYCells <= A.ny;
  __shared__ unsigned long long ybar;
  if (tma) {
    // every thread's earlier accesses of this shared memory (a previous tile of the block)
    // precede the copy's writes (generic before async proxy)
    asm volatile("fence.proxy.async.shared::cta;" : : : "memory");
    if (tid == 0) mbar_init(&ybar, 1);
    __syncthreads();
    if (tid == 0)
      tma_load_3d(su, &A.ymap, &ybar, (int)c0, (int)(r0 - 5), 0, (unsigned)(sizeof(T) * NV * kYCells * kYCols));
    if (!mbar_wait(&ybar, 0)) {
      if (A.status) atomicOr(A.status, 2);
      (void)mbar_wait(&ybar, 0);  // the copy may still land: wait (bounded) once more before the tile is used
    }
  } else if (tx < ncol) {
    if (!A.f.active) {
      for (int s = ty; s < ntile + 10; s += kYRowsT) {
        const int64_t gr = ghost(r0 - 5 + s, A.ny, A.bc);
#pragma unroll
        for (int v = 0; v < NV; ++v) su[(v * kYCells + s) * kYCols + tx] = A.u[v * A.fstride + gr * A.pitch + c0 + tx];
      }
    } else {
      const double tf = sweep_time(A);
      for (int s = ty; s < ntile + 10; s += kYRowsT)
        for (int v = 0; v < NV; ++v)
          su[(v * kYCells + s) * kYCols + tx] =
              face_cell<T>(A.u, A.pitch, A.fstride, 1, c0 + tx, r0 - 5 + s, A.ny, A.bc, v, A.f, tf);
    }
  }
  __syncthreads();
  if (tma && tid == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" : : "r"(smem_u32(&ybar)) : "memory");
  // the sweep's normal ordering swaps the two momentum components
  constexpr int p1 = (NV == 4) ? 2 : 1;
  constexpr int p2 = (NV == 4) ? 1 : 2;
  for (int q = 0; q < kYPer; ++q) {
    const int t = ty + kYRowsT * q;
    bool fb = false;
    if (tx < ncol && t < ntile + 5) {
      T S[6][NV];
#pragma unroll
      for (int m = 0; m < 6; ++m) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          const int src = (NV == 4 && k == 1) ? p1 : ((NV == 4 && k == 2) ? p2 : k);
          S[m][k] = su[(src * kYCells + t + m) * kYCols + tx];
        }
      }
      T F[NV];
      if constexpr (sizeof(T) == 4 && NV > 1) {
        fb = pk::interface_flux_pair<NV, FIX>(S, A.s, 1, F);
      } else {
        fb = interface_flux<T, NV, FIX>(S, A.s, 1, F);
      }
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const int dst = (NV == 4 && k == 1) ? p1 : ((NV == 4 && k == 2) ? p2 : k);
        sf[(dst * kYIfc + t) * kYCols + tx] = F[k];
      }
      const bool owned = (r0 + kYTile >= A.ny) ? true : (t < kYTile);
      fb = fb && owned;
    }
    count_fallbacks(fb, A.fallbacks);
  }
  __syncthreads();
  // epilogue: all loads of R first (one latency per block), then the sums
  T rv[kYPer][NV];
#pragma unroll
  for (int q = 0; q < kYPer; ++q) {
    const int t = ty + kYRowsT * q;
    const bool on = tx < ncol && t < ntile;
    const T* rb = R + (r0 + t - rrow0) * A.pitch + c0 + tx;
#pragma unroll
    for (int k = 0; k < NV; ++k) rv[q][k] = on ? __ldcg(rb + k * rstride) : T(0);
  }
  T wmx = T(0), wmy = T(0);
  bool wbad = false;
#pragma unroll
  for (int q = 0; q < kYPer; ++q) {
    const int t = ty + kYRowsT * q;
    if (tx < ncol && t < ntile) {
      const int64_t off = (r0 + t) * A.pitch + c0 + tx;
      T val[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const T* f = sf + (k * kYIfc + t) * kYCols + tx;
        T Ly = flux_difference_family<T>(WCNS_OPT(FIX, A.s, family), f[0], f[kYCols], f[2 * kYCols], f[3 * kYCols], f[4 * kYCols],
                                  f[5 * kYCols], A.inv_h);
        // RHS: R = L_x.  Stage: R = a*un + b*(u + dt*L_x) from the x sweep.
        val[k] = (MODE == kWriteL) ? sadd<T>(rv[q][k], Ly)
                                   : sfma<T>(smul<T>(A.general ? A.e : A.b, dt), Ly, rv[q][k]);
        A.out[k * A.fstride + off] = val[k];
      }
      if constexpr (MODE == kStage && NV == 4) {
        if (A.wave) {
          T wx, wy;
          if (cell_wave<T>(val[0], val[1], val[2], val[3], A.s.gamma, A.s.gm1, wx, wy)) {
            wmx = fmax(wmx, wx);
            wmy = fmax(wmy, wy);
          } else {
            wbad = true;
          }
        }
      }
    }
  }
  if constexpr (MODE == kStage && NV == 4) {
    if (A.wave) warp_wave<T>(wmx, wmy, wbad, vblock, A.wave, A.err);  // the same for every thread of the launch
  }
}

template <typename T, int NV, int MODE, int FIX>
__global__ void __launch_bounds__(kYCols * kYRowsT, sweep_min_blocks<T>())
    sweep_y_kernel(const __grid_constant__ SweepArgs<T> A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  sweep_y_body<T, NV, MODE, FIX>(A, blockIdx.x, blockIdx.y, A.R, A.fstride, 0, blockIdx.y * gridDim.x + blockIdx.x,
                                 smem_raw);
}

// ---------------------------------------------------------------------------
// Block reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kRedThreads = 256;

// One 16-byte load of VW consecutive elements (p 16-byte aligned).
template <typename T, int VW>
__device__ __forceinline__ void load16(const T* p, T (&out)[VW]) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
  } else {
    const double2 v = *reinterpret_cast<const double2*>(p);
    out[0] = v.x; out[1] = v.y;
  }
}

// One 16-byte store of VW consecutive elements (p 16-byte aligned).
template <typename T, int VW>
__device__ __forceinline__ void store16(T* p, const T (&in)[VW]) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(in[0], in[1], in[2], in[3]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(in[0], in[1]);
  }
}

// ---------------------------------------------------------------------------
// CFL step: max over cells of |u_d| + c per direction, then
// dt = cfl / sum_d(max_d / h_d), clipped at t_end; the device time advances.
// The last block to finish (ticket counter) combines the per-block partials.
// ---------------------------------------------------------------------------
struct DtArgs {
  const void* u;
  void* copy;            // if set (nvar > 1): every 16-byte vector read from u is stored here too
  int64_t nx, ny, pitch, fstride;
  int nvar, ndim, system, use_cfl;
  int bpr;               // blocks per row (1: each block takes whole rows)
  double gamma, cfl, hx, hy, fixed_dt, t_end;
  double adv_wave[2];    // |a_d| for advection
  double* partials;      // 2 * gridDim.x
  unsigned int* counter;
  double* dt_out;        // max-wave query (t == nullptr): the two maxima
  StepDt* step;          // step mode: the step the sweeps read
  double* t;
  long long* steps;
  int* err;              // bit 0: non-physical state
  // fused CFL maxima of a step's last stage (kWaveSlots slot pairs): cleared by the CFL
  // kernel, read and cleared by step_from_maxima_kernel (or null)
  unsigned long long* wave;
};

// The step of an RK step from the signal-speed maxima gx, gy (the CFL kernel's last block,
// or the maxima the previous step's last stage reduced): dt = cfl / sum_d(max_d / h_d)
// (or the fixed step), zero once a non-physical state was seen, clipped at t_end; writes
// the step record and advances the device time.  One thread.
__device__ __forceinline__ void finish_step(const DtArgs& A, double gx, double gy) {
  double d;
  if (!A.use_cfl) {
    d = A.fixed_dt;
  } else {
    if (A.nvar == 1) { gx = A.adv_wave[0]; gy = A.adv_wave[1]; }
    double s = gx / A.hx;
    if (A.ndim == 2) s += gy / A.hy;
    d = A.cfl / s;
  }
  if (__ldcg(A.err) & 1) d = 0.0;  // a non-physical state freezes the run (reported at sync)
  double t = *A.t;
  if (A.t_end > 0.0) {
    double rem = A.t_end - t;
    if (d > rem) d = rem;
    if (!(d > 0.0)) d = 0.0;
  }
  A.step->dt = d;
  A.step->t0 = t;
  A.step->dt32 = (float)d;
  A.step->zero = (d == 0.0);
  if (d > 0.0) {
    *A.t = (A.t_end > 0.0 && d == A.t_end - t) ? A.t_end : t + d;
    *A.steps += 1;
  }
}

// Step record of an RK step whose CFL maxima the previous step's last stage merged into
// the slots (the fused epilogue of the y sweep): one block takes their maxima, clears the
// slots for this step's last stage and computes the step.
template <typename T>
__global__ void __launch_bounds__(kWaveSlots) step_from_maxima_kernel(DtArgs A) {
  __shared__ double sx[kWaveSlots / 32], sy[kWaveSlots / 32];
  const int i = threadIdx.x;
  double gx = __longlong_as_double((long long)A.wave[2 * i]);
  double gy = __longlong_as_double((long long)A.wave[2 * i + 1]);
  A.wave[2 * i] = 0ull;
  A.wave[2 * i + 1] = 0ull;
  gx = warp_max(gx);
  gy = warp_max(gy);
  if ((i & 31) == 0) {
    sx[i >> 5] = gx;
    sy[i >> 5] = gy;
  }
  __syncthreads();
  if (i != 0) return;
  for (int w = 0; w < kWaveSlots / 32; ++w) { gx = fmax(gx, sx[w]); gy = fmax(gy, sy[w]); }
  finish_step(A, gx, gy);
}

template <typename T, int NV>
__global__ void __launch_bounds__(kRedThreads) dt_kernel(DtArgs A) {
  __shared__ double smx[kRedThreads / 32], smy[kRedThreads / 32];
  __shared__ int s_last, s_bad;
  const T* u = static_cast<const T*>(A.u);
  // maxima in the state's precision (exact: max never rounds), widened once per thread
  T mxT = T(0), myT = T(0);
  int bad = 0;
  if (NV > 1) {
    const T g = T(A.gamma), gm1 = T(A.gamma - 1.0);
    // 16-byte vectors along the rows (rows start on 128-byte lines, pitch % 32 == 0);
    // a block takes whole rows, or one chunk of one row when rows are few
    constexpr int VW = 16 / (int)sizeof(T);
    const int64_t nvec = (A.nx + VW - 1) / VW;
    int64_t rbeg, rend, vbeg, vend;
    if (A.bpr > 1) {
      rbeg = blockIdx.x / A.bpr;
      rend = rbeg + 1;
      const int64_t per = (nvec + A.bpr - 1) / A.bpr;
      vbeg = (blockIdx.x % A.bpr) * per;
      vend = min(nvec, vbeg + per);
    } else {
      const int64_t rpb = (A.ny + gridDim.x - 1) / gridDim.x;
      rbeg = (int64_t)blockIdx.x * rpb;
      rend = min(A.ny, rbeg + rpb);
      vbeg = 0;
      vend = nvec;
    }
    // two vectors per thread and pass, both loaded before either is evaluated
    for (int64_t r = rbeg; r < rend; ++r) {
      for (int64_t q0 = vbeg + threadIdx.x; q0 < vend; q0 += 2 * kRedThreads) {
        T v[2][NV][VW];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int64_t q = q0 + j * kRedThreads;
          if (q < vend) {
#pragma unroll
            for (int w = 0; w < NV; ++w) load16<T, VW>(u + w * A.fstride + r * A.pitch + q * VW, v[j][w]);
            if (A.copy) {
#pragma unroll
              for (int w = 0; w < NV; ++w)
                store16<T, VW>(static_cast<T*>(A.copy) + w * A.fstride + r * A.pitch + q * VW, v[j][w]);
            }
          }
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int64_t q = q0 + j * kRedThreads;
          if (q >= vend) break;
#pragma unroll
          for (int l = 0; l < VW; ++l) {
            if (q * VW + l >= A.nx) break;
            // wave speeds in the state's own precision
            const T rho = v[j][0][l], mu = v[j][1][l], mv = (NV == 4) ? v[j][2][l] : T(0), E = v[j][NV - 1][l];
            T wx, wy;
            if (!cell_wave<T>(rho, mu, mv, E, g, gm1, wx, wy)) { bad = 1; continue; }
            mxT = fmax(mxT, wx);
            myT = fmax(myT, wy);
          }
        }
      }
    }
  }
  double mx = (double)mxT, my = (double)myT;
  mx = warp_max(mx);
  my = warp_max(my);
  bad = __any_sync(0xffffffffu, bad);
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    smx[threadIdx.x >> 5] = mx;
    smy[threadIdx.x >> 5] = my;
    if (bad) atomicOr(&s_bad, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bx = 0.0, by = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) { bx = fmax(bx, smx[w]); by = fmax(by, smy[w]); }
    A.partials[2 * blockIdx.x] = bx;
    A.partials[2 * blockIdx.x + 1] = by;
    if (s_bad) atomicOr(A.err, 1);
    __threadfence();
    unsigned int ticket = atomicAdd(A.counter, 1u);
    s_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  // the last block combines the per-block maxima with all of its threads
  __threadfence();
  double gx = 0.0, gy = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kRedThreads) {
    gx = fmax(gx, __ldcg(&A.partials[2 * b]));
    gy = fmax(gy, __ldcg(&A.partials[2 * b + 1]));
  }
  gx = warp_max(gx);
  gy = warp_max(gy);
  if ((threadIdx.x & 31) == 0) {
    smx[threadIdx.x >> 5] = gx;
    smy[threadIdx.x >> 5] = gy;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  gx = 0.0;
  gy = 0.0;
  for (int w = 0; w < kRedThreads / 32; ++w) { gx = fmax(gx, smx[w]); gy = fmax(gy, smy[w]); }
  *A.counter = 0u;  // ready for the next launch
  if (A.t == nullptr) {  // max-wave query: report the maxima, leave the time alone
    A.dt_out[0] = gx;
    A.dt_out[1] = gy;
    return;
  }
  if (A.wave)  // this step's last stage merges the next step's maxima from zero
    for (int k = 0; k < 2 * kWaveSlots; ++k) A.wave[k] = 0ull;
  finish_step(A, gx, gy);
}

// ---------------------------------------------------------------------------
// FP64 reductions per variable plane: SUM, L1 (mean |a - b|), LINF (max |a - b|).
// blockIdx.y = variable.  Partials [nvar][gridDim.x]; the last block per variable
// writes out[v].
// ---------------------------------------------------------------------------
struct ReduceArgs {
  const void* a;
  const void* b;   // may be null
  int64_t nx, ny, pitch, fstride;
  int what;        // 0 sum, 1 l1, 2 linf
  double* partials;
  unsigned int* counters;  // one per variable
  double* out;
};

template <typename T>
__global__ void __launch_bounds__(kRedThreads) reduce_kernel(ReduceArgs A) {
  __shared__ double sacc[kRedThreads / 32];
  __shared__ int s_last;
  const T* a = static_cast<const T*>(A.a) + blockIdx.y * A.fstride;
  const T* b = A.b ? static_cast<const T*>(A.b) + blockIdx.y * A.fstride : nullptr;
  const int64_t ncell = A.nx * A.ny;
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * kRedThreads;
  const int64_t c0 = (int64_t)blockIdx.x * kRedThreads + threadIdx.x;
  const int64_t sj = stride / A.nx, si = stride - sj * A.nx;
  int64_t j = c0 / A.nx, i = c0 - j * A.nx;
  for (int64_t c = c0; c < ncell; c += stride) {
    const int64_t off = j * A.pitch + i;
    i += si;
    j += sj;
    if (i >= A.nx) { i -= A.nx; ++j; }
    double x = (double)a[off];
    if (b) x -= (double)b[off];
    if (A.what == 0) acc += x;
    else if (A.what == 1) acc += fabs(x);
    else acc = fmax(acc, fabs(x));
  }
  acc = (A.what == 2) ? warp_max(acc) : warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sacc[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) r = (A.what == 2) ? fmax(r, sacc[w]) : r + sacc[w];
    A.partials[blockIdx.y * gridDim.x + blockIdx.x] = r;
    __threadfence();
    unsigned int ticket = atomicAdd(&A.counters[blockIdx.y], 1u);
    s_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double r = 0.0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += kRedThreads) {
    double p = __ldcg(&A.partials[blockIdx.y * gridDim.x + k]);
    r = (A.what == 2) ? fmax(r, p) : r + p;
  }
  r = (A.what == 2) ? warp_max(r) : warp_sum(r);
  __syncthreads();  // sacc is reused
  if ((threadIdx.x & 31) == 0) sacc[threadIdx.x >> 5] = r;
  __syncthreads();
  if (threadIdx.x != 0) return;
  r = 0.0;
  for (int w = 0; w < kRedThreads / 32; ++w) r = (A.what == 2) ? fmax(r, sacc[w]) : r + sacc[w];
  A.counters[blockIdx.y] = 0u;
  A.out[blockIdx.y] = (A.what == 1) ? r / (double)ncell : r;
}

}  // namespace wcns
