// Launchers for one element type T; included once per type by wcns_f32.cu / wcns_f64.cu.
#pragma once

#include "wcns_internal.h"
#include "wcns_kernels.cuh"

namespace wcns {

template <typename T, int NV, int MODE>
static cudaError_t run_sweep_x(const GridInfo& g, const SweepArgs<T>& A, cudaStream_t st) {
  const size_t smem = sweep_x_smem<T, NV>();
  dim3 grid((unsigned)((g.nx + kXTile - 1) / kXTile), (unsigned)g.ny);
  sweep_x_kernel<T, NV, MODE><<<grid, kXThreads, smem, st>>>(A);
  return cudaGetLastError();
}

template <typename T, int NV, int MODE>
static cudaError_t run_sweep_y(const GridInfo& g, const SweepArgs<T>& A, cudaStream_t st) {
  const size_t smem = sweep_y_smem<T, NV>();
  dim3 grid((unsigned)((g.nx + kYCols - 1) / kYCols), (unsigned)((g.ny + kYTile - 1) / kYTile));
  dim3 block(kYCols, kYRowsT);
  sweep_y_kernel<T, NV, MODE><<<grid, block, smem, st>>>(A);
  return cudaGetLastError();
}

template <typename T>
static SweepArgs<T> make_args(const GridInfo& g, const Scheme& s, int dir, const SweepCall<T>& c) {
  SweepArgs<T> A{};
  A.nx = g.nx; A.ny = g.ny; A.pitch = g.pitch; A.fstride = g.ny * g.pitch;
  A.bc = g.bc[dir];
  A.inv_h = T(1.0 / g.h[dir]);
  A.s = s;
  A.fallbacks = c.fallbacks;
  A.u = c.u; A.un = c.un; A.R = c.R; A.out = c.out; A.dt = c.dt;
  A.a = T(c.a); A.b = T(c.b);
  return A;
}

template <typename T, int NV>
static cudaError_t configure_nv() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(sweep_x_kernel<T, NV, kWriteL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sweep_x_smem<T, NV>())) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(sweep_x_kernel<T, NV, kStage>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sweep_x_smem<T, NV>())) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(sweep_y_kernel<T, NV, kWriteL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sweep_y_smem<T, NV>())) != cudaSuccess) return e;
  return cudaFuncSetAttribute(sweep_y_kernel<T, NV, kStage>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sweep_y_smem<T, NV>());
}

template <typename T>
cudaError_t configure_kernels(int nvar) {
  switch (nvar) {
    case 1: return configure_nv<T, 1>();
    case 3: return configure_nv<T, 3>();
    case 4: return configure_nv<T, 4>();
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_sweep_x(const GridInfo& g, const Scheme& s, const SweepCall<T>& c, cudaStream_t st) {
  SweepArgs<T> A = make_args<T>(g, s, 0, c);
  switch (g.nvar) {
    case 1: return c.stage ? run_sweep_x<T, 1, kStage>(g, A, st) : run_sweep_x<T, 1, kWriteL>(g, A, st);
    case 3: return c.stage ? run_sweep_x<T, 3, kStage>(g, A, st) : run_sweep_x<T, 3, kWriteL>(g, A, st);
    case 4: return c.stage ? run_sweep_x<T, 4, kStage>(g, A, st) : run_sweep_x<T, 4, kWriteL>(g, A, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_sweep_y(const GridInfo& g, const Scheme& s, const SweepCall<T>& c, cudaStream_t st) {
  SweepArgs<T> A = make_args<T>(g, s, 1, c);
  switch (g.nvar) {
    case 1: return c.stage ? run_sweep_y<T, 1, kStage>(g, A, st) : run_sweep_y<T, 1, kWriteL>(g, A, st);
    case 4: return c.stage ? run_sweep_y<T, 4, kStage>(g, A, st) : run_sweep_y<T, 4, kWriteL>(g, A, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_dt(const GridInfo& g, const DtLaunch& d, cudaStream_t st) {
  DtArgs A{};
  A.u = d.u; A.nx = g.nx; A.ny = g.ny; A.pitch = g.pitch; A.fstride = g.ny * g.pitch;
  A.nvar = g.nvar; A.ndim = g.ndim; A.use_cfl = d.use_cfl;
  A.gamma = d.gamma; A.cfl = d.cfl; A.hx = g.h[0]; A.hy = g.h[1];
  A.fixed_dt = d.fixed_dt; A.t_end = d.t_end;
  A.adv_wave[0] = d.adv_wave[0]; A.adv_wave[1] = d.adv_wave[1];
  A.partials = d.partials; A.counter = d.counter; A.dt_out = d.dt_out; A.t = d.t;
  A.steps = d.steps; A.err = d.err;
  const int64_t ncell = g.nx * g.ny;
  int blocks = 1;
  if (g.nvar > 1) {
    int64_t want = (ncell + kRedThreads * 4 - 1) / (kRedThreads * 4);
    blocks = (int)(want < 1 ? 1 : (want > d.max_blocks ? d.max_blocks : want));
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

#define WCNS_INSTANTIATE(T)                                                                          \
  namespace wcns {                                                                                   \
  template cudaError_t configure_kernels<T>(int);                                                    \
  template cudaError_t launch_sweep_x<T>(const GridInfo&, const Scheme&, const SweepCall<T>&,       \
                                         cudaStream_t);                                              \
  template cudaError_t launch_sweep_y<T>(const GridInfo&, const Scheme&, const SweepCall<T>&,       \
                                         cudaStream_t);                                              \
  template cudaError_t launch_dt<T>(const GridInfo&, const DtLaunch&, cudaStream_t);                 \
  template cudaError_t launch_reduce<T>(const GridInfo&, const void*, const void*, int, double*, int, \
                                        unsigned int*, double*, cudaStream_t);                       \
  }
