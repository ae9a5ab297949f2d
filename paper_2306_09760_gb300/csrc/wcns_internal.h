// Internal host-side interface between the C-ABI layer and the per-type kernel
// translation units.  Not installed; not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "wcns_device.cuh"

namespace wcns {

struct GridInfo {
  int ndim, nvar;
  int64_t nx, ny, pitch;
  int bc[2];
  double h[2];
};

// Raises the dynamic shared-memory limit of every sweep kernel for `nvar` (call once
// per device before the first launch and before any stream capture).
template <typename T>
cudaError_t configure_kernels(int nvar);

// One sweep kernel.  x sweep: 1D stage (out = a*un + b*(u + dt*L)) or L / L_x into
// `out` (dt may be null for a plain RHS).  y sweep: L = R + L_y, then either L into
// `out` (dt null) or the stage update.
template <typename T>
struct SweepCall {
  const T* u;
  const T* un;
  const T* R;
  T* out;
  const StepDt* dt;
  double a, b;
  bool stage;  // apply the RK stage update (else write L)
  unsigned long long* fallbacks;
  // general stage form out = a*un + b*u + e*dt*L + c1*X1 + c2*X2 (RK4); else TVD-RK3 form
  bool general;
  double e, c1, c2;
  const T* X1;
  const T* X2;
  const Faces<double>* faces;  // boundary faces (active == 0: the grid's bc only)
  double cstage;               // the state read is at t0 + cstage * dt of the step
  const double* tnow;          // device time (RHS evaluations)
  // y sweep of a 2D Euler stage that completes an RK step: CFL maxima of the written
  // state merged into the slots of wave (kWaveSlots pairs) and non-physical cells
  // flagged in *err (else null)
  unsigned long long* wave;
  int* err;
  int* status;  // sticky error word for bounded waits (always set)
};
template <typename T>
cudaError_t launch_sweep_x(const GridInfo& g, const Scheme& s, const SweepCall<T>& c, cudaStream_t st);
template <typename T>
cudaError_t launch_sweep_y(const GridInfo& g, const Scheme& s, const SweepCall<T>& c, cudaStream_t st);

// One 2D Euler stage (the x and y sweep calls of a stage) as a single banded persistent
// launch whose partial stage lives in a ring of band-sized slots (wcns_band.cuh).
// band_applies: whether the banded form can run this grid and scheme; ring bytes from
// band_ring_bytes_of; ctr: kBandCounterWords zeroed words.
template <typename T>
bool band_applies(const GridInfo& g, const Scheme& s);
template <typename T>
cudaError_t launch_stage_band(const GridInfo& g, const Scheme& s, const SweepCall<T>& x, const SweepCall<T>& y,
                              T* ring, unsigned* ctr, int* err, cudaStream_t st);
size_t band_ring_bytes_of(const GridInfo& g, size_t elem);
// One-thread kernel whose two bounded waits (a completion counter that nothing
// increments, an mbarrier that no copy fills) must both give up: gave_up[0..1] (device)
// receive 1 when they did; each sets bit 1 of *err.  `never` must stay 0.
cudaError_t launch_wait_selftest(const unsigned* never, int* err, int* gave_up, cudaStream_t st);
constexpr int kBandCounterWords = 2 + 2 * 64;

// Adjoint sweep: out = c1*X1 + c2*X2 + b*(mu + dt*(R + J^T mu)) (combine) or
// out = J^T mu (x part of a 2D grid, combine == false).
template <typename T>
struct AdjCall {
  const T* u;
  const T* mu;
  const T* R;
  const T* X1;
  const T* X2;
  T* out;
  double c1, c2, b, dt;
  bool combine;
};
template <typename T>
cudaError_t launch_adjoint_x(const GridInfo& g, const Scheme& s, const AdjCall<T>& c, cudaStream_t st);
template <typename T>
cudaError_t launch_adjoint_y(const GridInfo& g, const Scheme& s, const AdjCall<T>& c, cudaStream_t st);

struct DtLaunch {
  const void* u;
  void* copy;  // optional: the CFL kernel also copies u here (same layout)
  double cfl, fixed_dt, t_end;
  int use_cfl;
  double adv_wave[2];
  double gamma;
  double* partials;
  int max_blocks;
  unsigned int* counter;
  double* dt_out;
  StepDt* step;
  double* t;
  long long* steps;
  int* err;
  unsigned long long* wave;  // fused CFL maxima slots of a step's last stage (2 * kWaveSlots), or null
};
template <typename T>
cudaError_t launch_dt(const GridInfo& g, const DtLaunch& d, cudaStream_t st);
// The step record from the maxima in d.wave (reduced by the previous step's last stage).
template <typename T>
cudaError_t launch_step_from_maxima(const GridInfo& g, const DtLaunch& d, cudaStream_t st);

// App. A weight statistics of one evaluation of L(u), accumulated into
// hist[2][3][nbins] (device, 64-bit counters).
template <typename T>
cudaError_t launch_weight_hist(const GridInfo& g, const Scheme& s, const Faces<double>& f, const double* tnow,
                               const void* u, int nbins, unsigned long long* hist, cudaStream_t st);

template <typename T>
cudaError_t launch_reduce(const GridInfo& g, const void* a, const void* b, int what, double* partials,
                          int max_blocks, unsigned int* counters, double* out, cudaStream_t st);

// Number of blocks the reductions use at most (partials are sized for this).
constexpr int kMaxRedBlocks = 152 * 8;

}  // namespace wcns
