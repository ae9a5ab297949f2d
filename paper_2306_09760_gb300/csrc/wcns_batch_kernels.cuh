// Kernels for many independent 1D Euler problems in one concatenated buffer.
//
// Problem k owns columns off_k .. off_k + n_k - 1 of each of the three variable planes
// (plane stride `total`).  Each RK3 stage is one persistent launch: every block claims
// (problem, tile) work items from a list sorted by problem size (largest first) with
// an atomic ticket, so uneven problems balance across the SMs without any waiting.
// Every problem advances with its own CFL step dt_k = cfl * h_k / max(|u| + c).
#pragma once

#include "wcns_kernels.cuh"

namespace wcns {

struct BatchItem {
  int prob;
  int c0;  // first cell of the tile
};

template <typename T>
struct BatchStageArgs {
  const T* u;        // state the RHS is evaluated on
  const T* un;       // u^n (when a != 0)
  T* out;
  const int64_t* off;
  const int* n;
  const double* inv_h;
  const StepDt* dt;  // per problem
  const BatchItem* items;
  int nitems;
  unsigned int* ticket;
  int64_t total;
  int bc;
  T a, b;
  SchemeT<T> s;
  unsigned long long* fallbacks;
};

// Persistent stage kernel; NT threads = NT - 5 output cells per work item.
template <typename T, int NT, int FIX>
__global__ void __launch_bounds__(NT) batch_stage_kernel(BatchStageArgs<T> A) {
  constexpr int NV = 3;
  constexpr int TILE = NT - 5;
  constexpr int CELLS = NT + 5;
  __shared__ T su[NV][CELLS];
  __shared__ T sf[NV][NT];
  __shared__ int s_item;
  const int t = threadIdx.x;
  for (;;) {
    if (t == 0) s_item = (int)atomicAdd(A.ticket, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= A.nitems) break;
    const BatchItem item = A.items[it];
    const StepDt& step = A.dt[item.prob];
    if (!step.zero) {
      const int n = A.n[item.prob];
      const int64_t off = A.off[item.prob];
      const int c0 = item.c0;
      const int ntile = min(TILE, n - c0);
      for (int s = t; s < ntile + 10; s += NT) {
        const int64_t gi = off + ghost(c0 - 5 + s, n, A.bc);
#pragma unroll
        for (int v = 0; v < NV; ++v) su[v][s] = A.u[v * A.total + gi];
      }
      __syncthreads();
      bool fb = false;
      if (t < ntile + 5) {
        T S[6][NV];
#pragma unroll
        for (int m = 0; m < 6; ++m)
#pragma unroll
          for (int k = 0; k < NV; ++k) S[m][k] = su[k][t + m];
        T F[NV];
        if constexpr (sizeof(T) == 4 && NV > 1) {
          fb = pk::interface_flux_pair<NV, FIX>(S, A.s, 0, F);
        } else {
          fb = interface_flux<T, NV, FIX>(S, A.s, 0, F);
        }
#pragma unroll
        for (int k = 0; k < NV; ++k) sf[k][t] = F[k];
        const bool last = (c0 + TILE >= n);
        fb = fb && (last || t < TILE);
      }
      count_fallbacks(fb, A.fallbacks);
      __syncthreads();
      if (t < ntile) {
        const T dt = (sizeof(T) == 4) ? T(step.dt32) : T(step.dt);
        const T inv_h = T(A.inv_h[item.prob]);
        const int64_t o = off + c0 + t;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          const T* f = &sf[k][t];
          T L = flux_difference_family<T>(WCNS_OPT(FIX, A.s, family), f[0], f[1], f[2], f[3], f[4], f[5], inv_h);
          T v = A.b * (su[k][t + 5] + dt * L);
          if (A.a != T(0)) v = A.a * A.un[k * A.total + o] + v;
          A.out[k * A.total + o] = v;
        }
      }
    }
    __syncthreads();  // the next item reuses the shared tiles and s_item
  }
}

// Per-problem CFL step: one block per problem.  dt_k = cfl h_k / max(|u| + c), clipped so
// that t_k never passes t_end; with `advance` the problem time moves on.  A non-physical
// cell sets the error flag and freezes that problem (dt_k = 0).
struct BatchDtArgs {
  const void* u;
  const int64_t* off;
  const int* n;
  const double* h;
  StepDt* dt;
  double* t;
  long long* steps;
  int64_t total;
  double gamma, cfl, t_end;
  int advance;
  int* err;
};

template <typename T>
__global__ void __launch_bounds__(256) batch_dt_kernel(BatchDtArgs A) {
  __shared__ double sm[8];
  __shared__ int sbad;
  const T* u = static_cast<const T*>(A.u);
  const int k = blockIdx.x;
  const int n = A.n[k];
  const int64_t off = A.off[k];
  // the maximum in the state's precision (exact), widened once per thread
  T mxT = T(0);
  int bad = 0;
  const T gam = T(A.gamma), gm1 = T(A.gamma - 1.0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const T rho = u[off + i];
    const T m = u[A.total + off + i];
    const T E = u[2 * A.total + off + i];
    const T inv = T(1) / rho;
    const T vel = m * inv;
    const T p = gm1 * (E - T(0.5) * rho * vel * vel);
    if (!(rho > T(0)) || !(p > T(0))) { bad = 1; continue; }
    mxT = fmax(mxT, Num<T>::abs_(vel) + Num<T>::sqrt_(gam * p * inv));
  }
  double mx = (double)mxT;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  bad = __any_sync(0xffffffffu, bad);
  if (threadIdx.x == 0) sbad = 0;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    sm[threadIdx.x >> 5] = mx;
    if (bad) atomicOr(&sbad, 1);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double g = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) g = fmax(g, sm[w]);
  double d = A.cfl * A.h[k] / g;
  if (sbad) {
    atomicOr(A.err, 1);
    d = 0.0;
  }
  double t = A.t[k];
  if (A.t_end > 0.0) {
    double rem = A.t_end - t;
    if (d > rem) d = rem;
    if (!(d > 0.0)) d = 0.0;
  }
  A.dt[k].dt = d;
  A.dt[k].dt32 = (float)d;
  A.dt[k].zero = (d == 0.0);
  if (A.advance && d > 0.0) {
    A.t[k] = (A.t_end > 0.0 && d == A.t_end - t) ? A.t_end : t + d;
    A.steps[k] += 1;
  }
}

}  // namespace wcns
