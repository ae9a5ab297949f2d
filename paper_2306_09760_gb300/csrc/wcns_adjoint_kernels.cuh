// Adjoint sweeps: out = (dL/du)^T mu for one direction, in gather form (no atomics).
//
// L_i = -(1/h) sum_m d_m (F_{i+m-1/2} - F_{i-m+1/2}) (Eq. 3), so the cotangent of the
// flux at interface k+1/2 is phi_k = (1/h) sum_m d_m (mu_{k+m} - mu_{k+1-m}), where mu
// is the cotangent of L.  Each interface's reverse sweep gives six stencil-cell
// cotangents; a tile stages them in shared memory and every output cell sums the six
// entries that belong to it.  Boundaries: periodic lines treat interface and cell
// indices modulo n; transmissive lines use mu = 0 outside the grid and fold the
// cotangents of ghost cells into the boundary cell they copy.
#pragma once

#include "wcns_adjoint.cuh"
#include "wcns_kernels.cuh"

namespace wcns {

template <typename T>
struct AdjArgs {
  const T* u;    // state at which the Jacobian is taken
  const T* mu;   // cotangent of L
  const T* R;    // x-sweep result (y sweep of a 2D grid) or null
  const T* X1;   // optional pointwise terms of the combination
  const T* X2;
  T* out;
  T c1, c2, b, dt;
  int64_t nx, ny, pitch, fstride;
  int bc;
  T inv_h;
  SchemeT<T> s;
};

enum AdjMode { kAdjWrite = 0, kAdjCombine = 1 };

// out = c1 X1 + c2 X2 + b (mu + dt (R + J^T mu))   (kAdjCombine)
// out = J^T mu                                      (kAdjWrite)
template <typename T>
WCNS_HD T adj_combine(const AdjArgs<T>& A, int64_t off, int k, T jt, T mu) {
  T v = A.b * (mu + A.dt * jt);
  if (A.X1) v = A.c1 * A.X1[k * A.fstride + off] + v;
  if (A.X2) v = A.c2 * A.X2[k * A.fstride + off] + v;
  return v;
}

template <typename T, int NV>
constexpr size_t adj_x_smem() { return sizeof(T) * NV * (2 * kXCells + 6 * kXThreads); }

// The x adjoint covers the forward tile (kXThreads interfaces, kXTile cells) with
// kAXThreads threads, two interfaces each: on the 512^2 adjoint workload 128-thread
// blocks ran 0.171 ms per launch against 0.214 for 256 threads with one interface each
// (the block waits on its slowest warp's reverse sweep at the barrier) and 0.275 for 64
// threads with four each.  Single precision asks for six resident blocks (at most 80
// registers; a few spills): 0.150 ms against 0.173 at four.
constexpr int kAXThreads = 128;
template <typename T>
constexpr int adj_x_min_blocks() { return sizeof(T) == 4 ? 6 : 1; }

template <typename T, int NV, int MODE>
__global__ void __launch_bounds__(kAXThreads, adj_x_min_blocks<T>()) adjoint_x_kernel(AdjArgs<T> A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* su = reinterpret_cast<T*>(smem_raw);   // [NV][kXCells]
  T* sm = su + NV * kXCells;                // [NV][kXCells] mu
  T* sc = sm + NV * kXCells;                // [NV][6][kXThreads] per-interface stencil cotangents
  const int64_t row = blockIdx.y;
  const int64_t c0 = (int64_t)blockIdx.x * kXTile;
  const int ntile = (int)min((int64_t)kXTile, A.nx - c0);
  const int64_t n = A.nx;
  const T* ub = A.u + row * A.pitch;
  const T* mb = A.mu + row * A.pitch;
  for (int idx = threadIdx.x; idx < NV * kXCells; idx += kAXThreads) {
    const int v = idx / kXCells, s = idx - v * kXCells;
    if (s < ntile + 10) {
      const int64_t i = c0 - 5 + s;
      su[idx] = ub[v * A.fstride + ghost(i, n, A.bc)];
      const bool inside = (i >= 0 && i < n);
      sm[idx] = (A.bc == 0 || inside) ? mb[v * A.fstride + ghost(i, n, A.bc)] : T(0);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < ntile + 5; t += kAXThreads) {
    T S[6][NV], Sb[6][NV], phi[NV];
#pragma unroll
    for (int m = 0; m < 6; ++m)
#pragma unroll
      for (int k = 0; k < NV; ++k) { S[m][k] = su[k * kXCells + t + m]; Sb[m][k] = T(0); }
    const T d1 = T(75.0 / 64.0), d2 = T(-25.0 / 384.0), d3 = T(3.0 / 640.0);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const T* q = sm + k * kXCells + t;  // q[j] = mu at cell (interface k) - 2 + j
      phi[k] = A.inv_h * (d1 * (q[3] - q[2]) + d2 * (q[4] - q[1]) + d3 * (q[5] - q[0]));
    }
    interface_flux_vjp<T, NV>(S, A.s, 0, phi, Sb);
#pragma unroll
    for (int m = 0; m < 6; ++m)
#pragma unroll
      for (int k = 0; k < NV; ++k) sc[(k * 6 + m) * kXThreads + t] = Sb[m][k];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < ntile; t += kAXThreads) {
    const int64_t c = c0 + t;
    const int64_t off = row * A.pitch + c;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      T acc = T(0);
#pragma unroll
      for (int j = 0; j < 6; ++j) acc = acc + sc[(k * 6 + (5 - j)) * kXThreads + t + j];
      if (A.bc != 0) {
        // transmissive: ghost cells copy the boundary cell, so their cotangents land there
        if (c == 0) {
          for (int tk = 0; tk < 5; ++tk)        // interfaces k = -3 .. 1
            for (int m = 0; m < 6; ++m)
              if (tk - 5 + m < 0) acc = acc + sc[(k * 6 + m) * kXThreads + tk];
        }
        if (c == n - 1) {
          for (int tk = ntile; tk < ntile + 5; ++tk)  // interfaces k = n-3 .. n+1
            for (int m = 0; m < 6; ++m)
              if (c0 + tk - 5 + m > n - 1) acc = acc + sc[(k * 6 + m) * kXThreads + tk];
        }
      }
      if (MODE == kAdjWrite) {
        A.out[k * A.fstride + off] = acc;
      } else {
        const T mu_c = sm[k * kXCells + t + 5];
        A.out[k * A.fstride + off] = adj_combine<T>(A, off, k, acc, mu_c);
      }
    }
  }
}

// The y adjoint stages six cotangents per interface, so its tile is smaller than the
// forward one: 16 columns x 32 interfaces (27 output rows), 16 x 16 threads.
constexpr int kAYCols = 16;
constexpr int kAYRowsT = 16;
constexpr int kAYPer = 2;
constexpr int kAYIfc = kAYRowsT * kAYPer;  // 32
constexpr int kAYTile = kAYIfc - 5;        // 27
constexpr int kAYCells = kAYIfc + 5;       // 37

template <typename T, int NV>
constexpr size_t adj_y_smem() { return sizeof(T) * NV * (2 * kAYCells + 6 * kAYIfc) * kAYCols; }

// Single precision keeps two 256-thread blocks resident per SM (at most 128 registers);
// double precision keeps the compiler's choice (a cap would spill).
template <typename T>
constexpr int adj_y_min_blocks() { return sizeof(T) == 4 ? 2 : 1; }

template <typename T, int NV>
__global__ void __launch_bounds__(kAYCols * kAYRowsT, adj_y_min_blocks<T>()) adjoint_y_kernel(AdjArgs<T> A) {
  constexpr int kYCols = kAYCols, kYRowsT = kAYRowsT, kYPer = kAYPer, kYIfc = kAYIfc, kYTile = kAYTile,
                kYCells = kAYCells;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* su = reinterpret_cast<T*>(smem_raw);     // [NV][kYCells][kYCols]
  T* sm = su + NV * kYCells * kYCols;         // [NV][kYCells][kYCols]
  T* sc = sm + NV * kYCells * kYCols;         // [NV][6][kYIfc][kYCols]
  const int64_t c0 = (int64_t)blockIdx.x * kYCols;
  const int64_t r0 = (int64_t)blockIdx.y * kYTile;
  const int ntile = (int)min((int64_t)kYTile, A.ny - r0);
  const int ncol = (int)min((int64_t)kYCols, A.nx - c0);
  const int64_t n = A.ny;
  const int tid = threadIdx.y * kYCols + threadIdx.x;
  for (int idx = tid; idx < NV * kYCells * kYCols; idx += kYCols * kYRowsT) {
    const int x = idx % kYCols;
    const int rest = idx / kYCols;
    const int s = rest % kYCells, v = rest / kYCells;
    if (x < ncol && s < ntile + 10) {
      const int64_t j = r0 - 5 + s;
      const int64_t off = v * A.fstride + ghost(j, n, A.bc) * A.pitch + c0 + x;
      su[idx] = A.u[off];
      const bool inside = (j >= 0 && j < n);
      sm[idx] = (A.bc == 0 || inside) ? A.mu[off] : T(0);
    }
  }
  __syncthreads();
  const int tx = threadIdx.x;
  constexpr int p1 = (NV == 4) ? 2 : 1;
  constexpr int p2 = (NV == 4) ? 1 : 2;
  if (tx < ncol) {
    for (int q = 0; q < kYPer; ++q) {
      const int t = threadIdx.y + kYRowsT * q;
      if (t >= ntile + 5) break;
      T S[6][NV], Sb[6][NV], phi[NV];
#pragma unroll
      for (int m = 0; m < 6; ++m)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          const int src = (NV == 4 && k == 1) ? p1 : ((NV == 4 && k == 2) ? p2 : k);
          S[m][k] = su[(src * kYCells + t + m) * kYCols + tx];
          Sb[m][k] = T(0);
        }
      const T d1 = T(75.0 / 64.0), d2 = T(-25.0 / 384.0), d3 = T(3.0 / 640.0);
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const int src = (NV == 4 && k == 1) ? p1 : ((NV == 4 && k == 2) ? p2 : k);
        const T* qv = sm + (src * kYCells + t) * kYCols + tx;
        phi[k] = A.inv_h * (d1 * (qv[3 * kYCols] - qv[2 * kYCols]) + d2 * (qv[4 * kYCols] - qv[kYCols]) +
                            d3 * (qv[5 * kYCols] - qv[0]));
      }
      interface_flux_vjp<T, NV>(S, A.s, 1, phi, Sb);
#pragma unroll
      for (int m = 0; m < 6; ++m)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          const int dst = (NV == 4 && k == 1) ? p1 : ((NV == 4 && k == 2) ? p2 : k);
          sc[((dst * 6 + m) * kYIfc + t) * kYCols + tx] = Sb[m][k];
        }
    }
  }
  __syncthreads();
  if (tx < ncol) {
    for (int q = 0; q < kYPer; ++q) {
      const int t = threadIdx.y + kYRowsT * q;
      if (t >= ntile) break;
      const int64_t c = r0 + t;
      const int64_t off = c * A.pitch + c0 + tx;
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        T acc = T(0);
#pragma unroll
        for (int j = 0; j < 6; ++j) acc = acc + sc[((k * 6 + (5 - j)) * kYIfc + t + j) * kYCols + tx];
        if (A.bc != 0) {
          if (c == 0) {
            for (int tk = 0; tk < 5; ++tk)
              for (int m = 0; m < 6; ++m)
                if (tk - 5 + m < 0) acc = acc + sc[((k * 6 + m) * kYIfc + tk) * kYCols + tx];
          }
          if (c == n - 1) {
            for (int tk = ntile; tk < ntile + 5; ++tk)
              for (int m = 0; m < 6; ++m)
                if (r0 + tk - 5 + m > n - 1) acc = acc + sc[((k * 6 + m) * kYIfc + tk) * kYCols + tx];
          }
        }
        if (A.R) acc = acc + A.R[k * A.fstride + off];
        const T mu_c = sm[(k * kYCells + t + 5) * kYCols + tx];
        A.out[k * A.fstride + off] = adj_combine<T>(A, off, k, acc, mu_c);
      }
    }
  }
}

}  // namespace wcns
