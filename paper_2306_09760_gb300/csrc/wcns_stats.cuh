// Weight statistics of App. A: histograms of the base (Z, or JS) weights and of the
// final weights (FE / PFE / M mapped, renormalised, or kept) of every one-sided
// interpolation of one evaluation of L(u).  One thread per interface; the stencil is
// read straight from global memory and the interface flux is evaluated with a weight
// recorder, so the weights are those of the same arithmetic as the sweeps (the generic
// per-interface path).  Interfaces per line: k + 1/2 for k = -3 .. n + 1 (the six
// fluxes each cell's Eq. 3 difference uses, with the halo), or k = -1 .. n - 1 for the
// WENO family's two-point difference; periodic lines count their wrapped halo
// interfaces again, as the difference uses them.
#pragma once

#include "wcns_device.cuh"

namespace wcns {

template <typename T>
struct HistArgs {
  const T* u;
  int64_t n, lines, pitch, fstride;  // cells along the sweep, lines of the sweep
  int dir, bc;
  int64_t kmin, nk;                  // interfaces kmin .. kmin + nk - 1 of every line
  SchemeT<T> s;
  WeightRecorder rec;
  Faces<T> f;
  const double* tnow;   // device time (moving-shock faces)
};

template <typename T, int NV>
__global__ void __launch_bounds__(256) weight_hist_kernel(HistArgs<T> A) {
  const int64_t idx = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (idx >= A.lines * A.nk) return;
  const int64_t line = idx / A.nk;
  const int64_t k = A.kmin + (idx - line * A.nk);
  const double tf = A.f.active ? *A.tnow : 0.0;
  T S[6][NV];
#pragma unroll
  for (int m = 0; m < 6; ++m) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      // the y sweep's normal ordering swaps the two momentum components
      const int src = (A.dir == 1 && NV == 4 && v == 1) ? 2 : ((A.dir == 1 && NV == 4 && v == 2) ? 1 : v);
      S[m][v] = face_cell<T>(A.u, A.pitch, A.fstride, A.dir, line, k - 2 + m, A.n, A.bc, src, A.f, tf);
    }
  }
  T F[NV];
  interface_flux<T, NV, 0>(S, A.s, A.dir, F, &A.rec);
}

}  // namespace wcns
