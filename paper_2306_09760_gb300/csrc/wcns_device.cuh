// Device-side numerics of the WCNS-FE scheme (one interface per thread).
//
// Paper: Liu, Min, Cai, Ma, Yan, "A filtered embedded weighted compact nonlinear
// scheme for hyperbolic conservation law", arXiv 2306.09760.
//   Eq. 5      sub-stencil midpoint values q0, q1, q2
//   Eq. 9-10   smoothness indicators IS_k = (h f_k)^2 + (h^2 s_k)^2
//   Eq. 11     JS weights;  Eq. 12-13 M weights;  Eq. 14-15 Z weights
//   Eq. 20-21  FE mapping function with the Table 2 coefficients
//   App. A     PFE switch
//   Eq. 6      midpoint flux from an approximate Riemann solver
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

// Device numerics are also host-callable so that tools can evaluate them on the CPU.
#define WCNS_HD __host__ __device__ __forceinline__

namespace wcns {

// Scheme parameters as the kernels see them.
struct Scheme {
  int system;          // 0 advection, 1 Euler
  int weights;         // 0 JS, 1 Z, 2 FE, 3 PFE, 4 M
  int flux;            // 0 LLF, 1 Roe, 2 HLLC, 3 LLF with frozen alpha
  int characteristic;  // project onto characteristic fields (Euler)
  int zp;              // Z exponent p (1 or 2)
  int renorm;          // renormalise mapped weights
  int family;          // 0 WCNS (midpoint interpolation, Eq. 3); 1 finite-difference WENO (App. B)
  double gamma, eps, xi, cv, harten;
  double speed[2];     // advection speed (advection) or frozen LF alpha (LLF_FROZEN), per direction
  // Null points kappa*(psi_j + psi_{j-1}) of Eq. 20 for the three weights (Table 2 rows,
  // or Table B.2 rows for the WENO family).
  double null0[3], null1[4], null2[3];
  // Ideal weights and the interior control values omega_{i,j} of those rows.
  double ideal[3], ctrl0[2], ctrl1[3], ctrl2[2];
};

// The step of the current RK step as the sweeps read it: the double value, its
// single-precision copy and a flag for dt == 0 (the run has reached t_end), written
// together by the step kernel so that single-precision sweeps never use the double pipe.
struct StepDt {
  double dt;
  double t0;   // time at the start of the step (stage times t0 + c_k dt)
  float dt32;
  int zero;
};

// Slot pairs into which the last RK stage of a 2D Euler step merges the CFL maxima of the
// state it writes (one slot per warp, modulo the count).
constexpr int kWaveSlots = 256;

// Boundary faces x-lo, x-hi, y-lo, y-hi beyond periodic / transmissive lines (Sec. 4.3):
// 0 the direction's bc, 1 transmissive, 2 inviscid wall (mirror cell, normal momentum
// reversed), 3 fixed state A, 4 state A for x < wall_x and a wall beyond, 5 the moving
// oblique shock (state A for x < x0 + (y + speed t) dxdy, state B beyond).  Ghost values
// are evaluated at the ghost cell's centre.  States: conservative, storage ordering.
enum FaceType { kFaceGrid = 0, kFaceTransmissive = 1, kFaceWall = 2, kFaceFixed = 3, kFaceFixedThenWall = 4,
                kFaceShock = 5 };
template <typename T>
struct Faces {
  int active;
  int type[4];
  T ua[4], ub[4];
  double wall_x, x0, dxdy, speed, lo_x, lo_y, hx, hy;
};

// The same parameters in the kernel's own precision (no conversions inside kernels).
template <typename T>
struct SchemeT {
  int system, weights, flux, characteristic, zp, renorm, family;
  int xi_small;  // single precision with xi < 1e4: the FE map uses the exponential form of tanh
  T gamma, gm1, eps, xi, cv, harten;
  T sat_dist;    // |w - null| at and beyond which every FE tanh term is saturated (kSat / xi)
  // Ideal-plateau test of the FE map (weights == FE only; 0 = off): where every base weight
  // w_k lies within ideal_margin[k] of the ideal weight d_k, it is farther than the
  // saturation distance from every null point, inside the plateau whose control value is
  // d_k, so Eq. 20 returns the ideal weights exactly; they sum to exactly 1, so the
  // renormalised weights are the ideal weights, which the kernels then use directly.
  T ideal_margin[3];
  // The same test on the Z ratios before normalisation (0 = off): where every ratio
  // r_k^p of Eq. 14 is below ideal_ratio, each Z weight lies within d_k * ideal_ratio
  // < ideal_margin[k] of d_k (the weights are d_k (1 + r_k^p) / (1 + sum_l d_l r_l^p)).
  T ideal_ratio;
  T speed[2];
  T null0[3], null1[4], null2[3];
  T ideal[3], ctrl0[2], ctrl1[3], ctrl2[2];
};

// Control rows of Eq. 20 for a family: Table 2 (WCNS) or Table B.2 (WENO).  Fills the
// null points kappa (psi_{i,j} + psi_{i,j-1}), the ideal weights and the interior
// control values.  Host code; independent of the CPU oracle's tables.
inline void fill_family_tables(Scheme& s, int family, double kappa) {
  static const double psi_wcns[3][5] = {{0.0, 1.0 / 16.0, 1.0 / 11.0, 1.0, 0.0},
                                        {0.0, 10.0 / 16.0, 2.0 / 3.0, 10.0 / 11.0, 1.0},
                                        {0.0, 5.0 / 16.0, 1.0 / 3.0, 1.0, 0.0}};
  static const double psi_weno[3][5] = {{0.0, 1.0 / 10.0, 1.0 / 7.0, 1.0, 0.0},
                                        {0.0, 6.0 / 10.0, 2.0 / 3.0, 6.0 / 7.0, 1.0},
                                        {0.0, 3.0 / 10.0, 1.0 / 3.0, 1.0, 0.0}};
  const double(*psi)[5] = family == 1 ? psi_weno : psi_wcns;
  for (int j = 1; j <= 3; ++j) s.null0[j - 1] = kappa * (psi[0][j] + psi[0][j - 1]);
  for (int j = 1; j <= 4; ++j) s.null1[j - 1] = kappa * (psi[1][j] + psi[1][j - 1]);
  for (int j = 1; j <= 3; ++j) s.null2[j - 1] = kappa * (psi[2][j] + psi[2][j - 1]);
  s.family = family;
  if (family == 1) {
    s.ideal[0] = 1.0 / 10.0; s.ideal[1] = 6.0 / 10.0; s.ideal[2] = 3.0 / 10.0;
    s.ctrl0[0] = 1.0 / 10.0; s.ctrl0[1] = 1.0 / 4.0;
    s.ctrl1[0] = 6.0 / 10.0; s.ctrl1[1] = 1.0 / 2.0; s.ctrl1[2] = 3.0 / 4.0;
    s.ctrl2[0] = 3.0 / 10.0; s.ctrl2[1] = 1.0 / 2.0;
  } else {
    s.ideal[0] = 1.0 / 16.0; s.ideal[1] = 10.0 / 16.0; s.ideal[2] = 5.0 / 16.0;
    s.ctrl0[0] = 1.0 / 16.0; s.ctrl0[1] = 1.0 / 6.0;
    s.ctrl1[0] = 10.0 / 16.0; s.ctrl1[1] = 1.0 / 2.0; s.ctrl1[2] = 5.0 / 6.0;
    s.ctrl2[0] = 5.0 / 16.0; s.ctrl2[1] = 1.0 / 2.0;
  }
}

template <typename T>
inline Faces<T> faces_as(const Faces<double>& f) {
  Faces<T> r;
  r.active = f.active;
  for (int k = 0; k < 4; ++k) { r.type[k] = f.type[k]; r.ua[k] = T(f.ua[k]); r.ub[k] = T(f.ub[k]); }
  r.wall_x = f.wall_x; r.x0 = f.x0; r.dxdy = f.dxdy; r.speed = f.speed;
  r.lo_x = f.lo_x; r.lo_y = f.lo_y; r.hx = f.hx; r.hy = f.hy;
  return r;
}

// Margins of the ideal-plateau test (SchemeT::ideal_margin), from the null points of each
// map: the distance from d_k to its nearest null point, less the saturation distance of
// the saturated evaluation (with the single-precision test's own allowance in double
// precision) and a rounding allowance.  Off (0) unless the weights are FE, the map is
// evaluated in saturated form, d_k lies strictly inside the plateau whose control value
// it is (true for both families at kappa = 0.5), and the ideal weights sum to exactly 1
// in the kernel's precision.
template <typename T>
inline void ideal_margins(const Scheme& s, SchemeT<T>& r) {
  for (int k = 0; k < 3; ++k) r.ideal_margin[k] = T(0);
  r.ideal_ratio = T(0);
  if (s.weights != 2 || r.xi_small) return;
  if (T(T(s.ideal[0]) + T(s.ideal[1])) + T(s.ideal[2]) != T(1)) return;
  const double sat = (sizeof(T) == 4 ? 9.1 : 20.0 + 1.0e-4 + 4.0e-7 * s.xi) / s.xi;
  const double* nulls[3] = {s.null0, s.null1, s.null2};
  const int count[3] = {3, 4, 3};
  const double ctrl0[3] = {s.ctrl0[0], s.ctrl1[0], s.ctrl2[0]};
  double m[3];
  for (int k = 0; k < 3; ++k) {
    const double d = s.ideal[k];
    if (ctrl0[k] != d) return;
    double lo = -1.0, hi = 2.0;
    for (int j = 0; j < count[k]; ++j) {
      const double n = nulls[k][j];
      if (n <= d && n > lo) lo = n;
      if (n > d && n < hi) hi = n;
    }
    // d must lie between the first two null points (the plateau of control value d)
    if (!(lo == nulls[k][0] && hi == nulls[k][1])) return;
    m[k] = (d - lo < hi - d ? d - lo : hi - d) * (1.0 - 1.0e-6) - sat * (1.0 + 1.0e-3) - 1.0e-6;
    if (!(m[k] > 0.0)) return;
  }
  double ratio = 1.0;
  for (int k = 0; k < 3; ++k) {
    r.ideal_margin[k] = T(m[k]);
    ratio = m[k] / s.ideal[k] < ratio ? m[k] / s.ideal[k] : ratio;
  }
  r.ideal_ratio = T(ratio * (1.0 - 1.0e-3));
}

template <typename T>
inline SchemeT<T> scheme_as(const Scheme& s) {
  SchemeT<T> r;
  r.system = s.system; r.weights = s.weights; r.flux = s.flux;
  r.xi_small = (sizeof(T) == 4 && s.xi < 1e4) ? 1 : 0;
  r.characteristic = s.characteristic; r.zp = s.zp; r.renorm = s.renorm; r.family = s.family;
  r.gamma = T(s.gamma); r.gm1 = T(s.gamma - 1.0); r.xi = T(s.xi);
  // eps = 1e-40 is below the smallest normal float and single-precision kernels flush
  // subnormals to zero, so it is raised to 2^-126 there (IS + eps then never vanishes).
  r.eps = (sizeof(T) == 4 && s.eps < 1.1754943508222875e-38) ? T(1.1754943508222875e-38) : T(s.eps);
  r.cv = T(s.cv); r.harten = T(s.harten);
  // rounded up so that xi * |w - null| >= kSat holds whenever the distance test passes
  r.sat_dist = T((sizeof(T) == 4 ? 9.1 : 20.0) / s.xi * (1.0 + 1e-6));
  for (int d = 0; d < 2; ++d) r.speed[d] = T(s.speed[d]);
  for (int j = 0; j < 3; ++j) { r.null0[j] = T(s.null0[j]); r.null2[j] = T(s.null2[j]); }
  for (int j = 0; j < 4; ++j) r.null1[j] = T(s.null1[j]);
  for (int k = 0; k < 3; ++k) { r.ideal[k] = T(s.ideal[k]); r.ctrl1[k] = T(s.ctrl1[k]); }
  for (int k = 0; k < 2; ++k) { r.ctrl0[k] = T(s.ctrl0[k]); r.ctrl2[k] = T(s.ctrl2[k]); }
  ideal_margins<T>(s, r);
  return r;
}

// Compile-time specialisation of the option switches.  FIX = 0: every option read
// from the scheme at run time.  FIX = 1: WCNS family, FE weights (Z, p = 1,
// renormalised, kappa = 0.5, xi >= 1e4), HLLC, characteristic projection -- the default
// configuration (fixed_config), compiled without the other branches.
template <int FIX> struct Fixed {
  static constexpr bool on = false;
  static constexpr int weights = 0, flux = 0, characteristic = 0, zp = 1, renorm = 1, family = 0;
};
template <> struct Fixed<1> {
  static constexpr bool on = true;
  static constexpr int weights = 2, flux = 2, characteristic = 1, zp = 1, renorm = 1, family = 0;
};
#define WCNS_OPT(FIX, s, field) (Fixed<FIX>::on ? Fixed<FIX>::field : (s).field)

// ---------------------------------------------------------------------------
// Small math helpers
// ---------------------------------------------------------------------------
template <typename T> struct Num;
// 1/y in double precision by Newton's iteration for the reciprocal, x <- x + x (1 - y x)
// (each step squares the relative error), from the reciprocal unit's approximation
// (PTX rcp.approx.ftz.f64) with two steps, each two fused multiply-adds.  On GB300 a
// double-precision division is a longer sequence on the FP64 pipe, which is the roof of
// the FP64 sweeps; x * rcp_nr(y) differs from x / y by at most a couple of ulps
// (checked against IEEE division through wcns_reciprocal_f64).  Normal, finite y only
// (the scheme divides by densities, sums of positive weights and nonzero wave-speed
// differences).
__device__ __forceinline__ double rcp_nr(double y) {
  double x;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(y));
  double e = fma(-y, x, 1.0);
  x = fma(x, e, x);
  e = fma(-y, x, 1.0);
  return fma(x, e, x);
}

template <> struct Num<double> {
  // |z| at and beyond which tanh(z) rounds to +-1 exactly in double precision
  // (1 - tanh(20) = 8.5e-18 < half an ulp of 1).
  static constexpr double kSat = 20.0;
  WCNS_HD static double tanh_(double z) { return tanh(z); }
  WCNS_HD static double sqrt_(double x) { return sqrt(x); }
  WCNS_HD static double abs_(double x) { return fabs(x); }
#ifdef __CUDA_ARCH__
  WCNS_HD static double div_(double x, double y) { return x * rcp_nr(y); }
  WCNS_HD static double rcp_(double x) { return rcp_nr(x); }
#else
  WCNS_HD static double div_(double x, double y) { return x / y; }
  WCNS_HD static double rcp_(double x) { return 1.0 / x; }
#endif
  WCNS_HD static double z_ratio(double tau, double b) { return div_(tau, b); }
};
template <> struct Num<float> {
  // 1 - tanh(9.1) = 2.5e-8 < half an ulp of 1 in single precision.
  static constexpr float kSat = 9.1f;
  WCNS_HD static float tanh_(float z) { return tanhf(z); }
  WCNS_HD static float sqrt_(float x) { return sqrtf(x); }
  WCNS_HD static float abs_(float x) { return fabsf(x); }
  // Division through the reciprocal unit (error within 2 ulp for |y| in [2^-126, 2^126];
  // every divisor of the scheme stays in that range for data below ~1e18).
  WCNS_HD static float div_(float x, float y) {
#ifdef __CUDA_ARCH__
    return __fdividef(x, y);
#else
    return x / y;
#endif
  }
  WCNS_HD static float rcp_(float x) { return div_(1.0f, x); }
  // Z ratio tau / (IS + eps) (Eq. 15).  In single precision eps is at least the smallest
  // normal float, so next to a jump (tau > 4 with IS = 0) the quotient can overflow;
  // it is capped at 1e18, where the weight of that stencil is already 1 to within
  // rounding, as in the double-precision evaluation with eps = 1e-40.
  WCNS_HD static float z_ratio(float tau, float b) { return fminf(div_(tau, b), 1.0e18f); }
};

// tanh(z) with an exact select where the result rounds to +-1 anyway.
template <typename T>
WCNS_HD T tanh_sat(T z) {
  T a = Num<T>::abs_(z);
  if (a >= Num<T>::kSat) return z > T(0) ? T(1) : T(-1);
  return Num<T>::tanh_(z);
}

// ---------------------------------------------------------------------------
// Eq. 20-21 (Table 2).  phi(i, j) = -1 multiplies both the amplitude and the tanh
// argument and tanh is odd, so every term reduces to
//   (omega_{i,j} - omega_{i,j-1}) / 2 * tanh(xi * (w - null_j)),
// with omega_{i,0} = omega_{i,J} = w.  The map is a smoothed staircase whose
// plateaus are the control values.
// ---------------------------------------------------------------------------
// Exact evaluation of map i at w (any tanh argument).
template <typename T>
WCNS_HD T fe_map_exact(int i, T w, const SchemeT<T>& s) {
  const T xi = s.xi;
  if (i == 0) {
    T t1 = tanh_sat<T>(xi * (w - s.null0[0]));
    T t2 = tanh_sat<T>(xi * (w - s.null0[1]));
    T t3 = tanh_sat<T>(xi * (w - s.null0[2]));
    T acc = ((s.ctrl0[0] - w) / T(2)) * t1;
    acc = acc + ((s.ctrl0[1] - s.ctrl0[0]) / T(2)) * t2;
    acc = acc + ((w - s.ctrl0[1]) / T(2)) * t3;
    return acc + w;
  }
  if (i == 1) {
    T t1 = tanh_sat<T>(xi * (w - s.null1[0]));
    T t2 = tanh_sat<T>(xi * (w - s.null1[1]));
    T t3 = tanh_sat<T>(xi * (w - s.null1[2]));
    T t4 = tanh_sat<T>(xi * (w - s.null1[3]));
    T acc = ((s.ctrl1[0] - w) / T(2)) * t1;
    acc = acc + ((s.ctrl1[1] - s.ctrl1[0]) / T(2)) * t2;
    acc = acc + ((s.ctrl1[2] - s.ctrl1[1]) / T(2)) * t3;
    acc = acc + ((w - s.ctrl1[2]) / T(2)) * t4;
    return acc + w;
  }
  T t1 = tanh_sat<T>(xi * (w - s.null2[0]));
  T t2 = tanh_sat<T>(xi * (w - s.null2[1]));
  T t3 = tanh_sat<T>(xi * (w - s.null2[2]));
  T acc = ((s.ctrl2[0] - w) / T(2)) * t1;
  acc = acc + ((s.ctrl2[1] - s.ctrl2[0]) / T(2)) * t2;
  acc = acc + ((w - s.ctrl2[1]) / T(2)) * t3;
  return acc + w;
}

// Out-of-line copy of the exact map: the tanh code exists once per kernel instead of
// once per inlined call site.
template <typename T>
__host__ __device__ __noinline__ T fe_map_slow(int i, T w, const SchemeT<T>& s) {
  return fe_map_exact<T>(i, w, s);
}

// Sign of z as the value tanh(z) rounds to once |z| >= kSat.
template <typename T>
WCNS_HD T sat_sign(T z) { return z > T(0) ? T(1) : T(-1); }

// Saturation test of xi (w - n) for every null point n of one map.  In double
// precision the test runs in single precision (fast pipe) with a margin that covers
// the rounding of w, n and xi * (w - n) to float: |xi (w - n)| >= 20 holds whenever the
// float estimate is >= 20 + 1e-4 + 1.2e-7 * xi * (|w| + |n|).  The signs are then exact.
template <typename T, int K>
WCNS_HD bool all_saturated(T w, const T (&n)[K], T xi) {
  if constexpr (sizeof(T) == 8) {
    const float wf = (float)w, xf = (float)xi;
    bool sat = true;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const float nf = (float)n[j];
      const float z = xf * (wf - nf);
      const float margin = 1.0e-4f + 1.2e-7f * xf * (fabsf(wf) + fabsf(nf));
      sat = sat && (fabsf(z) >= 20.0f + margin);
    }
    return sat;
  } else {
    bool sat = true;
#pragma unroll
    for (int j = 0; j < K; ++j) sat = sat && (Num<T>::abs_(xi * (w - n[j])) >= Num<T>::kSat);
    return sat;
  }
}

// Sign of w - n once the test above passed (|w - n| is then far from zero).
template <typename T>
WCNS_HD T side_of(T w, T n) { return w > n ? T(1) : T(-1); }

// Eq. 20 for weight i.  When every tanh argument is saturated (the usual case at
// large xi) each term is exactly +-amplitude and the map is evaluated with signs;
// otherwise the exact out-of-line path runs.  Both give the same value there.
// tanh(z) = 1 - 2 / (e^{2z} + 1) (Eq. 19 rearranged), evaluated with the fast exponential
// and reciprocal of the single-precision pipe; it reaches +-1 exactly for large |z|
// (e^{2z} overflows to inf or underflows to 0), so no branch is needed.  Absolute error
// about 1e-7, well inside the single-precision path's tolerance.
WCNS_HD float tanh_expf(float z) {
#ifdef __CUDA_ARCH__
  return 1.0f - __fdividef(2.0f, __expf(2.0f * z) + 1.0f);
#else
  return tanhf(z);
#endif
}

// Eq. 20 for the single-precision path at moderate xi (every term evaluated).
template <typename T, int K>
WCNS_HD T fe_map_expf(T w, const T (&n)[K], const T (&amp)[K + 1], T xi) {
  T acc = T(0);
#pragma unroll
  for (int j = 0; j < K; ++j) acc = acc + amp[j] * tanh_expf(xi * (w - n[j]));
  return acc;
}

template <typename T>
WCNS_HD T fe_map0(T w, const SchemeT<T>& s) {
  const T c0 = s.ctrl0[0], c1 = s.ctrl0[1];
  if constexpr (sizeof(T) == 4) {
    if (s.xi_small) {
      const T amp[4] = {(c0 - w) / T(2), (c1 - c0) / T(2), (w - c1) / T(2), T(0)};
      return fe_map_expf<T, 3>(w, s.null0, amp, s.xi) + w;
    }
  }
  if (!all_saturated<T, 3>(w, s.null0, s.xi)) return fe_map_slow<T>(0, w, s);
  T acc = ((c0 - w) / T(2)) * side_of(w, s.null0[0]);
  acc = acc + ((c1 - c0) / T(2)) * side_of(w, s.null0[1]);
  acc = acc + ((w - c1) / T(2)) * side_of(w, s.null0[2]);
  return acc + w;
}
template <typename T>
WCNS_HD T fe_map1(T w, const SchemeT<T>& s) {
  const T c0 = s.ctrl1[0], c1 = s.ctrl1[1], c2 = s.ctrl1[2];
  if constexpr (sizeof(T) == 4) {
    if (s.xi_small) {
      const T amp[5] = {(c0 - w) / T(2), (c1 - c0) / T(2), (c2 - c1) / T(2), (w - c2) / T(2), T(0)};
      return fe_map_expf<T, 4>(w, s.null1, amp, s.xi) + w;
    }
  }
  if (!all_saturated<T, 4>(w, s.null1, s.xi)) return fe_map_slow<T>(1, w, s);
  T acc = ((c0 - w) / T(2)) * side_of(w, s.null1[0]);
  acc = acc + ((c1 - c0) / T(2)) * side_of(w, s.null1[1]);
  acc = acc + ((c2 - c1) / T(2)) * side_of(w, s.null1[2]);
  acc = acc + ((w - c2) / T(2)) * side_of(w, s.null1[3]);
  return acc + w;
}
template <typename T>
WCNS_HD T fe_map2(T w, const SchemeT<T>& s) {
  const T c0 = s.ctrl2[0], c1 = s.ctrl2[1];
  if constexpr (sizeof(T) == 4) {
    if (s.xi_small) {
      const T amp[4] = {(c0 - w) / T(2), (c1 - c0) / T(2), (w - c1) / T(2), T(0)};
      return fe_map_expf<T, 3>(w, s.null2, amp, s.xi) + w;
    }
  }
  if (!all_saturated<T, 3>(w, s.null2, s.xi)) return fe_map_slow<T>(2, w, s);
  T acc = ((c0 - w) / T(2)) * side_of(w, s.null2[0]);
  acc = acc + ((c1 - c0) / T(2)) * side_of(w, s.null2[1]);
  acc = acc + ((w - c1) / T(2)) * side_of(w, s.null2[2]);
  return acc + w;
}

// Null points of the default configuration (WCNS family, Table 2 rows, kappa = 0.5) as
// compile-time constants, formed with the same double operations as fill_family_tables.
WCNS_HD constexpr double fe_null_default(int i, int j) {
  return i == 0 ? (j == 0 ? 0.5 * (1.0 / 16.0 + 0.0) : j == 1 ? 0.5 * (1.0 / 11.0 + 1.0 / 16.0) : 0.5 * (1.0 + 1.0 / 11.0))
       : i == 1 ? (j == 0 ? 0.5 * (10.0 / 16.0 + 0.0) : j == 1 ? 0.5 * (2.0 / 3.0 + 10.0 / 16.0)
                   : j == 2 ? 0.5 * (10.0 / 11.0 + 2.0 / 3.0) : 0.5 * (1.0 + 10.0 / 11.0))
                : (j == 0 ? 0.5 * (5.0 / 16.0 + 0.0) : j == 1 ? 0.5 * (1.0 / 3.0 + 5.0 / 16.0) : 0.5 * (1.0 + 1.0 / 3.0));
}

// The configuration the FIX = 1 kernels are compiled for: WCNS family, FE weights (Z,
// p = 1, renormalised) with kappa = 0.5 and xi >= 1e4, HLLC, characteristic projection.
inline bool fixed_config(const Scheme& s) {
  if (!(s.weights == 2 && s.flux == 2 && s.characteristic == 1 && s.zp == 1 && s.renorm == 1 && s.family == 0))
    return false;
  if (s.xi < 1e4) return false;  // single precision evaluates the map differently below 1e4

  for (int j = 0; j < 3; ++j)
    if (s.null0[j] != fe_null_default(0, j) || s.null2[j] != fe_null_default(2, j)) return false;
  for (int j = 0; j < 4; ++j)
    if (s.null1[j] != fe_null_default(1, j)) return false;
  return true;
}

// Null point j of map i: a compile-time constant for FAM = 0, else the scheme's.
template <typename T, int FAM>
WCNS_HD T fe_null(const SchemeT<T>& s, int i, int j) {
  if (FAM == 0) return T(fe_null_default(i, j));
  return i == 0 ? s.null0[j] : (i == 1 ? s.null1[j] : s.null2[j]);
}

// Smallest |w_i - null| over the ten null points of the three maps.
template <typename T, int FAM>
WCNS_HD T fe_null_distance(T w0, T w1, T w2, const SchemeT<T>& s) {
  T d = fmin(fmin(Num<T>::abs_(w0 - fe_null<T, FAM>(s, 0, 0)), Num<T>::abs_(w0 - fe_null<T, FAM>(s, 0, 1))),
             Num<T>::abs_(w0 - fe_null<T, FAM>(s, 0, 2)));
  d = fmin(d, fmin(fmin(Num<T>::abs_(w1 - fe_null<T, FAM>(s, 1, 0)), Num<T>::abs_(w1 - fe_null<T, FAM>(s, 1, 1))),
                   fmin(Num<T>::abs_(w1 - fe_null<T, FAM>(s, 1, 2)), Num<T>::abs_(w1 - fe_null<T, FAM>(s, 1, 3)))));
  return fmin(d, fmin(fmin(Num<T>::abs_(w2 - fe_null<T, FAM>(s, 2, 0)), Num<T>::abs_(w2 - fe_null<T, FAM>(s, 2, 1))),
                      Num<T>::abs_(w2 - fe_null<T, FAM>(s, 2, 2))));
}

// The saturated map (every tanh term +-1): the identity below the first and above the
// last null point, the control values of Table 1 (Table B.1) in between.
// a < b for a non-negative a (a weight, a ratio, a distance) and any non-NaN b: in double
// precision the bit patterns, read as signed 64-bit integers, order like the values there,
// so the compare runs on the integer pipe instead of the FP64 pipe; in single precision
// the plain compare.
template <typename T>
WCNS_HD bool lt_nonneg(T a, T b) { return a < b; }
template <>
WCNS_HD bool lt_nonneg<double>(double a, double b) {
#ifdef __CUDA_ARCH__
  return __double_as_longlong(a) < __double_as_longlong(b);
#else
  return a < b;
#endif
}

template <typename T, int FAM>
WCNS_HD void fe_staircase(T& w0, T& w1, T& w2, const SchemeT<T>& s) {
  const T c00 = FAM == 0 ? T(1.0 / 16.0) : s.ctrl0[0], c01 = FAM == 0 ? T(1.0 / 6.0) : s.ctrl0[1];
  const T c10 = FAM == 0 ? T(10.0 / 16.0) : s.ctrl1[0], c11 = FAM == 0 ? T(0.5) : s.ctrl1[1];
  const T c12 = FAM == 0 ? T(5.0 / 6.0) : s.ctrl1[2];
  const T c20 = FAM == 0 ? T(5.0 / 16.0) : s.ctrl2[0], c21 = FAM == 0 ? T(0.5) : s.ctrl2[1];
  const T g0 = lt_nonneg<T>(w0, fe_null<T, FAM>(s, 0, 1)) ? c00 : c01;
  w0 = (lt_nonneg<T>(w0, fe_null<T, FAM>(s, 0, 0)) || lt_nonneg<T>(fe_null<T, FAM>(s, 0, 2), w0)) ? w0 : g0;
  const T g1 = lt_nonneg<T>(w1, fe_null<T, FAM>(s, 1, 1)) ? c10 : (lt_nonneg<T>(w1, fe_null<T, FAM>(s, 1, 2)) ? c11 : c12);
  w1 = (lt_nonneg<T>(w1, fe_null<T, FAM>(s, 1, 0)) || lt_nonneg<T>(fe_null<T, FAM>(s, 1, 3), w1)) ? w1 : g1;
  const T g2 = lt_nonneg<T>(w2, fe_null<T, FAM>(s, 2, 1)) ? c20 : c21;
  w2 = (lt_nonneg<T>(w2, fe_null<T, FAM>(s, 2, 0)) || lt_nonneg<T>(fe_null<T, FAM>(s, 2, 2), w2)) ? w2 : g2;
}

// Eq. 20 for the three weights together.  Where every tanh argument of all three maps
// is saturated (|xi (w - n)| >= kSat for each null point n), each term is exactly
// +-amplitude and the sum collapses to a staircase evaluated by comparisons
// (fe_staircase); otherwise (any argument unsaturated) the exact path runs.
// FAM = 0: the default configuration's null points and control values are compile-time
// constants; FAM = -1: they are read from the scheme (either family).
template <typename T, int FAM = -1>
WCNS_HD void fe_map_all(T& w0, T& w1, T& w2, const SchemeT<T>& s) {
  bool sat;
  if constexpr (sizeof(T) == 8) {
    // the distance test in single precision, with a margin for the rounding to float
    const float xf = (float)s.xi;
    const float a = (float)w0, b = (float)w1, c = (float)w2;
    float d = fminf(fminf(fabsf(a - (float)s.null0[0]), fabsf(a - (float)s.null0[1])), fabsf(a - (float)s.null0[2]));
    d = fminf(d, fminf(fminf(fabsf(b - (float)s.null1[0]), fabsf(b - (float)s.null1[1])),
                       fminf(fabsf(b - (float)s.null1[2]), fabsf(b - (float)s.null1[3]))));
    d = fminf(d, fminf(fminf(fabsf(c - (float)s.null2[0]), fabsf(c - (float)s.null2[1])), fabsf(c - (float)s.null2[2])));
    sat = xf * d >= 20.0f + 1.0e-4f + 4.0e-7f * xf;
  } else {
    if (FAM != 0 && s.xi_small) {  // the default configuration has xi >= 1e4
      w0 = fe_map0<T>(w0, s); w1 = fe_map1<T>(w1, s); w2 = fe_map2<T>(w2, s);
      return;
    }
    sat = fe_null_distance<T, FAM>(w0, w1, w2, s) >= s.sat_dist;
  }
  if (!sat) {
    w0 = fe_map_slow<T>(0, w0, s); w1 = fe_map_slow<T>(1, w1, s); w2 = fe_map_slow<T>(2, w2, s);
    return;
  }
  fe_staircase<T, FAM>(w0, w1, w2, s);
}

// Eq. 13: Henrick's mapping of a JS weight with ideal value d.
template <typename T>
WCNS_HD T m_map(T w, T d) {
  return Num<T>::div_(w * (d + d * d - T(3) * d * w + w * w), d * d + (T(1) - T(2) * d) * w);
}

// Midpoint value at x_{i+1/2} from five values v0..v4 = u_{i-2}..u_{i+2} (left state), or
// the mirrored u_{i+3}..u_{i-1} (right state).  Returns the interpolated value.
// wz, wf (optional): receive the base weights (Z, or JS before the M map) and the final
// weights, for the weight statistics of App. A.
template <typename T, int FIX>
WCNS_HD T weno_side(T v0, T v1, T v2, T v3, T v4, const SchemeT<T>& s, T* wz = nullptr, T* wf = nullptr) {
  const int weights = WCNS_OPT(FIX, s, weights);
  const int zp = WCNS_OPT(FIX, s, zp);
  const int renorm = WCNS_OPT(FIX, s, renorm);
  const int family = WCNS_OPT(FIX, s, family);
  const T d0 = Fixed<FIX>::on ? T(1.0 / 16.0) : s.ideal[0];
  const T d1 = Fixed<FIX>::on ? T(10.0 / 16.0) : s.ideal[1];
  const T d2 = Fixed<FIX>::on ? T(5.0 / 16.0) : s.ideal[2];
  T q0, q1, q2;
  if (family == 0) {
    // Eq. 5 (coefficients divided by 8 beforehand; powers of two, so exactly)
    q0 = T(0.375) * v0 - T(1.25) * v1 + T(1.875) * v2;
    q1 = -T(0.125) * v1 + T(0.75) * v2 + T(0.375) * v3;
    q2 = T(0.375) * v2 + T(0.75) * v3 - T(0.125) * v4;
  } else {
    // App. B: the fifth-order WENO candidates at x_{i+1/2}
    q0 = (T(2) * v0 - T(7) * v1 + T(11) * v2) / T(6);
    q1 = (-v1 + T(5) * v2 + T(2) * v3) / T(6);
    q2 = (T(2) * v2 + T(5) * v3 - v4) / T(6);
  }
  // Eq. 10 scaled by h and h^2, then Eq. 9 (WENO family: the Jiang-Shu weighting 13/12
  // of the second-difference term)
  T f0 = (v0 - T(4) * v1 + T(3) * v2) / T(2), s0 = v0 - T(2) * v1 + v2;
  T f1 = (v3 - v1) / T(2), s1 = v1 - T(2) * v2 + v3;
  T f2 = (T(-3) * v2 + T(4) * v3 - v4) / T(2), s2 = v2 - T(2) * v3 + v4;
  const T cs = (family == 0) ? T(1) : T(13.0 / 12.0);
  T is0 = f0 * f0 + cs * (s0 * s0);
  T is1 = f1 * f1 + cs * (s1 * s1);
  T is2 = f2 * f2 + cs * (s2 * s2);
  const T eps = s.eps;
  T w0, w1, w2;
  if (weights == 0 || weights == 4) {
    // Eq. 11
    T b0 = is0 + eps, b1 = is1 + eps, b2 = is2 + eps;
    T a0 = Num<T>::div_(d0, b0 * b0), a1 = Num<T>::div_(d1, b1 * b1), a2 = Num<T>::div_(d2, b2 * b2);
    const T isa = Num<T>::rcp_(a0 + a1 + a2);
    w0 = a0 * isa; w1 = a1 * isa; w2 = a2 * isa;
    if (wz) { wz[0] = w0; wz[1] = w1; wz[2] = w2; }
    if (weights == 4) {
      // Eq. 12-13
      T g0 = m_map<T>(w0, d0), g1 = m_map<T>(w1, d1), g2 = m_map<T>(w2, d2);
      const T isg = Num<T>::rcp_(g0 + g1 + g2);
      w0 = g0 * isg; w1 = g1 * isg; w2 = g2 * isg;
    }
  } else {
    // Eq. 14-15
    T tau = Num<T>::abs_(is0 - is2);
    T r0 = T(0), r1 = T(0), r2 = T(0);
    const T b0 = is0 + eps, b1 = is1 + eps, b2 = is2 + eps;
    // the ratios, tau and |w_k - d_k| are non-negative, so the plateau tests compare bit
    // patterns in double precision (lt_nonneg)
    bool small = false;
    if (weights == 2 && !wz && zp == 1) {
      // r_k = tau / b_k < ideal_ratio  <=>  tau < ideal_ratio b_k (b_k > 0), tested before
      // the ratios are formed, against a bound lowered by 1e-6; just below the bound the
      // tests that follow reach the same weights
      const T qv = s.ideal_ratio * T(0.999999);
      small = lt_nonneg<T>(tau, qv * b0) && lt_nonneg<T>(tau, qv * b1) && lt_nonneg<T>(tau, qv * b2);
    }
    if (!small) {
      if constexpr (sizeof(T) == 8) {
        // one division for the three ratios (the product of three IS + eps stays in range)
        const T q = Num<T>::div_(tau, b0 * b1 * b2);
        r0 = q * (b1 * b2); r1 = q * (b0 * b2); r2 = q * (b0 * b1);
      } else {
        r0 = Num<T>::z_ratio(tau, b0); r1 = Num<T>::z_ratio(tau, b1); r2 = Num<T>::z_ratio(tau, b2);
      }
      if (zp == 2) {
        r0 = r0 * r0; r1 = r1 * r1; r2 = r2 * r2;
        small = weights == 2 && !wz && lt_nonneg<T>(r0, s.ideal_ratio) && lt_nonneg<T>(r1, s.ideal_ratio) &&
                lt_nonneg<T>(r2, s.ideal_ratio);
      }
    }
    T a0 = T(0), a1 = T(0), a2 = T(0);
    if (!small) {
      a0 = d0 * (T(1) + r0); a1 = d1 * (T(1) + r1); a2 = d2 * (T(1) + r2);
      const T isa = Num<T>::rcp_(a0 + a1 + a2);
      w0 = a0 * isa; w1 = a1 * isa; w2 = a2 * isa;
      if (wz) { wz[0] = w0; wz[1] = w1; wz[2] = w2; }
    }
    if (small || (weights == 2 && s.ideal_margin[0] > T(0) && lt_nonneg<T>(Num<T>::abs_(w0 - d0), s.ideal_margin[0]) &&
                  lt_nonneg<T>(Num<T>::abs_(w1 - d1), s.ideal_margin[1]) &&
                  lt_nonneg<T>(Num<T>::abs_(w2 - d2), s.ideal_margin[2]))) {
      // inside the ideal plateaus (tested on the ratios, or on the weights): Eq. 20 and the
      // renormalisation give the ideal weights
      w0 = d0; w1 = d1; w2 = d2;
    } else if (weights >= 2) {
      bool keep = false;
      if (weights == 3) {
        // App. A: keep the Z weights inside the closed box |w_k - d_k| <= cv
        const T cv = s.cv;
        keep = (w0 >= d0 - cv) && (w0 <= d0 + cv) && (w1 >= d1 - cv) && (w1 <= d1 + cv) &&
               (w2 >= d2 - cv) && (w2 <= d2 + cv);
      }
      if (!keep) {
        // Eq. 20 on each weight, then renormalised
        T g0 = w0, g1 = w1, g2 = w2;
        fe_map_all<T, Fixed<FIX>::on ? 0 : -1>(g0, g1, g2, s);
        if (renorm) {
          const T isg = Num<T>::rcp_(g0 + g1 + g2);
          w0 = g0 * isg; w1 = g1 * isg; w2 = g2 * isg;
        } else {
          w0 = g0; w1 = g1; w2 = g2;
        }
      }
    }
  }
  if (wf) { wf[0] = w0; wf[1] = w1; wf[2] = w2; }
  // Eq. 6: convex combination
  return w0 * q0 + w1 * q1 + w2 * q2;
}

// Weight statistics of App. A: histograms [2][3][nbins] (base, final) x (weight index)
// of every one-sided interpolation, bin = clamp(floor(w * nbins + 1e-6), 0, nbins - 1).
// The ideal weights and the control values of Tables 1 and B.1 are multiples of 1e-4,
// so with 1e4 bins they sit exactly on bin edges; the offset (1e-10 in w) puts a
// weight that round-off leaves just below such an edge into the edge's bin.
struct WeightRecorder {
  unsigned long long* hist;
  int nbins;
};

template <typename T>
WCNS_HD int weight_bin(T w, int nbins) {
  const double x = (double)w * (double)nbins + 1e-6;
  const int b = x < 0.0 ? 0 : (int)x;
  return b >= nbins ? nbins - 1 : b;
}

// weno_side, recording its weights when a recorder is given.
template <typename T, int FIX>
WCNS_HD T weno_rec(const WeightRecorder* rec, T v0, T v1, T v2, T v3, T v4, const SchemeT<T>& s) {
  if (!rec) return weno_side<T, FIX>(v0, v1, v2, v3, v4, s);
  T wz[3], wf[3];
  const T r = weno_side<T, FIX>(v0, v1, v2, v3, v4, s, wz, wf);
#ifdef __CUDA_ARCH__
  for (int k = 0; k < 3; ++k) {
    atomicAdd(&rec->hist[(0 * 3 + k) * rec->nbins + weight_bin(wz[k], rec->nbins)], 1ull);
    atomicAdd(&rec->hist[(1 * 3 + k) * rec->nbins + weight_bin(wf[k], rec->nbins)], 1ull);
  }
#endif
  return r;
}

// ---------------------------------------------------------------------------
// Euler equations in a sweep normal.  State ordering within a sweep:
// NV = 3: (rho, rho un, E);  NV = 4: (rho, rho un, rho ut, E).
// ---------------------------------------------------------------------------
template <typename T, int NV>
struct EulerState {
  T rho, un, ut, p, H;
};

template <typename T, int NV>
WCNS_HD EulerState<T, NV> euler_prim(const T (&U)[NV], T gm1) {
  EulerState<T, NV> st;
  st.rho = U[0];
  T inv = Num<T>::rcp_(U[0]);
  st.un = U[1] * inv;
  T E;
  if (NV == 4) {
    st.ut = U[2] * inv;
    E = U[3];
    st.p = gm1 * (E - T(0.5) * st.rho * (st.un * st.un + st.ut * st.ut));
  } else {
    st.ut = T(0);
    E = U[NV - 1];
    st.p = gm1 * (E - T(0.5) * st.rho * st.un * st.un);
  }
  st.H = (E + st.p) * inv;
  return st;
}

template <typename T, int NV>
WCNS_HD void euler_flux(const T (&U)[NV], const EulerState<T, NV>& st, T (&F)[NV]) {
  F[0] = U[1];
  F[1] = U[1] * st.un + st.p;
  if (NV == 4) {
    F[2] = U[2] * st.un;
    F[3] = (U[3] + st.p) * st.un;
  } else {
    F[NV - 1] = (U[NV - 1] + st.p) * st.un;
  }
}

// Roe-averaged velocity, enthalpy and sound speed of two states.
template <typename T, int NV>
struct RoeAvg {
  T u, v, H, c;
};
template <typename T, int NV>
WCNS_HD RoeAvg<T, NV> roe_avg(const EulerState<T, NV>& a, const EulerState<T, NV>& b, T gm1) {
  RoeAvg<T, NV> r;
  T sa = Num<T>::sqrt_(a.rho), sb = Num<T>::sqrt_(b.rho);
  T inv = Num<T>::rcp_(sa + sb);
  r.u = (sa * a.un + sb * b.un) * inv;
  r.v = (NV == 4) ? (sa * a.ut + sb * b.ut) * inv : T(0);
  r.H = (sa * a.H + sb * b.H) * inv;
  T q2 = r.u * r.u + r.v * r.v;
  r.c = Num<T>::sqrt_(gm1 * (r.H - T(0.5) * q2));
  return r;
}

// Characteristic projection with the left eigenvectors at the Roe state, written in
// factored form:  P = b (E - u m - v n + q^2 rho / 2) with b = (gamma-1)/c^2,
// A = (u rho - m) / c;  W = ((P + A)/2, rho - P, [n - v rho,] (P - A)/2).
template <typename T, int NV>
struct CharBasis {
  T u, v, H, c, b, ic, hq2;
};
template <typename T, int NV>
WCNS_HD CharBasis<T, NV> char_basis(const RoeAvg<T, NV>& r, T gm1) {
  CharBasis<T, NV> cb;
  cb.u = r.u; cb.v = r.v; cb.H = r.H; cb.c = r.c;
  cb.ic = Num<T>::rcp_(r.c);
  cb.b = gm1 * cb.ic * cb.ic;
  cb.hq2 = T(0.5) * (r.u * r.u + r.v * r.v);
  return cb;
}
template <typename T, int NV>
WCNS_HD void char_project(const CharBasis<T, NV>& cb, const T (&U)[NV], T (&W)[NV]) {
  const T rho = U[0], m = U[1];
  const T E = U[NV - 1];
  T P;
  if (NV == 4) P = cb.b * (E - cb.u * m - cb.v * U[2] + cb.hq2 * rho);
  else P = cb.b * (E - cb.u * m + cb.hq2 * rho);
  T A = (cb.u * rho - m) * cb.ic;
  W[0] = T(0.5) * (P + A);
  W[1] = rho - P;
  if (NV == 4) W[2] = U[2] - cb.v * rho;
  W[NV - 1] = T(0.5) * (P - A);
}
// Back-projection with the right eigenvectors (u - c, u, [u,] u + c columns).
template <typename T, int NV>
WCNS_HD void char_unproject(const CharBasis<T, NV>& cb, const T (&W)[NV], T (&U)[NV]) {
  const T wa = W[0], wb = W[1], wd = W[NV - 1];
  T s = wa + wb + wd;
  T dlt = wd - wa;
  U[0] = s;
  U[1] = cb.u * s + cb.c * dlt;
  if (NV == 4) {
    U[2] = cb.v * s + W[2];
    U[3] = cb.H * (wa + wd) + cb.u * cb.c * dlt + cb.hq2 * wb + cb.v * W[2];
  } else {
    U[2] = cb.H * (wa + wd) + cb.u * cb.c * dlt + cb.hq2 * wb;
  }
}

// Approximate Riemann solvers (Eq. 6).
template <typename T, int NV, int FIX>
WCNS_HD void riemann(const T (&UL)[NV], const T (&UR)[NV], const SchemeT<T>& s, int dir,
                                        T (&F)[NV]) {
  const int flux = WCNS_OPT(FIX, s, flux);
  const T g = s.gamma, gm1 = s.gm1;
  EulerState<T, NV> a = euler_prim<T, NV>(UL, gm1), b = euler_prim<T, NV>(UR, gm1);
  T FL[NV], FR[NV];
  euler_flux<T, NV>(UL, a, FL);
  euler_flux<T, NV>(UR, b, FR);
  if (flux == 0 || flux == 3) {
    T alpha;
    if (flux == 3) {
      alpha = s.speed[dir];
    } else {
      T sl = Num<T>::abs_(a.un) + Num<T>::sqrt_(Num<T>::div_(g * a.p, a.rho));
      T sr = Num<T>::abs_(b.un) + Num<T>::sqrt_(Num<T>::div_(g * b.p, b.rho));
      alpha = sl >= sr ? sl : sr;
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) F[k] = T(0.5) * (FL[k] + FR[k]) - T(0.5) * alpha * (UR[k] - UL[k]);
    return;
  }
  RoeAvg<T, NV> r = roe_avg<T, NV>(a, b, gm1);
  if (flux == 1) {
    // Roe: F = (FL + FR)/2 - 1/2 R |Lambda| L (UR - UL), Harten's fix on u -/+ c
    CharBasis<T, NV> cb = char_basis<T, NV>(r, gm1);
    T dU[NV], dW[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) dU[k] = UR[k] - UL[k];
    char_project<T, NV>(cb, dU, dW);
    T delta = s.harten * (Num<T>::abs_(r.u) + r.c);
    T l0 = Num<T>::abs_(r.u - r.c), lm = Num<T>::abs_(r.u), l3 = Num<T>::abs_(r.u + r.c);
    if (l0 < delta) l0 = Num<T>::div_((r.u - r.c) * (r.u - r.c) + delta * delta, T(2) * delta);
    if (l3 < delta) l3 = Num<T>::div_((r.u + r.c) * (r.u + r.c) + delta * delta, T(2) * delta);
    dW[0] = l0 * dW[0];
    dW[1] = lm * dW[1];
    if (NV == 4) dW[2] = lm * dW[2];
    dW[NV - 1] = l3 * dW[NV - 1];
    T D[NV];
    char_unproject<T, NV>(cb, dW, D);
#pragma unroll
    for (int k = 0; k < NV; ++k) F[k] = T(0.5) * (FL[k] + FR[k]) - T(0.5) * D[k];
    return;
  }
  // HLLC with Einfeldt speed estimates
  T cl = Num<T>::sqrt_(Num<T>::div_(g * a.p, a.rho)), cr = Num<T>::sqrt_(Num<T>::div_(g * b.p, b.rho));
  T SL = a.un - cl, SR = b.un + cr;
  if (r.u - r.c < SL) SL = r.u - r.c;
  if (r.u + r.c > SR) SR = r.u + r.c;
  if (SL >= T(0)) {
#pragma unroll
    for (int k = 0; k < NV; ++k) F[k] = FL[k];
    return;
  }
  if (SR <= T(0)) {
#pragma unroll
    for (int k = 0; k < NV; ++k) F[k] = FR[k];
    return;
  }
  T ml = a.rho * (SL - a.un), mr = b.rho * (SR - b.un);
  T Sst = Num<T>::div_(b.p - a.p + a.un * ml - b.un * mr, ml - mr);
  const bool left = Sst >= T(0);
  const EulerState<T, NV>& st = left ? a : b;
  T SK = left ? SL : SR;
  T fac = Num<T>::div_(st.rho * (SK - st.un), SK - Sst);
  T EK = left ? UL[NV - 1] : UR[NV - 1];
  T Est = fac * (Num<T>::div_(EK, st.rho) + (Sst - st.un) * (Sst + Num<T>::div_(st.p, st.rho * (SK - st.un))));
  T Us[NV];
  Us[0] = fac;
  Us[1] = fac * Sst;
  if (NV == 4) Us[2] = fac * st.ut;
  Us[NV - 1] = Est;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    T fk = left ? FL[k] : FR[k];
    T uk = left ? UL[k] : UR[k];
    F[k] = fk + SK * (Us[k] - uk);
  }
}

template <typename T, int NV>
WCNS_HD bool physical(const T (&U)[NV], T gm1) {
  if (!(U[0] > T(0))) return false;
  T inv = Num<T>::rcp_(U[0]);
  T kin = (NV == 4) ? (U[1] * U[1] + U[2] * U[2]) * inv : U[1] * U[1] * inv;
  T p = gm1 * (U[NV - 1] - T(0.5) * kin);
  return p > T(0);
}

// App. B (WENO family): the flux at x_{i+1/2} from Lax-Friedrichs split fluxes
// f+-_m = (F(U_m) +- alpha U_m) / 2 of the six stencil cells, alpha = max over those
// cells of |u_n| + c (|a| for advection); f+ is reconstructed from cells i-2..i+2,
// f- from the mirrored cells i+3..i-1, in characteristic fields at the Roe state of
// (U_i, U_{i+1}) when selected, and the flux is R (f+^ + f-^).
template <typename T, int NV, int FIX>
WCNS_HD void weno_split_flux(const T (&S)[6][NV], const SchemeT<T>& s, int dir, T (&F)[NV],
                             const WeightRecorder* rec = nullptr) {
  if (NV == 1) {
    const T a = s.speed[dir];
    const T ap = T(0.5) * (a + Num<T>::abs_(a)), am = T(0.5) * (a - Num<T>::abs_(a));
    const T fp = weno_rec<T, FIX>(rec, ap * S[0][0], ap * S[1][0], ap * S[2][0], ap * S[3][0], ap * S[4][0], s);
    const T fm = weno_rec<T, FIX>(rec, am * S[5][0], am * S[4][0], am * S[3][0], am * S[2][0], am * S[1][0], s);
    F[0] = fp + fm;
    return;
  }
  const T gm1 = s.gm1;
  T gp[6][NV], gmn[6][NV];
  T alpha = T(0);
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    const EulerState<T, NV> st = euler_prim<T, NV>(S[m], gm1);
    T Fm[NV];
    euler_flux<T, NV>(S[m], st, Fm);
    const T sp = Num<T>::abs_(st.un) + Num<T>::sqrt_(Num<T>::div_(s.gamma * st.p, st.rho));
    alpha = sp > alpha ? sp : alpha;
#pragma unroll
    for (int k = 0; k < NV; ++k) { gp[m][k] = Fm[k]; gmn[m][k] = S[m][k]; }
  }
#pragma unroll
  for (int m = 0; m < 6; ++m)
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const T f = gp[m][k], u = gmn[m][k];
      gp[m][k] = T(0.5) * (f + alpha * u);
      gmn[m][k] = T(0.5) * (f - alpha * u);
    }
  T Fh[NV];
  if (WCNS_OPT(FIX, s, characteristic)) {
    T Ui[NV], Uj[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) { Ui[k] = S[2][k]; Uj[k] = S[3][k]; }
    const EulerState<T, NV> a = euler_prim<T, NV>(Ui, gm1), b = euler_prim<T, NV>(Uj, gm1);
    const RoeAvg<T, NV> r = roe_avg<T, NV>(a, b, gm1);
    const CharBasis<T, NV> cb = char_basis<T, NV>(r, gm1);
    T Wp[6][NV], Wm[6][NV];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      char_project<T, NV>(cb, gp[m], Wp[m]);
      char_project<T, NV>(cb, gmn[m], Wm[m]);
    }
    T Wh[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k)
      Wh[k] = weno_rec<T, FIX>(rec, Wp[0][k], Wp[1][k], Wp[2][k], Wp[3][k], Wp[4][k], s) +
              weno_rec<T, FIX>(rec, Wm[5][k], Wm[4][k], Wm[3][k], Wm[2][k], Wm[1][k], s);
    char_unproject<T, NV>(cb, Wh, Fh);
  } else {
#pragma unroll
    for (int k = 0; k < NV; ++k)
      Fh[k] = weno_rec<T, FIX>(rec, gp[0][k], gp[1][k], gp[2][k], gp[3][k], gp[4][k], s) +
              weno_rec<T, FIX>(rec, gmn[5][k], gmn[4][k], gmn[3][k], gmn[2][k], gmn[1][k], s);
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) F[k] = Fh[k];
}

// Midpoint flux at one interface from the six stencil states S[0..5] = U_{i-2..i+3}
// (already in the sweep's normal ordering).  Returns true if the interpolated states
// were non-physical and the interface fell back to (U_i, U_{i+1}).
template <typename T, int NV, int FIX>
WCNS_HD bool interface_flux(const T (&S)[6][NV], const SchemeT<T>& s, int dir, T (&F)[NV],
                            const WeightRecorder* rec = nullptr) {
  if (WCNS_OPT(FIX, s, family) == 1) {
    weno_split_flux<T, NV, FIX>(S, s, dir, F, rec);
    return false;
  }
  if (NV == 1) {
    const T a = s.speed[dir];
    T v;
    if (rec) {  // statistics count both one-sided interpolations
      const T vl = weno_rec<T, FIX>(rec, S[0][0], S[1][0], S[2][0], S[3][0], S[4][0], s);
      const T vr = weno_rec<T, FIX>(rec, S[5][0], S[4][0], S[3][0], S[2][0], S[1][0], s);
      v = (a >= T(0)) ? vl : vr;
    } else if (a >= T(0)) {
      v = weno_side<T, FIX>(S[0][0], S[1][0], S[2][0], S[3][0], S[4][0], s);
    } else {
      v = weno_side<T, FIX>(S[5][0], S[4][0], S[3][0], S[2][0], S[1][0], s);
    }
    F[0] = a * v;
    return false;
  }
  const T gm1 = s.gm1;
  T UL[NV], UR[NV];
  if (WCNS_OPT(FIX, s, characteristic)) {
    T Ui[NV], Uj[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) { Ui[k] = S[2][k]; Uj[k] = S[3][k]; }
    EulerState<T, NV> a = euler_prim<T, NV>(Ui, gm1), b = euler_prim<T, NV>(Uj, gm1);
    RoeAvg<T, NV> r = roe_avg<T, NV>(a, b, gm1);
    CharBasis<T, NV> cb = char_basis<T, NV>(r, gm1);
    T W[6][NV];
#pragma unroll
    for (int m = 0; m < 6; ++m) char_project<T, NV>(cb, S[m], W[m]);
    T WL[NV], WR[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      WL[k] = weno_rec<T, FIX>(rec, W[0][k], W[1][k], W[2][k], W[3][k], W[4][k], s);
      WR[k] = weno_rec<T, FIX>(rec, W[5][k], W[4][k], W[3][k], W[2][k], W[1][k], s);
    }
    char_unproject<T, NV>(cb, WL, UL);
    char_unproject<T, NV>(cb, WR, UR);
  } else {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      UL[k] = weno_rec<T, FIX>(rec, S[0][k], S[1][k], S[2][k], S[3][k], S[4][k], s);
      UR[k] = weno_rec<T, FIX>(rec, S[5][k], S[4][k], S[3][k], S[2][k], S[1][k], s);
    }
  }
  bool fallback = false;
  if (!physical<T, NV>(UL, gm1) || !physical<T, NV>(UR, gm1)) {
    fallback = true;
#pragma unroll
    for (int k = 0; k < NV; ++k) { UL[k] = S[2][k]; UR[k] = S[3][k]; }
  }
  riemann<T, NV, FIX>(UL, UR, s, dir, F);
  return fallback;
}

// Eq. 3: -(1/h) sum_m d_m (F_{i+m-1/2} - F_{i-m+1/2}) from the six interface fluxes
// f[0..5] = F_{i-5/2} .. F_{i+5/2}.
// a * b + c, a * b and a + b of the Eq. 3 difference and the stage updates.  In single
// precision they are explicitly rounded (one rounding for a * b + c): no compiler pass
// may fuse or split them, so these expressions round the same way in every kernel they
// are inlined into -- the banded stage kernel and the separate x- and y-sweep kernels
// give the same single-precision states bit for bit.  In double precision they are the
// plain expressions, which both forms compile alike (checked bit for bit as well).
template <typename T> WCNS_HD T sfma(T a, T b, T c) { return a * b + c; }
template <typename T> WCNS_HD T smul(T a, T b) { return a * b; }
template <typename T> WCNS_HD T sadd(T a, T b) { return a + b; }
#ifdef __CUDA_ARCH__
template <> WCNS_HD float sfma<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> WCNS_HD float smul<float>(float a, float b) { return __fmul_rn(a, b); }
template <> WCNS_HD float sadd<float>(float a, float b) { return __fadd_rn(a, b); }
#endif

template <typename T>
WCNS_HD T flux_difference(T f0, T f1, T f2, T f3, T f4, T f5, T inv_h) {
  const T d1 = T(75.0 / 64.0), d2 = T(-25.0 / 384.0), d3 = T(3.0 / 640.0);
  T acc = smul<T>(d1, f3 - f2);
  acc = sfma<T>(d2, f4 - f1, acc);
  acc = sfma<T>(d3, f5 - f0, acc);
  return -smul<T>(acc, inv_h);
}

// Spatial derivative from the six interface fluxes f[0..5] = F_{i-5/2} .. F_{i+5/2}:
// Eq. 3 for the WCNS family, -(F_{i+1/2} - F_{i-1/2}) / h for the WENO family (App. B).
template <typename T>
WCNS_HD T flux_difference_family(int family, T f0, T f1, T f2, T f3, T f4, T f5, T inv_h) {
  if (family == 1) return -smul<T>(f3 - f2, inv_h);
  return flux_difference<T>(f0, f1, f2, f3, f4, f5, inv_h);
}

WCNS_HD int64_t ghost(int64_t i, int64_t n, int bc) {
  if (i >= 0 && i < n) return i;
  if (bc == 0) {
    int64_t r = i % n;
    return r < 0 ? r + n : r;
  }
  return i < 0 ? 0 : n - 1;
}

// Double-precision a + b * c rounded in two steps (no contraction), as the positions of
// ghost cells and of the moving shock are formed.
WCNS_HD double add_mul_rn(double a, double b, double c) {
#ifdef __CUDA_ARCH__
  return __dadd_rn(a, __dmul_rn(b, c));
#else
  return a + b * c;
#endif
}

// Storage component v of cell m (possibly outside [0, n)) of sweep line `line` in
// direction dir, with the face rules for ghost cells; `time` is the time of the state
// (moving-shock faces).
template <typename T>
WCNS_HD T face_cell(const T* u, int64_t pitch, int64_t fstride, int dir, int64_t line, int64_t m, int64_t n, int bc,
                    int v, const Faces<T>& f, double time) {
  const int64_t base = (int64_t)v * fstride;
  if (!f.active || (m >= 0 && m < n)) {
    const int64_t mm = ghost(m, n, bc);
    return dir == 0 ? u[base + line * pitch + mm] : u[base + mm * pitch + line];
  }
  int type = f.type[2 * dir + (m < 0 ? 0 : 1)];
  if (type == kFaceGrid || type == kFaceTransmissive) {
    const int64_t mm = ghost(m, n, type == kFaceGrid ? bc : 1);
    return dir == 0 ? u[base + line * pitch + mm] : u[base + mm * pitch + line];
  }
  const double x = add_mul_rn(f.lo_x, double(dir == 0 ? m : line) + 0.5, f.hx);
  const double y = add_mul_rn(f.lo_y, double(dir == 0 ? line : m) + 0.5, f.hy);
  if (type == kFaceFixedThenWall) type = (x < f.wall_x) ? kFaceFixed : kFaceWall;
  if (type == kFaceWall) {
    const int64_t mm = m < 0 ? -1 - m : 2 * n - 1 - m;
    const T val = dir == 0 ? u[base + line * pitch + mm] : u[base + mm * pitch + line];
    return (v == 1 + dir) ? -val : val;
  }
  if (type == kFaceShock)
    return (x < add_mul_rn(f.x0, add_mul_rn(y, f.speed, time), f.dxdy)) ? f.ua[v] : f.ub[v];
  return f.ua[v];
}

}  // namespace wcns
