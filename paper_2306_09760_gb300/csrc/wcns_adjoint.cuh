// Hand-written reverse mode of the interface flux (vector-Jacobian products).
//
// Forward (see wcns_device.cuh): six stencil states S -> Roe average -> eigenvector
// basis -> characteristic projection W (a1) -> per field and side: Eq. 5 values, Eq. 9-10
// smoothness indicators, Eq. 11 / Eq. 14-15 weights, Eq. 20 map and renormalisation,
// Eq. 6 combination (b1-b5) -> back-projection -> Lax-Friedrichs flux with a frozen
// dissipation speed (c).  The reverse sweep below differentiates exactly these steps,
// in reverse order, with the same branch decisions (saturated tanh, PFE box,
// positivity fallback).  Supported options: weights JS, Z, FE, PFE (Z exponent 1 or
// 2, with or without renormalisation), characteristic projection on or off, flux
// LLF_FROZEN.  |IS_0 - IS_2| uses sign(0) = 0.
#pragma once

#include "wcns_device.cuh"

namespace wcns {

// d/dw of Eq. 20 for one weight: the map is w + 1/2 sum_j a_j(w) tanh(xi (w - n_j)) with
// a_1 = c_1 - w, a_J = w - c_{J-1} and constant middle amplitudes.
template <typename T>
WCNS_HD T tanh_sat_d(T z, T& t) {
  T a = Num<T>::abs_(z);
  if (a >= Num<T>::kSat) {
    t = z > T(0) ? T(1) : T(-1);
    return T(0);
  }
  t = Num<T>::tanh_(z);
  return T(1) - t * t;
}

template <typename T>
WCNS_HD T fe_map0_d(T w, const SchemeT<T>& s) {
  const T xi = s.xi;
  T t1, t2, t3;
  T e1 = tanh_sat_d<T>(xi * (w - s.null0[0]), t1);
  T e2 = tanh_sat_d<T>(xi * (w - s.null0[1]), t2);
  T e3 = tanh_sat_d<T>(xi * (w - s.null0[2]), t3);
  T acc = -t1 + (T(1.0 / 16.0) - w) * xi * e1;
  acc = acc + T(1.0 / 6.0 - 1.0 / 16.0) * xi * e2;
  acc = acc + t3 + (w - T(1.0 / 6.0)) * xi * e3;
  return T(1) + acc / T(2);
}
template <typename T>
WCNS_HD T fe_map1_d(T w, const SchemeT<T>& s) {
  const T xi = s.xi;
  T t1, t2, t3, t4;
  T e1 = tanh_sat_d<T>(xi * (w - s.null1[0]), t1);
  T e2 = tanh_sat_d<T>(xi * (w - s.null1[1]), t2);
  T e3 = tanh_sat_d<T>(xi * (w - s.null1[2]), t3);
  T e4 = tanh_sat_d<T>(xi * (w - s.null1[3]), t4);
  T acc = -t1 + (T(10.0 / 16.0) - w) * xi * e1;
  acc = acc + T(1.0 / 2.0 - 10.0 / 16.0) * xi * e2;
  acc = acc + T(5.0 / 6.0 - 1.0 / 2.0) * xi * e3;
  acc = acc + t4 + (w - T(5.0 / 6.0)) * xi * e4;
  return T(1) + acc / T(2);
}
template <typename T>
WCNS_HD T fe_map2_d(T w, const SchemeT<T>& s) {
  const T xi = s.xi;
  T t1, t2, t3;
  T e1 = tanh_sat_d<T>(xi * (w - s.null2[0]), t1);
  T e2 = tanh_sat_d<T>(xi * (w - s.null2[1]), t2);
  T e3 = tanh_sat_d<T>(xi * (w - s.null2[2]), t3);
  T acc = -t1 + (T(5.0 / 16.0) - w) * xi * e1;
  acc = acc + T(1.0 / 2.0 - 5.0 / 16.0) * xi * e2;
  acc = acc + t3 + (w - T(1.0 / 2.0)) * xi * e3;
  return T(1) + acc / T(2);
}

// Reverse of weno_side: given the cotangent gv of the interpolated value, adds the
// cotangents of the five inputs to dv[0..4].
template <typename T>
WCNS_HD void weno_side_vjp(const T (&v)[5], T gv, const SchemeT<T>& s, T (&dv)[5]) {
  const T d[3] = {T(1.0 / 16.0), T(10.0 / 16.0), T(5.0 / 16.0)};
  // ---- forward, keeping what the reverse needs
  T q[3], f[3], sm[3], IS[3];
  q[0] = (T(3) * v[0] - T(10) * v[1] + T(15) * v[2]) / T(8);
  q[1] = (-v[1] + T(6) * v[2] + T(3) * v[3]) / T(8);
  q[2] = (T(3) * v[2] + T(6) * v[3] - v[4]) / T(8);
  f[0] = (v[0] - T(4) * v[1] + T(3) * v[2]) / T(2); sm[0] = v[0] - T(2) * v[1] + v[2];
  f[1] = (v[3] - v[1]) / T(2);                      sm[1] = v[1] - T(2) * v[2] + v[3];
  f[2] = (T(-3) * v[2] + T(4) * v[3] - v[4]) / T(2); sm[2] = v[2] - T(2) * v[3] + v[4];
  #pragma unroll
  for (int k = 0; k < 3; ++k) IS[k] = f[k] * f[k] + sm[k] * sm[k];
  const T eps = s.eps;
  T w[3], om[3], alpha[3], A = T(0), r[3] = {T(0), T(0), T(0)}, tau = T(0), sgn = T(0);
  T G = T(1);
  bool mapped = false;
  const bool js = (s.weights == 0);
  if (js) {
    #pragma unroll
    for (int k = 0; k < 3; ++k) {
      T b = IS[k] + eps;
      alpha[k] = d[k] / (b * b);
      A = A + alpha[k];
    }
  } else {
    T diff = IS[0] - IS[2];
    tau = Num<T>::abs_(diff);
    sgn = diff > T(0) ? T(1) : (diff < T(0) ? T(-1) : T(0));
    #pragma unroll
    for (int k = 0; k < 3; ++k) {
      r[k] = tau / (IS[k] + eps);
      T rp = (s.zp == 2) ? r[k] * r[k] : r[k];
      alpha[k] = d[k] * (T(1) + rp);
      A = A + alpha[k];
    }
  }
  #pragma unroll
  for (int k = 0; k < 3; ++k) om[k] = alpha[k] / A;
  T g[3] = {om[0], om[1], om[2]};
  if (s.weights == 2 || s.weights == 3) {
    bool keep = false;
    if (s.weights == 3) {
      keep = true;
      #pragma unroll
      for (int k = 0; k < 3; ++k) keep = keep && (om[k] >= d[k] - s.cv) && (om[k] <= d[k] + s.cv);
    }
    if (!keep) {
      mapped = true;
      g[0] = fe_map0<T>(om[0], s);
      g[1] = fe_map1<T>(om[1], s);
      g[2] = fe_map2<T>(om[2], s);
    }
  }
  if (mapped && s.renorm) {
    G = g[0] + g[1] + g[2];
    #pragma unroll
    for (int k = 0; k < 3; ++k) w[k] = g[k] / G;
  } else {
    #pragma unroll
    for (int k = 0; k < 3; ++k) w[k] = g[k];
  }
  // ---- reverse
  T qb[3], wb[3];
  #pragma unroll
  for (int k = 0; k < 3; ++k) { wb[k] = gv * q[k]; qb[k] = gv * w[k]; }
  T gb[3];
  if (mapped && s.renorm) {
    T dotw = wb[0] * w[0] + wb[1] * w[1] + wb[2] * w[2];
    #pragma unroll
    for (int k = 0; k < 3; ++k) gb[k] = (wb[k] - dotw) / G;
  } else {
    #pragma unroll
    for (int k = 0; k < 3; ++k) gb[k] = wb[k];
  }
  T omb[3];
  if (mapped) {
    omb[0] = gb[0] * fe_map0_d<T>(om[0], s);
    omb[1] = gb[1] * fe_map1_d<T>(om[1], s);
    omb[2] = gb[2] * fe_map2_d<T>(om[2], s);
  } else {
    #pragma unroll
    for (int k = 0; k < 3; ++k) omb[k] = gb[k];
  }
  T doto = omb[0] * om[0] + omb[1] * om[1] + omb[2] * om[2];
  T ab[3];
  #pragma unroll
  for (int k = 0; k < 3; ++k) ab[k] = (omb[k] - doto) / A;
  T ISb[3] = {T(0), T(0), T(0)};
  if (js) {
    #pragma unroll
    for (int k = 0; k < 3; ++k) ISb[k] = T(-2) * ab[k] * alpha[k] / (IS[k] + eps);
  } else {
    T taub = T(0);
    #pragma unroll
    for (int k = 0; k < 3; ++k) {
      T rpb = ab[k] * d[k];
      T rb = (s.zp == 2) ? rpb * T(2) * r[k] : rpb;
      T inv = T(1) / (IS[k] + eps);
      taub = taub + rb * inv;
      ISb[k] = ISb[k] - rb * r[k] * inv;
    }
    ISb[0] = ISb[0] + taub * sgn;
    ISb[2] = ISb[2] - taub * sgn;
  }
  T fb[3], sb[3];
  #pragma unroll
  for (int k = 0; k < 3; ++k) { fb[k] = T(2) * f[k] * ISb[k]; sb[k] = T(2) * sm[k] * ISb[k]; }
  dv[0] = dv[0] + T(3.0 / 8.0) * qb[0] + T(0.5) * fb[0] + sb[0];
  dv[1] = dv[1] - T(10.0 / 8.0) * qb[0] - T(1.0 / 8.0) * qb[1] - T(2) * fb[0] - T(2) * sb[0] - T(0.5) * fb[1] + sb[1];
  dv[2] = dv[2] + T(15.0 / 8.0) * qb[0] + T(6.0 / 8.0) * qb[1] + T(3.0 / 8.0) * qb[2] + T(1.5) * fb[0] + sb[0] -
          T(2) * sb[1] - T(1.5) * fb[2] + sb[2];
  dv[3] = dv[3] + T(3.0 / 8.0) * qb[1] + T(6.0 / 8.0) * qb[2] + T(0.5) * fb[1] + sb[1] + T(2) * fb[2] - T(2) * sb[2];
  dv[4] = dv[4] - T(1.0 / 8.0) * qb[2] - T(0.5) * fb[2] + sb[2];
}

// Reverse of the physical flux F(U) in the sweep normal: adds (dF/dU)^T Fb to Ub.
template <typename T, int NV>
WCNS_HD void euler_flux_vjp(const T (&U)[NV], T gm1, const T (&Fb)[NV], T (&Ub)[NV]) {
  const T rho = U[0], m = U[1];
  const T n = (NV == 4) ? U[2] : T(0);
  const T E = U[NV - 1];
  const T inv = T(1) / rho;
  const T un = m * inv, ut = n * inv;
  const T p = gm1 * (E - T(0.5) * (m * m + n * n) * inv);
  const T H = (E + p) * inv;
  T rb = T(0), mb = Fb[0], nb = T(0), Eb = T(0), pb = T(0);
  // F1 = m un + p
  mb = mb + Fb[1] * T(2) * un;
  rb = rb - Fb[1] * un * un;
  pb = pb + Fb[1];
  if (NV == 4) {
    // F2 = n un
    nb = nb + Fb[2] * un;
    mb = mb + Fb[2] * ut;
    rb = rb - Fb[2] * un * ut;
  }
  // F_E = (E + p) un
  const T FEb = Fb[NV - 1];
  Eb = Eb + FEb * un;
  pb = pb + FEb * un;
  mb = mb + FEb * H;
  rb = rb - FEb * H * un;
  // p = gm1 (E - (m^2 + n^2) / (2 rho))
  Eb = Eb + gm1 * pb;
  mb = mb - gm1 * un * pb;
  nb = nb - gm1 * ut * pb;
  rb = rb + gm1 * T(0.5) * (un * un + ut * ut) * pb;
  Ub[0] = Ub[0] + rb;
  Ub[1] = Ub[1] + mb;
  if (NV == 4) Ub[2] = Ub[2] + nb;
  Ub[NV - 1] = Ub[NV - 1] + Eb;
}

// Cotangents of the characteristic basis (u, v, H, c) and of the derived quantities.
template <typename T>
struct BasisBar {
  T u, v, H, c, b, ic, hq2;
};

// Reverse of char_unproject: U = R(cb) W.
template <typename T, int NV>
WCNS_HD void char_unproject_vjp(const CharBasis<T, NV>& cb, const T (&W)[NV], const T (&Ub)[NV], T (&Wb)[NV],
                                BasisBar<T>& bb) {
  const T wa = W[0], wb = W[1], wd = W[NV - 1];
  const T sum = wa + wb + wd, dl = wd - wa;
  const T U2b = (NV == 4) ? Ub[2] : T(0);
  const T W2 = (NV == 4) ? W[2] : T(0);
  const T UEb = Ub[NV - 1];
  T sb = Ub[0] + cb.u * Ub[1] + cb.v * U2b;
  T dlb = cb.c * Ub[1] + cb.u * cb.c * UEb;
  Wb[0] = sb - dlb + cb.H * UEb;
  Wb[1] = sb + cb.hq2 * UEb;
  if (NV == 4) Wb[2] = U2b + cb.v * UEb;
  Wb[NV - 1] = sb + dlb + cb.H * UEb;
  bb.u = bb.u + sum * Ub[1] + cb.c * dl * UEb;
  bb.c = bb.c + dl * Ub[1] + cb.u * dl * UEb;
  bb.v = bb.v + sum * U2b + W2 * UEb;
  bb.H = bb.H + (wa + wd) * UEb;
  bb.hq2 = bb.hq2 + wb * UEb;
}

// Reverse of char_project for one cell: W = L(cb) U.  Adds to Ub and bb.
template <typename T, int NV>
WCNS_HD void char_project_vjp(const CharBasis<T, NV>& cb, const T (&U)[NV], const T (&Wb)[NV], T (&Ub)[NV],
                              BasisBar<T>& bb) {
  const T rho = U[0], m = U[1];
  const T n = (NV == 4) ? U[2] : T(0);
  const T E = U[NV - 1];
  const T X = E - cb.u * m - cb.v * n + cb.hq2 * rho;
  const T Pb = T(0.5) * Wb[0] - Wb[1] + T(0.5) * Wb[NV - 1];
  const T Ab = T(0.5) * Wb[0] - T(0.5) * Wb[NV - 1];
  T rb = Wb[1], nb = T(0);
  if (NV == 4) {
    rb = rb - cb.v * Wb[2];
    nb = Wb[2];
    bb.v = bb.v - rho * Wb[2];
  }
  bb.b = bb.b + X * Pb;
  const T Xb = cb.b * Pb;
  T Eb = Xb;
  T mb = -cb.u * Xb;
  nb = nb - cb.v * Xb;
  rb = rb + cb.hq2 * Xb;
  bb.u = bb.u - m * Xb;
  bb.v = bb.v - n * Xb;
  bb.hq2 = bb.hq2 + rho * Xb;
  // A = (u rho - m) ic
  bb.u = bb.u + rho * cb.ic * Ab;
  rb = rb + cb.u * cb.ic * Ab;
  mb = mb - cb.ic * Ab;
  bb.ic = bb.ic + (cb.u * rho - m) * Ab;
  Ub[0] = Ub[0] + rb;
  Ub[1] = Ub[1] + mb;
  if (NV == 4) Ub[2] = Ub[2] + nb;
  Ub[NV - 1] = Ub[NV - 1] + Eb;
}

// Reverse of (primitive states of U_i, U_{i+1}) -> Roe average -> basis.  Adds to Sb2, Sb3.
template <typename T, int NV>
WCNS_HD void roe_basis_vjp(const T (&Ua)[NV], const T (&Ub_)[NV], T gm1, const BasisBar<T>& bbin, T (&Sa)[NV],
                           T (&Sb)[NV]) {
  EulerState<T, NV> a = euler_prim<T, NV>(Ua, gm1), b = euler_prim<T, NV>(Ub_, gm1);
  RoeAvg<T, NV> r = roe_avg<T, NV>(a, b, gm1);
  BasisBar<T> bb = bbin;
  const T ic = T(1) / r.c;
  // b = gm1 ic^2, hq2 = (u^2 + v^2)/2, ic = 1/c
  bb.ic = bb.ic + bb.b * gm1 * T(2) * ic;
  bb.u = bb.u + bb.hq2 * r.u;
  bb.v = bb.v + bb.hq2 * r.v;
  bb.c = bb.c - bb.ic * ic * ic;
  // c = sqrt(gm1 (H - (u^2 + v^2)/2))
  const T c2b = bb.c / (T(2) * r.c);
  bb.H = bb.H + gm1 * c2b;
  bb.u = bb.u - gm1 * r.u * c2b;
  bb.v = bb.v - gm1 * r.v * c2b;
  // u = (sa ua + sb ub)/(sa + sb), same for v and H
  const T sa = Num<T>::sqrt_(a.rho), sb = Num<T>::sqrt_(b.rho);
  const T inv = T(1) / (sa + sb);
  T uab = bb.u * sa * inv, ubb = bb.u * sb * inv;
  T vab = bb.v * sa * inv, vbb = bb.v * sb * inv;
  T Hab = bb.H * sa * inv, Hbb = bb.H * sb * inv;
  T sab = (bb.u * (a.un - r.u) + bb.v * (a.ut - r.v) + bb.H * (a.H - r.H)) * inv;
  T sbb = (bb.u * (b.un - r.u) + bb.v * (b.ut - r.v) + bb.H * (b.H - r.H)) * inv;
  if (NV != 4) { vab = T(0); vbb = T(0); }
  // primitives -> conservative for each state
  auto prim_vjp = [&](const T (&U)[NV], const EulerState<T, NV>& st, T sqrt_rho, T unb, T utb, T Hb, T sqb,
                      T (&Ux)[NV]) {
    const T inv_r = T(1) / st.rho;
    T rb = sqb / (T(2) * sqrt_rho);
    // H = (E + p)/rho
    T Eb = Hb * inv_r;
    T pb = Hb * inv_r;
    rb = rb - Hb * st.H * inv_r;
    // p = gm1 (E - (m^2 + n^2)/(2 rho))
    Eb = Eb + gm1 * pb;
    T mb = -gm1 * st.un * pb;
    T nb = -gm1 * st.ut * pb;
    rb = rb + gm1 * T(0.5) * (st.un * st.un + st.ut * st.ut) * pb;
    // un = m / rho, ut = n / rho
    mb = mb + unb * inv_r;
    rb = rb - unb * st.un * inv_r;
    nb = nb + utb * inv_r;
    rb = rb - utb * st.ut * inv_r;
    Ux[0] = Ux[0] + rb;
    Ux[1] = Ux[1] + mb;
    if (NV == 4) Ux[2] = Ux[2] + nb;
    Ux[NV - 1] = Ux[NV - 1] + Eb;
    (void)U;
  };
  prim_vjp(Ua, a, sa, uab, vab, Hab, sab, Sa);
  prim_vjp(Ub_, b, sb, ubb, vbb, Hbb, sbb, Sb);
}

// Reverse of interface_flux for LLF_FROZEN: Sb[m][k] += d(F . Fb)/d S[m][k].
template <typename T, int NV>
WCNS_HD void interface_flux_vjp(const T (&S)[6][NV], const SchemeT<T>& s, int dir, const T (&Fb)[NV],
                                T (&Sb)[6][NV]) {
  const T gm1 = s.gm1;
  const T alpha = s.speed[dir];
  // ---- forward to the interpolated states
  T UL[NV], UR[NV];
  CharBasis<T, NV> cb{};
  T WL[NV], WR[NV];
  const bool ch = s.characteristic != 0;
  if (ch) {
    T Ui[NV], Uj[NV];
    #pragma unroll
    for (int k = 0; k < NV; ++k) { Ui[k] = S[2][k]; Uj[k] = S[3][k]; }
    EulerState<T, NV> a = euler_prim<T, NV>(Ui, gm1), b = euler_prim<T, NV>(Uj, gm1);
    RoeAvg<T, NV> r = roe_avg<T, NV>(a, b, gm1);
    cb = char_basis<T, NV>(r, gm1);
    T W[6][NV];
    #pragma unroll
    for (int m = 0; m < 6; ++m) char_project<T, NV>(cb, S[m], W[m]);
    #pragma unroll
    for (int k = 0; k < NV; ++k) {
      WL[k] = weno_side<T, 0>(W[0][k], W[1][k], W[2][k], W[3][k], W[4][k], s);
      WR[k] = weno_side<T, 0>(W[5][k], W[4][k], W[3][k], W[2][k], W[1][k], s);
    }
    char_unproject<T, NV>(cb, WL, UL);
    char_unproject<T, NV>(cb, WR, UR);
  } else {
    #pragma unroll
    for (int k = 0; k < NV; ++k) {
      UL[k] = weno_side<T, 0>(S[0][k], S[1][k], S[2][k], S[3][k], S[4][k], s);
      UR[k] = weno_side<T, 0>(S[5][k], S[4][k], S[3][k], S[2][k], S[1][k], s);
    }
  }
  const bool fallback = !physical<T, NV>(UL, gm1) || !physical<T, NV>(UR, gm1);
  if (fallback) {
    #pragma unroll
    for (int k = 0; k < NV; ++k) { UL[k] = S[2][k]; UR[k] = S[3][k]; }
  }
  // ---- reverse of F = (F(UL) + F(UR))/2 - alpha (UR - UL)/2
  T ULb[NV], URb[NV], half[NV];
  #pragma unroll
  for (int k = 0; k < NV; ++k) {
    half[k] = T(0.5) * Fb[k];
    ULb[k] = T(0.5) * alpha * Fb[k];
    URb[k] = -T(0.5) * alpha * Fb[k];
  }
  euler_flux_vjp<T, NV>(UL, gm1, half, ULb);
  euler_flux_vjp<T, NV>(UR, gm1, half, URb);
  if (fallback) {
    #pragma unroll
    for (int k = 0; k < NV; ++k) { Sb[2][k] = Sb[2][k] + ULb[k]; Sb[3][k] = Sb[3][k] + URb[k]; }
    return;
  }
  if (!ch) {
    #pragma unroll
    for (int k = 0; k < NV; ++k) {
      T dv[5] = {T(0), T(0), T(0), T(0), T(0)};
      T v[5] = {S[0][k], S[1][k], S[2][k], S[3][k], S[4][k]};
      weno_side_vjp<T>(v, ULb[k], s, dv);
      #pragma unroll
      for (int m = 0; m < 5; ++m) Sb[m][k] = Sb[m][k] + dv[m];
      T dw[5] = {T(0), T(0), T(0), T(0), T(0)};
      T w[5] = {S[5][k], S[4][k], S[3][k], S[2][k], S[1][k]};
      weno_side_vjp<T>(w, URb[k], s, dw);
      #pragma unroll
      for (int m = 0; m < 5; ++m) Sb[5 - m][k] = Sb[5 - m][k] + dw[m];
    }
    return;
  }
  BasisBar<T> bb{T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
  T WLb[NV], WRb[NV];
  char_unproject_vjp<T, NV>(cb, WL, ULb, WLb, bb);
  char_unproject_vjp<T, NV>(cb, WR, URb, WRb, bb);
  // recompute the projected stencil (cheaper than keeping it live)
  T W[6][NV];
  #pragma unroll
  for (int m = 0; m < 6; ++m) char_project<T, NV>(cb, S[m], W[m]);
  T Wb[6][NV];
  #pragma unroll
  for (int m = 0; m < 6; ++m)
    #pragma unroll
    for (int k = 0; k < NV; ++k) Wb[m][k] = T(0);
  #pragma unroll
  for (int k = 0; k < NV; ++k) {
    T dv[5] = {T(0), T(0), T(0), T(0), T(0)};
    T v[5] = {W[0][k], W[1][k], W[2][k], W[3][k], W[4][k]};
    weno_side_vjp<T>(v, WLb[k], s, dv);
    #pragma unroll
    for (int m = 0; m < 5; ++m) Wb[m][k] = Wb[m][k] + dv[m];
    T dw[5] = {T(0), T(0), T(0), T(0), T(0)};
    T w[5] = {W[5][k], W[4][k], W[3][k], W[2][k], W[1][k]};
    weno_side_vjp<T>(w, WRb[k], s, dw);
    #pragma unroll
    for (int m = 0; m < 5; ++m) Wb[5 - m][k] = Wb[5 - m][k] + dw[m];
  }
  #pragma unroll
  for (int m = 0; m < 6; ++m) char_project_vjp<T, NV>(cb, S[m], Wb[m], Sb[m], bb);
  T Ui[NV], Uj[NV];
  #pragma unroll
  for (int k = 0; k < NV; ++k) { Ui[k] = S[2][k]; Uj[k] = S[3][k]; }
  roe_basis_vjp<T, NV>(Ui, Uj, gm1, bb, Sb[2], Sb[3]);
}

}  // namespace wcns
