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

// tanh(z) in t and its derivative 1 - t^2 as the return value, with the exact select
// where tanh rounds to +-1 (the derivative is then 0).
template <typename T>
WCNS_HD T tanh_sat_d(T z, T& t) {
  if (Num<T>::abs_(z) >= Num<T>::kSat) {
    t = z > T(0) ? T(1) : T(-1);
    return T(0);
  }
  t = Num<T>::tanh_(z);
  return T(1) - t * t;
}

// Eq. 20 for one weight together with its derivative.  With amplitudes a_1 = (c_1 - w)/2,
// a_j = (c_j - c_{j-1})/2 in the middle and a_J = (w - c_{J-1})/2 the map is
//   g(w) = w + sum_j a_j tanh(xi (w - n_j)),
// so g'(w) = 1 + (t_J - t_1)/2 + xi sum_j a_j (1 - t_j^2) with t_j the tanh terms.  Each
// term is evaluated once and serves both.  The value is the forward map's (fe_map0..2):
// the exponential form of tanh in single precision at moderate xi, otherwise tanh with
// the exact select where it rounds to +-1 (there the term's derivative is 0; where every
// term is saturated this is the forward map's staircase, with slope 0 or 1).
template <typename T, int K>
WCNS_HD T fe_map_vd(T w, const T (&n)[K], const T (&c)[K - 1], const SchemeT<T>& s, T& dg) {
  T amp[K];
  amp[0] = (c[0] - w) / T(2);
#pragma unroll
  for (int j = 1; j < K - 1; ++j) amp[j] = (c[j] - c[j - 1]) / T(2);
  amp[K - 1] = (w - c[K - 2]) / T(2);
  bool expf_form = false;
  if constexpr (sizeof(T) == 4) expf_form = s.xi_small != 0;
  T acc = T(0), dacc = T(0), t_first = T(0), t_last = T(0);
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const T z = s.xi * (w - n[j]);
    T t, e;
    if constexpr (sizeof(T) == 4) {
      if (expf_form) {
        t = tanh_expf(z);
        e = T(1) - t * t;
      } else {
        e = tanh_sat_d<T>(z, t);
      }
    } else {
      e = tanh_sat_d<T>(z, t);
    }
    acc = acc + amp[j] * t;
    dacc = dacc + amp[j] * e;
    if (j == 0) t_first = t;
    if (j == K - 1) t_last = t;
  }
  dg = T(1) + (t_last - t_first) / T(2) + s.xi * dacc;
  return acc + w;
}

// One-sided interpolation and its gradient: the value of weno_side (WCNS family; JS,
// Z with p = 1 or 2, FE and PFE weights, with or without renormalisation) from the five
// inputs v, and d(value)/d v_m in gr[m].  Forward: Eq. 5 values, Eq. 9-10 indicators,
// Eq. 11 or Eq. 14-15 weights, the App. A box, the Eq. 20 map and its renormalisation,
// the Eq. 6 combination, with the forward's ideal-plateau tests (where they hold the
// weights are the ideal ones and the map is flat, so only the Eq. 5 values carry
// derivatives).  Reverse: the same steps backwards from a unit seed on the value.
template <typename T>
WCNS_HD T weno_side_grad(const T (&v)[5], const SchemeT<T>& s, T (&gr)[5]) {
  const T d[3] = {T(1.0 / 16.0), T(10.0 / 16.0), T(5.0 / 16.0)};
  // ---- forward, keeping what the reverse needs
  T q[3], f[3], sm[3], IS[3];
  q[0] = T(0.375) * v[0] - T(1.25) * v[1] + T(1.875) * v[2];
  q[1] = -T(0.125) * v[1] + T(0.75) * v[2] + T(0.375) * v[3];
  q[2] = T(0.375) * v[2] + T(0.75) * v[3] - T(0.125) * v[4];
  f[0] = (v[0] - T(4) * v[1] + T(3) * v[2]) / T(2); sm[0] = v[0] - T(2) * v[1] + v[2];
  f[1] = (v[3] - v[1]) / T(2);                      sm[1] = v[1] - T(2) * v[2] + v[3];
  f[2] = (T(-3) * v[2] + T(4) * v[3] - v[4]) / T(2); sm[2] = v[2] - T(2) * v[3] + v[4];
#pragma unroll
  for (int k = 0; k < 3; ++k) IS[k] = f[k] * f[k] + sm[k] * sm[k];
  const T eps = s.eps;
  const bool js = (s.weights == 0);
  T b[3], om[3], alpha[3], r[3] = {T(0), T(0), T(0)}, inv[3] = {T(0), T(0), T(0)};
  T A = T(0), sgn = T(0), tau = T(0);
  bool plateau = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) b[k] = IS[k] + eps;
  if (js) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      alpha[k] = Num<T>::div_(d[k], b[k] * b[k]);
      A = A + alpha[k];
    }
  } else {
    const T diff = IS[0] - IS[2];
    tau = Num<T>::abs_(diff);
    sgn = diff > T(0) ? T(1) : (diff < T(0) ? T(-1) : T(0));
    bool small = s.weights == 2;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      inv[k] = Num<T>::rcp_(b[k]);
      r[k] = Num<T>::z_ratio(tau, b[k]);
      const T rp = (s.zp == 2) ? r[k] * r[k] : r[k];
      small = small && rp < s.ideal_ratio;
      alpha[k] = d[k] * (T(1) + rp);
      A = A + alpha[k];
    }
    plateau = small;
  }
  const T iA = Num<T>::rcp_(A);
#pragma unroll
  for (int k = 0; k < 3; ++k) om[k] = alpha[k] * iA;
  if (s.weights == 2 && s.ideal_margin[0] > T(0) && Num<T>::abs_(om[0] - d[0]) < s.ideal_margin[0] &&
      Num<T>::abs_(om[1] - d[1]) < s.ideal_margin[1] && Num<T>::abs_(om[2] - d[2]) < s.ideal_margin[2])
    plateau = true;
  T w[3] = {om[0], om[1], om[2]}, dg[3] = {T(1), T(1), T(1)}, iG = T(1);
  bool mapped = false;
  if (plateau) {
#pragma unroll
    for (int k = 0; k < 3; ++k) w[k] = d[k];
  } else if (s.weights == 2 || s.weights == 3) {
    bool keep = false;
    if (s.weights == 3) {
      keep = true;
#pragma unroll
      for (int k = 0; k < 3; ++k) keep = keep && (om[k] >= d[k] - s.cv) && (om[k] <= d[k] + s.cv);
    }
    if (!keep) {
      mapped = true;
      w[0] = fe_map_vd<T, 3>(om[0], s.null0, s.ctrl0, s, dg[0]);
      w[1] = fe_map_vd<T, 4>(om[1], s.null1, s.ctrl1, s, dg[1]);
      w[2] = fe_map_vd<T, 3>(om[2], s.null2, s.ctrl2, s, dg[2]);
      if (s.renorm) {
        iG = Num<T>::rcp_(w[0] + w[1] + w[2]);
#pragma unroll
        for (int k = 0; k < 3; ++k) w[k] = w[k] * iG;
      }
    }
  }
  const T value = w[0] * q[0] + w[1] * q[1] + w[2] * q[2];
  // ---- reverse from a unit seed: qb = w, wb = q
  T ISb[3] = {T(0), T(0), T(0)};
  if (!plateau) {
    T gb[3];
    if (mapped && s.renorm) {
      const T dotw = q[0] * w[0] + q[1] * w[1] + q[2] * w[2];
#pragma unroll
      for (int k = 0; k < 3; ++k) gb[k] = (q[k] - dotw) * iG;
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k) gb[k] = q[k];
    }
    T omb[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) omb[k] = mapped ? gb[k] * dg[k] : gb[k];
    const T doto = omb[0] * om[0] + omb[1] * om[1] + omb[2] * om[2];
    T ab[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) ab[k] = (omb[k] - doto) * iA;
    if (js) {
#pragma unroll
      for (int k = 0; k < 3; ++k) ISb[k] = Num<T>::div_(T(-2) * ab[k] * alpha[k], b[k]);
    } else {
      T taub = T(0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const T rpb = ab[k] * d[k];
        const T rb = (s.zp == 2) ? rpb * T(2) * r[k] : rpb;
        taub = taub + rb * inv[k];
        ISb[k] = -rb * r[k] * inv[k];
      }
      ISb[0] = ISb[0] + taub * sgn;
      ISb[2] = ISb[2] - taub * sgn;
    }
  }
  const T qb0 = w[0], qb1 = w[1], qb2 = w[2];
  T fb[3], sb[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) { fb[k] = T(2) * f[k] * ISb[k]; sb[k] = T(2) * sm[k] * ISb[k]; }
  gr[0] = T(3.0 / 8.0) * qb0 + T(0.5) * fb[0] + sb[0];
  gr[1] = -T(10.0 / 8.0) * qb0 - T(1.0 / 8.0) * qb1 - T(2) * fb[0] - T(2) * sb[0] - T(0.5) * fb[1] + sb[1];
  gr[2] = T(15.0 / 8.0) * qb0 + T(6.0 / 8.0) * qb1 + T(3.0 / 8.0) * qb2 + T(1.5) * fb[0] + sb[0] - T(2) * sb[1] -
          T(1.5) * fb[2] + sb[2];
  gr[3] = T(3.0 / 8.0) * qb1 + T(6.0 / 8.0) * qb2 + T(0.5) * fb[1] + sb[1] + T(2) * fb[2] - T(2) * sb[2];
  gr[4] = -T(1.0 / 8.0) * qb2 - T(0.5) * fb[2] + sb[2];
  return value;
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

// Reverse of interface_flux for LLF_FROZEN: Sb[m][k] += d(F . Fb)/d S[m][k].  The forward
// pass keeps, for each field and side, the gradient of the interpolated value with
// respect to its five inputs (weno_side_grad), so the reverse needs no second pass
// through the weights.
template <typename T, int NV>
WCNS_HD void interface_flux_vjp(const T (&S)[6][NV], const SchemeT<T>& s, int dir, const T (&Fb)[NV],
                                T (&Sb)[6][NV]) {
  const T gm1 = s.gm1;
  const T alpha = s.speed[dir];
  // ---- forward to the interpolated states
  T UL[NV], UR[NV];
  CharBasis<T, NV> cb{};
  T WL[NV], WR[NV];
  T gL[NV][5], gR[NV][5];  // gL[k][m]: d WL_k / d v_m (v = cells i-2..i+2); gR: mirrored cells i+3..i-1
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
      const T vl[5] = {W[0][k], W[1][k], W[2][k], W[3][k], W[4][k]};
      const T vr[5] = {W[5][k], W[4][k], W[3][k], W[2][k], W[1][k]};
      WL[k] = weno_side_grad<T>(vl, s, gL[k]);
      WR[k] = weno_side_grad<T>(vr, s, gR[k]);
    }
    char_unproject<T, NV>(cb, WL, UL);
    char_unproject<T, NV>(cb, WR, UR);
  } else {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const T vl[5] = {S[0][k], S[1][k], S[2][k], S[3][k], S[4][k]};
      const T vr[5] = {S[5][k], S[4][k], S[3][k], S[2][k], S[1][k]};
      UL[k] = weno_side_grad<T>(vl, s, gL[k]);
      UR[k] = weno_side_grad<T>(vr, s, gR[k]);
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
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        Sb[m][k] = Sb[m][k] + ULb[k] * gL[k][m];
        Sb[5 - m][k] = Sb[5 - m][k] + URb[k] * gR[k][m];
      }
    return;
  }
  BasisBar<T> bb{T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
  T WLb[NV], WRb[NV];
  char_unproject_vjp<T, NV>(cb, WL, ULb, WLb, bb);
  char_unproject_vjp<T, NV>(cb, WR, URb, WRb, bb);
  T Wb[6][NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    Wb[0][k] = WLb[k] * gL[k][0];
    Wb[5][k] = WRb[k] * gR[k][0];
#pragma unroll
    for (int m = 1; m < 5; ++m) Wb[m][k] = WLb[k] * gL[k][m] + WRb[k] * gR[k][5 - m];
  }
#pragma unroll
  for (int m = 0; m < 6; ++m) char_project_vjp<T, NV>(cb, S[m], Wb[m], Sb[m], bb);
  T Ui[NV], Uj[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) { Ui[k] = S[2][k]; Uj[k] = S[3][k]; }
  roe_basis_vjp<T, NV>(Ui, Uj, gm1, bb, Sb[2], Sb[3]);
}

}  // namespace wcns
