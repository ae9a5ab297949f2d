// Packed single-precision evaluation of one interface.
//
// The left and right states of an interface go through the same arithmetic: Eq. 5-15
// on two mirrored five-point stencils, the characteristic projection of
// mirrored stencil cells, the back-projection of the two interpolated states and their
// primitive variables.  Each value is therefore held as a pair (left lane, right lane)
// in one 64-bit register and every add, multiply and fused multiply-add acts on both
// lanes at once (the f32x2 instructions of sm_100 and later), halving the issue slots
// of that arithmetic.  Comparisons, minima, the FE staircase, the reciprocal unit and
// the Riemann solver work lane by lane (packing those as well costs more in register
// spills than it saves in issue slots at four resident blocks per SM).
//
// Stencil rewrite (same values up to rounding).  With first differences
// d_j = v_{j+1} - v_j of a five-point stencil v0..v4:
//   Eq. 5:   q0 = v2 - 3/8 d0 + 7/8 d1,  q1 = v2 + 1/8 d1 + 3/8 d2,
//            q2 = v2 + 5/8 d2 - 1/8 d3;
//   Eq. 9-10 (times 4, with eps times 4, which leaves Eq. 11-15 unchanged):
//            4 IS_0 = (d0 - 3 d1)^2 + (2 (d1 - d0))^2,
//            4 IS_1 = (d1 + d2)^2   + (2 (d2 - d1))^2,
//            4 IS_2 = (d3 - 3 d2)^2 + (2 (d3 - d2))^2.
#pragma once

#include "wcns_device.cuh"

namespace wcns {
namespace pk {

struct P2 {
  unsigned long long v;
};

__device__ __forceinline__ P2 mk(float a, float b) {
  P2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ P2 bc(float a) { return mk(a, a); }
__device__ __forceinline__ void split(P2 p, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(p.v));
}
__device__ __forceinline__ float lo(P2 p) { float a, b; split(p, a, b); return a; }
__device__ __forceinline__ float hi(P2 p) { float a, b; split(p, a, b); return b; }
__device__ __forceinline__ P2 swap(P2 p) { float a, b; split(p, a, b); return mk(b, a); }

__device__ __forceinline__ P2 add(P2 a, P2 b) {
  P2 d;
  asm("add.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ P2 sub(P2 a, P2 b) {
  P2 d;
  asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ P2 mul(P2 a, P2 b) {
  P2 d;
  asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
// a * b + c
__device__ __forceinline__ P2 fma(P2 a, P2 b, P2 c) {
  P2 d;
  asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return d;
}
__device__ __forceinline__ P2 abs(P2 a) {
  P2 r;
  r.v = a.v & 0x7fffffff7fffffffull;
  return r;
}
// 1 / a through the reciprocal unit, lane by lane
__device__ __forceinline__ P2 rcp(P2 a) {
  float x, y;
  split(a, x, y);
  return mk(Num<float>::rcp_(x), Num<float>::rcp_(y));
}

// Eq. 5-15 and the option-dependent weight maps for the pair (left, right) of
// mirrored stencils v0..v4; returns the two interpolated midpoint values (Eq. 6).
template <int FIX>
__device__ __forceinline__ P2 weno_pair(P2 v0, P2 v1, P2 v2, P2 v3, P2 v4, const SchemeT<float>& s) {
  const int weights = WCNS_OPT(FIX, s, weights);
  const int zp = WCNS_OPT(FIX, s, zp);
  const int renorm = WCNS_OPT(FIX, s, renorm);
  constexpr float d0 = 1.0f / 16.0f, d1 = 10.0f / 16.0f, d2 = 5.0f / 16.0f;
  const P2 e0 = sub(v1, v0), e1 = sub(v2, v1), e2 = sub(v3, v2), e3 = sub(v4, v3);
  // Eq. 5
  const P2 q0 = fma(bc(0.875f), e1, fma(bc(-0.375f), e0, v2));
  const P2 q1 = fma(bc(0.375f), e2, fma(bc(0.125f), e1, v2));
  const P2 q2 = fma(bc(-0.125f), e3, fma(bc(0.625f), e2, v2));
  // Eq. 9-10, times 4
  const P2 g0 = fma(bc(-3.0f), e1, e0), h0 = sub(e1, e0), H0 = add(h0, h0);
  const P2 g1 = add(e1, e2), h1 = sub(e2, e1), H1 = add(h1, h1);
  const P2 g2 = fma(bc(-3.0f), e2, e3), h2 = sub(e3, e2), H2 = add(h2, h2);
  const P2 is0 = fma(g0, g0, mul(H0, H0));
  const P2 is1 = fma(g1, g1, mul(H1, H1));
  const P2 is2 = fma(g2, g2, mul(H2, H2));
  const P2 eps4 = bc(4.0f * s.eps);
  const P2 b0 = add(is0, eps4), b1 = add(is1, eps4), b2 = add(is2, eps4);
  P2 w0, w1, w2;
  if (weights == 0 || weights == 4) {
    // Eq. 11
    const P2 a0 = mul(bc(d0), rcp(mul(b0, b0)));
    const P2 a1 = mul(bc(d1), rcp(mul(b1, b1)));
    const P2 a2 = mul(bc(d2), rcp(mul(b2, b2)));
    const P2 isa = rcp(add(add(a0, a1), a2));
    w0 = mul(a0, isa); w1 = mul(a1, isa); w2 = mul(a2, isa);
    if (weights == 4) {
      // Eq. 12-13, lane by lane
      float l0, l1, l2, r0, r1, r2;
      split(w0, l0, r0); split(w1, l1, r1); split(w2, l2, r2);
      const P2 m0 = mk(m_map<float>(l0, d0), m_map<float>(r0, d0));
      const P2 m1 = mk(m_map<float>(l1, d1), m_map<float>(r1, d1));
      const P2 m2 = mk(m_map<float>(l2, d2), m_map<float>(r2, d2));
      const P2 isg = rcp(add(add(m0, m1), m2));
      w0 = mul(m0, isg); w1 = mul(m1, isg); w2 = mul(m2, isg);
    }
  } else {
    // Eq. 14-15 with the single-precision cap of the ratio
    const P2 tau = abs(sub(is0, is2));
    float t0, t1;
    if (weights == 2 && zp == 1 && (Fixed<FIX>::on || s.ideal_ratio > 0.0f)) {
      // r_k = tau / b_k < ideal_ratio  <=>  tau < ideal_ratio b_k (b_k > 0), tested before
      // the ratios are formed, against a bound lowered by 1e-6: where it holds, both lanes'
      // Z weights lie inside the ideal plateaus of Eq. 20 (see SchemeT::ideal_ratio) and
      // Eq. 6 takes the ideal weights; just below the bound the tests that follow reach
      // the same weights
      const P2 qv = bc(s.ideal_ratio * 0.999999f);
      float c0l, c0r, c1l, c1r, c2l, c2r;
      split(mul(qv, b0), c0l, c0r); split(mul(qv, b1), c1l, c1r); split(mul(qv, b2), c2l, c2r);
      split(tau, t0, t1);
      if (t0 < c0l && t1 < c0r && t0 < c1l && t1 < c1r && t0 < c2l && t1 < c2r)
        return fma(bc(d2), q2, fma(bc(d1), q1, mul(bc(d0), q0)));
    }
    P2 r0 = mul(tau, rcp(b0)), r1 = mul(tau, rcp(b1)), r2 = mul(tau, rcp(b2));
    split(r0, t0, t1); r0 = mk(fminf(t0, 1.0e18f), fminf(t1, 1.0e18f));
    split(r1, t0, t1); r1 = mk(fminf(t0, 1.0e18f), fminf(t1, 1.0e18f));
    split(r2, t0, t1); r2 = mk(fminf(t0, 1.0e18f), fminf(t1, 1.0e18f));
    if (zp == 2) { r0 = mul(r0, r0); r1 = mul(r1, r1); r2 = mul(r2, r2); }
    if (weights == 2 && zp == 2 && s.ideal_ratio > 0.0f) {
      // every ratio of both lanes below ideal_ratio: the Z weights lie inside the ideal
      // plateaus of Eq. 20 (see SchemeT::ideal_ratio), so the mapped and renormalised
      // weights are the ideal ones, without normalising the Z weights first
      float a, b, c, d, e, f;
      split(r0, a, b); split(r1, c, d); split(r2, e, f);
      const float q = s.ideal_ratio;
      if (a < q && b < q && c < q && d < q && e < q && f < q) return fma(bc(d2), q2, fma(bc(d1), q1, mul(bc(d0), q0)));
    }
    const P2 a0 = fma(bc(d0), r0, bc(d0)), a1 = fma(bc(d1), r1, bc(d1)), a2 = fma(bc(d2), r2, bc(d2));
    const P2 isa = rcp(add(add(a0, a1), a2));
    w0 = mul(a0, isa); w1 = mul(a1, isa); w2 = mul(a2, isa);
    if (weights == 2 && s.ideal_margin[0] > 0.0f) {
      // both lanes inside the ideal plateaus of Eq. 20: the map gives the ideal weights,
      // whose sum is exactly 1, so the renormalised weights are the ideal ones and Eq. 6
      // takes them as they are (the staircase below reaches the same weights through its
      // comparisons and a reciprocal of 1 from the reciprocal unit)
      float a, b;
      split(sub(w0, bc(d0)), a, b);
      bool ideal = fmaxf(fabsf(a), fabsf(b)) < s.ideal_margin[0];
      split(sub(w1, bc(d1)), a, b);
      ideal = ideal && fmaxf(fabsf(a), fabsf(b)) < s.ideal_margin[1];
      split(sub(w2, bc(d2)), a, b);
      ideal = ideal && fmaxf(fabsf(a), fabsf(b)) < s.ideal_margin[2];
      if (ideal) return fma(bc(d2), q2, fma(bc(d1), q1, mul(bc(d0), q0)));
    }
    if (weights >= 2) {
      float l0, l1, l2, r0s, r1s, r2s;
      split(w0, l0, r0s); split(w1, l1, r1s); split(w2, l2, r2s);
      bool keep_l = false, keep_r = false;
      if (weights == 3) {
        // App. A: keep the Z weights inside the closed box |w_k - d_k| <= cv
        const float cv = s.cv;
        keep_l = (l0 >= d0 - cv) && (l0 <= d0 + cv) && (l1 >= d1 - cv) && (l1 <= d1 + cv) &&
                 (l2 >= d2 - cv) && (l2 <= d2 + cv);
        keep_r = (r0s >= d0 - cv) && (r0s <= d0 + cv) && (r1s >= d1 - cv) && (r1s <= d1 + cv) &&
                 (r2s >= d2 - cv) && (r2s <= d2 + cv);
      }
      // Eq. 20 on each weight of each lane: the saturated staircase where every tanh
      // term of the lane's three maps is saturated (no weight within sat_dist of a null
      // point), else the exact map for that lane (the exponential form of the map at small
      // xi is evaluated here directly)
      constexpr int FAM = Fixed<FIX>::on ? 0 : -1;
      if (!Fixed<FIX>::on && s.xi_small) {
        if (!keep_l) fe_map_all<float, FAM>(l0, l1, l2, s);
        if (!keep_r) fe_map_all<float, FAM>(r0s, r1s, r2s, s);
      } else {
        if (!keep_l) {
          if (fe_null_distance<float, FAM>(l0, l1, l2, s) >= s.sat_dist) {
            fe_staircase<float, FAM>(l0, l1, l2, s);
          } else {
            l0 = fe_map_slow<float>(0, l0, s); l1 = fe_map_slow<float>(1, l1, s); l2 = fe_map_slow<float>(2, l2, s);
          }
        }
        if (!keep_r) {
          if (fe_null_distance<float, FAM>(r0s, r1s, r2s, s) >= s.sat_dist) {
            fe_staircase<float, FAM>(r0s, r1s, r2s, s);
          } else {
            r0s = fe_map_slow<float>(0, r0s, s); r1s = fe_map_slow<float>(1, r1s, s); r2s = fe_map_slow<float>(2, r2s, s);
          }
        }
      }
      const P2 m0 = mk(l0, r0s), m1 = mk(l1, r1s), m2 = mk(l2, r2s);
      // Eq. 6 on the mapped weights, renormalised (kept lanes are already normalised)
      const P2 acc = fma(m2, q2, fma(m1, q1, mul(m0, q0)));
      if (!renorm) return acc;
      float sl, sr;
      split(add(add(m0, m1), m2), sl, sr);
      const P2 isg = mk(keep_l ? 1.0f : Num<float>::rcp_(sl), keep_r ? 1.0f : Num<float>::rcp_(sr));
      return mul(acc, isg);
    }
  }
  // Eq. 6: convex combination
  return fma(w2, q2, fma(w1, q1, mul(w0, q0)));
}

// Characteristic projection of a pair of cells with the basis of one interface (the
// factored left eigenvectors at the Roe state; P and A carry the factor 1/2).
template <int NV>
__device__ __forceinline__ void project_pair(const CharBasis<float, NV>& cb, const P2 (&U)[NV], P2 (&W)[NV]) {
  const P2 rho = U[0], m = U[1], E = U[NV - 1];
  P2 t = fma(bc(-cb.u), m, E);
  if (NV == 4) t = fma(bc(-cb.v), U[2], t);
  t = fma(bc(cb.hq2), rho, t);
  const P2 Ph = mul(bc(0.5f * cb.b), t);
  const P2 Ah = fma(bc(0.5f * cb.u * cb.ic), rho, mul(bc(-0.5f * cb.ic), m));
  W[0] = add(Ph, Ah);
  W[1] = fma(bc(-2.0f), Ph, rho);
  if (NV == 4) W[2] = fma(bc(-cb.v), rho, U[2]);
  W[NV - 1] = sub(Ph, Ah);
}

// Back-projection of the pair (left, right) of interpolated characteristic states.
template <int NV>
__device__ __forceinline__ void unproject_pair(const CharBasis<float, NV>& cb, const P2 (&W)[NV], P2 (&U)[NV]) {
  const P2 wa = W[0], wb = W[1], wd = W[NV - 1];
  const P2 sum = add(add(wa, wb), wd);
  const P2 dlt = sub(wd, wa);
  U[0] = sum;
  U[1] = fma(bc(cb.c), dlt, mul(bc(cb.u), sum));
  P2 e = fma(bc(cb.hq2), wb, mul(bc(cb.u * cb.c), dlt));
  if (NV == 4) {
    U[2] = fma(bc(cb.v), sum, W[2]);
    e = fma(bc(cb.v), W[2], e);
  }
  U[NV - 1] = fma(bc(cb.H), add(wa, wd), e);
}

// Primitive variables of a pair of conservative states.
template <int NV>
struct PrimPair {
  P2 rho, inv, un, ut, p, H;
};
template <int NV>
__device__ __forceinline__ PrimPair<NV> prim_pair(const P2 (&U)[NV], float gm1) {
  PrimPair<NV> q;
  q.rho = U[0];
  q.inv = rcp(U[0]);
  q.un = mul(U[1], q.inv);
  P2 kin = mul(U[1], q.un);  // rho |u|^2
  if (NV == 4) {
    q.ut = mul(U[2], q.inv);
    kin = fma(U[2], q.ut, kin);
  } else {
    q.ut = bc(0.0f);
  }
  q.p = mul(bc(gm1), fma(bc(-0.5f), kin, U[NV - 1]));
  q.H = mul(add(U[NV - 1], q.p), q.inv);
  return q;
}

// Roe average of the two states of a pair (the state of the characteristic basis).
template <int NV>
__device__ __forceinline__ RoeAvg<float, NV> roe_pair(const PrimPair<NV>& q, float gm1) {
  float rl, rr;
  split(q.rho, rl, rr);
  const float sa = Num<float>::sqrt_(rl), sb = Num<float>::sqrt_(rr);
  const P2 wt = mul(mk(sa, sb), bc(Num<float>::rcp_(sa + sb)));
  float x, y;
  RoeAvg<float, NV> r;
  split(mul(wt, q.un), x, y); r.u = x + y;
  if (NV == 4) { split(mul(wt, q.ut), x, y); r.v = x + y; } else { r.v = 0.0f; }
  split(mul(wt, q.H), x, y); r.H = x + y;
  r.c = Num<float>::sqrt_(gm1 * (r.H - 0.5f * (r.u * r.u + r.v * r.v)));
  return r;
}

// Midpoint flux at one interface (single precision, Euler systems), the packed
// counterpart of interface_flux.  Returns true if the interpolated states were
// non-physical and the interface fell back to (U_i, U_{i+1}).
template <int NV, int FIX>
__device__ __forceinline__ bool interface_flux_pair(const float (&S)[6][NV], const SchemeT<float>& s, int dir,
                                                   float (&F)[NV]) {
  static_assert(NV == 3 || NV == 4, "packed path is for the Euler systems");
  if (WCNS_OPT(FIX, s, family) == 1) return interface_flux<float, NV, FIX>(S, s, dir, F);  // App. B, scalar
  const float gm1 = s.gm1;
  P2 U[NV];  // (left, right) interpolated states
  if (WCNS_OPT(FIX, s, characteristic)) {
    P2 Uc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) Uc[k] = mk(S[2][k], S[3][k]);
    const RoeAvg<float, NV> r = roe_pair<NV>(prim_pair<NV>(Uc, gm1), gm1);
    const CharBasis<float, NV> cb = char_basis<float, NV>(r, gm1);
    // W[m] = (W_m, W_{5-m}) for m = 0, 1, 2
    P2 W[3][NV];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      P2 Um[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) Um[k] = mk(S[m][k], S[5 - m][k]);
      project_pair<NV>(cb, Um, W[m]);
    }
    P2 WI[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k)
      WI[k] = weno_pair<FIX>(W[0][k], W[1][k], W[2][k], swap(W[2][k]), swap(W[1][k]), s);
    unproject_pair<NV>(cb, WI, U);
  } else {
#pragma unroll
    for (int k = 0; k < NV; ++k)
      U[k] = weno_pair<FIX>(mk(S[0][k], S[5][k]), mk(S[1][k], S[4][k]), mk(S[2][k], S[3][k]),
                            mk(S[3][k], S[2][k]), mk(S[4][k], S[1][k]), s);
  }
  // admissibility of the interpolated states (positive density and pressure)
  const PrimPair<NV> q = prim_pair<NV>(U, gm1);
  float rl, rr, pl, pr;
  split(q.rho, rl, rr);
  split(q.p, pl, pr);
  const bool fallback = !(rl > 0.0f && pl > 0.0f && rr > 0.0f && pr > 0.0f);
  if (fallback) {
#pragma unroll
    for (int k = 0; k < NV; ++k) U[k] = mk(S[2][k], S[3][k]);
  }
  float UL[NV], UR[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) split(U[k], UL[k], UR[k]);
  riemann<float, NV, FIX>(UL, UR, s, dir, F);
  return fallback;
}

}  // namespace pk
}  // namespace wcns
