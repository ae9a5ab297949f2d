// WCNS-FE oracle: a plain, slow, FP64 CPU restatement of the filtered embedded
// weighted compact nonlinear scheme (Liu, Min, Cai, Ma, Yan, arXiv 2306.09760).
//
// TEST INFRASTRUCTURE ONLY.  Nothing on the product path may load this library:
// only the test-suite, the smoke check and the benchmark's CPU-baseline leg use it.
// It shares no code, header, table or helper with the CUDA implementation.
//
// Every function follows the paper's steps in the paper's order:
//   * Sec. 2, Eq. 1-2: semi-discrete form du_i/dt = -df/dx|_i.
//   * Eq. 3: sixth-order midpoint flux difference with d = (75/64, -25/384, 3/640).
//   * Eq. 5: sub-stencil interpolations on S0, S1, S2.
//   * Eq. 6: midpoint flux from an approximate Riemann solver on (u^L, u^R).
//   * Eq. 7, 9-11: smoothness indicators and JS weights.
//   * Eq. 12-13: M weights.   Eq. 14-15: Z weights.
//   * Eq. 20-21 with Table 2: the FE mapping function (written with phi, as printed).
//   * App. A: the PFE switch.
//   * App. B: the FE-WENO family -- fifth-order finite-difference WENO on Lax-Friedrichs
//     split fluxes with the Table B.2 control rows (family = 1).
// Readings where the paper is silent (all listed in the design notes):
//   * the FE weights map the Z weights and are renormalised after mapping;
//   * the characteristic projection uses Roe-averaged eigenvectors of the Euler flux
//     Jacobian in the sweep normal, applied to the six stencil cells i-2..i+3;
//   * a non-physical interpolated state (rho <= 0 or p <= 0) falls back to the cell
//     states (U_i, U_{i+1}) at that interface;
//   * time integration is third-order TVD Runge-Kutta (Shu-Osher form), and the CFL
//     step is cfl / sum_d(max(|u_d| + c) / h_d), clipped at t_end.
//
// The arithmetic is templated on the scalar type so that one plain code gives
//   double   -- the values,
//   Dual     -- exact forward-mode tangents (Jacobian-vector products) for the
//               adjoint check,
//   Count    -- an exact count of the floating-point operations the method performs.
// Compiled with -ffp-contract=off so that every operation rounds separately.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------------------
// Scalar types
// ---------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}
inline Dual tanh(Dual a) {
  double t = std::tanh(a.v);
  return Dual(t, a.d * (1.0 - t * t));
}
// d|x| = sign(x) dx with sign(0) = 0.
inline Dual fabs(Dual a) {
  double s = (a.v > 0) ? 1.0 : ((a.v < 0) ? -1.0 : 0.0);
  return Dual(std::fabs(a.v), s * a.d);
}

double g_flops = 0.0;  // operation counter for Count (single-threaded use only)
struct Count {
  double v;
  Count() : v(0) {}
  Count(double x) : v(x) {}
};
inline Count operator+(Count a, Count b) { g_flops += 1; return Count(a.v + b.v); }
inline Count operator-(Count a, Count b) { g_flops += 1; return Count(a.v - b.v); }
inline Count operator-(Count a) { return Count(-a.v); }
inline Count operator*(Count a, Count b) { g_flops += 1; return Count(a.v * b.v); }
inline Count operator/(Count a, Count b) { g_flops += 1; return Count(a.v / b.v); }
inline Count sqrt(Count a) { g_flops += 1; return Count(std::sqrt(a.v)); }
inline Count tanh(Count a) { g_flops += 1; return Count(std::tanh(a.v)); }
inline Count fabs(Count a) { return Count(std::fabs(a.v)); }

inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
inline double val(const Count& x) { return x.v; }
using std::sqrt;
using std::tanh;
using std::fabs;

template <class R> inline R rmax(const R& a, const R& b) { return (val(a) >= val(b)) ? a : b; }
template <class R> inline R rmin(const R& a, const R& b) { return (val(a) <= val(b)) ? a : b; }

}  // namespace

// ---------------------------------------------------------------------------
// Configuration (the oracle's own structure; mirrored by oracle/oracle.py)
// ---------------------------------------------------------------------------
extern "C" {
typedef struct {
  int32_t ndim;            // 1 or 2
  int32_t nvar;            // 1 (scalar advection), 3 (Euler 1D), 4 (Euler 2D)
  int64_t nx, ny;          // cells per direction (ny = 1 in 1D)
  double hx, hy;           // grid spacing per direction
  int32_t bcx, bcy;        // 0 periodic, 1 transmissive (zero-gradient ghosts)
  int32_t system;          // 0 scalar advection, 1 Euler
  int32_t weights;         // 0 JS, 1 Z, 2 FE, 3 PFE, 4 M
  int32_t flux;            // 0 LLF (local alpha), 1 Roe + Harten fix, 2 HLLC, 3 LLF with frozen alpha
  int32_t characteristic;  // 1: interpolate characteristic variables, 0: conservative variables
  int32_t zp;              // Z-weight exponent p (1 or 2)
  int32_t renorm;          // 1: renormalise the mapped weights (FE, PFE)
  double ax, ay;           // advection speeds (scalar system)
  double gamma;            // ratio of specific heats
  double eps;              // epsilon of Eq. 11 / Eq. 14
  double xi, kappa;        // steepness and null-point parameters of Eq. 20
  double cv;               // PFE switch width (App. A)
  double alpha_x, alpha_y; // frozen LLF dissipation speeds (flux == 3)
  double harten;           // Roe entropy-fix fraction delta = harten * (|u| + c)
  int32_t family;          // 0 WCNS (Sec. 2-3), 1 finite-difference WENO on split fluxes (App. B)
  int32_t pad_;
  // Boundary faces x-lo, x-hi, y-lo, y-hi (Sec. 4.3): 0 the direction's bc, 1 transmissive,
  // 2 inviscid wall, 3 fixed state A, 4 state A for x < wall_x and a wall beyond,
  // 5 the moving oblique shock: state A for x < shock_x0 + (y + shock_speed t) shock_dxdy,
  // state B beyond.  States are primitive (rho, u, v, p).
  int32_t face[4];
  double state_a[4], state_b[4];
  double wall_x, shock_x0, shock_dxdy, shock_speed;
  double lo_x, lo_y;       // domain origin: cell centres lo + (i + 1/2) h
  double time;             // time of the state L is evaluated on (moving-shock faces)
} oracle_cfg;
}

namespace {

// ---------------------------------------------------------------------------
// Eq. 20-21 and Table 2: the FE mapping function, written as printed (with phi).
// Row i of Table 2 lists, for j = 0..J_i, the control values omega_{i,j} and the
// control points psi_{i,j}; omega_{i,0} and omega_{i,J_i} are the variable itself.
// ---------------------------------------------------------------------------
const int kJ[3] = {3, 4, 3};
// NaN marks "the variable omega_i itself" (Table 2, first and last rows).
const double kW = NAN;
const double kOmegaCtrl[3][5] = {
    {kW, 1.0 / 16.0, 1.0 / 6.0, kW, 0.0},
    {kW, 10.0 / 16.0, 1.0 / 2.0, 5.0 / 6.0, kW},
    {kW, 5.0 / 16.0, 1.0 / 2.0, kW, 0.0},
};
const double kPsi[3][5] = {
    {0.0, 1.0 / 16.0, 1.0 / 11.0, 1.0, 0.0},
    {0.0, 10.0 / 16.0, 2.0 / 3.0, 10.0 / 11.0, 1.0},
    {0.0, 5.0 / 16.0, 1.0 / 3.0, 1.0, 0.0},
};
// App. B, Table B.2: the same rows for the fifth-order WENO scheme (ideal weights
// 1/10, 6/10, 3/10; Table B.1 lists the cases these control points come from).
const double kOmegaCtrlB[3][5] = {
    {kW, 1.0 / 10.0, 1.0 / 4.0, kW, 0.0},
    {kW, 6.0 / 10.0, 1.0 / 2.0, 3.0 / 4.0, kW},
    {kW, 3.0 / 10.0, 1.0 / 2.0, kW, 0.0},
};
const double kPsiB[3][5] = {
    {0.0, 1.0 / 10.0, 1.0 / 7.0, 1.0, 0.0},
    {0.0, 6.0 / 10.0, 2.0 / 3.0, 6.0 / 7.0, 1.0},
    {0.0, 3.0 / 10.0, 1.0 / 3.0, 1.0, 0.0},
};
// Eq. 21
inline double phi_ij(int i, int j) {
  if ((i == 0 && j == 3) || (i == 2 && j == 3) || (i == 1 && j == 4)) return -1.0;
  return 1.0;
}

// Eq. 20: the mapping function of weight i, the weight plus one tanh step per null point
// kappa (psi_{i,j} + psi_{i,j-1}), each of half the jump between consecutive control values
// of Table 2 (Table B.2 for the App. B family; the weight itself on identity segments),
// phi of Eq. 21 as printed.
template <class R>
R fe_map(int i, const R& w, double xi, double kappa, int family = 0) {
  const double(*ctrl)[5] = family == 1 ? kOmegaCtrlB : kOmegaCtrl;
  const double(*psi)[5] = family == 1 ? kPsiB : kPsi;
  R sum = R(0.0);
  for (int j = 1; j <= kJ[i]; ++j) {
    R wj = std::isnan(ctrl[i][j]) ? w : R(ctrl[i][j]);
    R wjm1 = std::isnan(ctrl[i][j - 1]) ? w : R(ctrl[i][j - 1]);
    double phi = phi_ij(i, j);
    double null_point = kappa * (psi[i][j] + psi[i][j - 1]);
    R arg = R(xi * phi) * (w - R(null_point));
    sum = sum + R(phi) * ((wj - wjm1) / R(2.0)) * tanh(arg);
  }
  return sum + w;
}

// Eq. 13 (Henrick's mapping of the JS weights)
template <class R>
R m_map(const R& w, double d) {
  R num = w * (R(d) + R(d * d) - R(3.0 * d) * w + w * w);
  R den = R(d * d) + R(1.0 - 2.0 * d) * w;
  return num / den;
}

const double kIdeal[3] = {1.0 / 16.0, 10.0 / 16.0, 5.0 / 16.0};  // Sec. 2, ideal weights d_k
const double kIdealB[3] = {1.0 / 10.0, 6.0 / 10.0, 3.0 / 10.0};  // App. B, fifth-order WENO

struct WeightTrace {  // optional record of the weights used (statistics)
  double wz[3], wfinal[3];
  int mapped;
};

// One-sided fifth-order weighted interpolation to the midpoint (Eq. 5-15, 20).
// v[0..4] = u_{i-2}, u_{i-1}, u_i, u_{i+1}, u_{i+2} (left state at i+1/2), or the
// mirrored cells u_{i+3}, u_{i+2}, u_{i+1}, u_i, u_{i-1} (right state at i+1/2).
template <class R>
R weno_midpoint(const R v[5], const oracle_cfg& c, WeightTrace* tr) {
  const double* kId = (c.family == 1) ? kIdealB : kIdeal;
  R q[3];
  R hf[3], hhs[3];
  if (c.family == 1) {
    // App. B: the classical fifth-order WENO reconstruction at x_{i+1/2} from the
    // values v = f_{i-2..i+2}: third-order candidates on S0, S1, S2 ...
    q[0] = (R(2.0) * v[0] - R(7.0) * v[1] + R(11.0) * v[2]) / R(6.0);
    q[1] = (-v[1] + R(5.0) * v[2] + R(2.0) * v[3]) / R(6.0);
    q[2] = (R(2.0) * v[2] + R(5.0) * v[3] - v[4]) / R(6.0);
  } else {
    // Eq. 5
    q[0] = (R(3.0) * v[0] - R(10.0) * v[1] + R(15.0) * v[2]) / R(8.0);
    q[1] = (-v[1] + R(6.0) * v[2] + R(3.0) * v[3]) / R(8.0);
    q[2] = (R(3.0) * v[2] + R(6.0) * v[3] - v[4]) / R(8.0);
  }
  // Eq. 10 (h f_k and h^2 s_k in grid units; the factors of h cancel in Eq. 9)
  hf[0] = (v[0] - R(4.0) * v[1] + R(3.0) * v[2]) / R(2.0);
  hhs[0] = v[0] - R(2.0) * v[1] + v[2];
  hf[1] = (v[3] - v[1]) / R(2.0);
  hhs[1] = v[1] - R(2.0) * v[2] + v[3];
  hf[2] = (R(-3.0) * v[2] + R(4.0) * v[3] - v[4]) / R(2.0);
  hhs[2] = v[2] - R(2.0) * v[3] + v[4];
  R IS[3];
  if (c.family == 1) {
    // ... and the Jiang-Shu indicators IS_k = (h f_k)^2 + 13/12 (h^2 s_k)^2, with h f_k
    // and h^2 s_k the same differences as in Eq. 10
    for (int k = 0; k < 3; ++k) IS[k] = R(13.0 / 12.0) * hhs[k] * hhs[k] + hf[k] * hf[k];
  } else {
    // Eq. 9
    for (int k = 0; k < 3; ++k) IS[k] = hf[k] * hf[k] + hhs[k] * hhs[k];
  }

  R w[3];
  if (c.weights == 0 || c.weights == 4) {
    // Eq. 11 (JS); the sum runs over l = 0..2
    R a[3];
    for (int k = 0; k < 3; ++k) {
      R s = IS[k] + R(c.eps);
      a[k] = R(kId[k]) / (s * s);
    }
    R sa = a[0] + a[1] + a[2];
    for (int k = 0; k < 3; ++k) w[k] = a[k] / sa;
    if (tr) {
      for (int k = 0; k < 3; ++k) tr->wz[k] = val(w[k]);
      tr->mapped = 0;
    }
    if (c.weights == 4) {
      // Eq. 12-13 (M)
      R b[3];
      for (int k = 0; k < 3; ++k) b[k] = m_map(w[k], kId[k]);
      R sb = b[0] + b[1] + b[2];
      for (int k = 0; k < 3; ++k) w[k] = b[k] / sb;
    }
  } else {
    // Eq. 14-15 (Z)
    R tau = fabs(IS[0] - IS[2]);
    R a[3];
    for (int k = 0; k < 3; ++k) {
      R r = tau / (IS[k] + R(c.eps));
      R rp = r;
      for (int e = 1; e < c.zp; ++e) rp = rp * r;
      a[k] = R(kId[k]) * (R(1.0) + rp);
    }
    R sa = a[0] + a[1] + a[2];
    for (int k = 0; k < 3; ++k) w[k] = a[k] / sa;
    if (tr) {
      for (int k = 0; k < 3; ++k) tr->wz[k] = val(w[k]);
      tr->mapped = 0;
    }
    if (c.weights == 2 || c.weights == 3) {
      bool keep = false;
      if (c.weights == 3) {
        // App. A: keep the Z weights when all three lie in [d_k - cv, d_k + cv]
        keep = true;
        for (int k = 0; k < 3; ++k)
          if (!(val(w[k]) >= kId[k] - c.cv && val(w[k]) <= kId[k] + c.cv)) keep = false;
      }
      if (!keep) {
        // Eq. 20 applied to each Z weight, then renormalised
        R g[3];
        for (int k = 0; k < 3; ++k) g[k] = fe_map(k, w[k], c.xi, c.kappa, c.family);
        if (c.renorm) {
          R sg = g[0] + g[1] + g[2];
          for (int k = 0; k < 3; ++k) w[k] = g[k] / sg;
        } else {
          for (int k = 0; k < 3; ++k) w[k] = g[k];
        }
        if (tr) tr->mapped = 1;
      }
    }
  }
  if (tr)
    for (int k = 0; k < 3; ++k) tr->wfinal[k] = val(w[k]);
  // Eq. 6: convex combination of the sub-stencil values
  return w[0] * q[0] + w[1] * q[1] + w[2] * q[2];
}

// ---------------------------------------------------------------------------
// Euler equations in the sweep normal.  States are ordered with the normal
// momentum second: (rho, rho*un, [rho*ut,] E).  The y-sweep permutes (rho u, rho v).
// ---------------------------------------------------------------------------
template <class R>
struct Prim {
  R rho, un, ut, p, H, c2;
};

// Primitive variables of a conserved state (Sec. 2: ideal gas, p = (gamma - 1)(E - rho |v|^2 / 2)),
// with the total enthalpy H and the squared sound speed.
template <class R>
Prim<R> primitive(const R* U, int nvar, double gamma) {
  Prim<R> s;
  s.rho = U[0];
  s.un = U[1] / U[0];
  R E;
  R kin;
  if (nvar == 4) {
    s.ut = U[2] / U[0];
    E = U[3];
    kin = R(0.5) * s.rho * (s.un * s.un + s.ut * s.ut);
  } else {
    s.ut = R(0.0);
    E = U[2];
    kin = R(0.5) * s.rho * s.un * s.un;
  }
  s.p = R(gamma - 1.0) * (E - kin);
  s.H = (E + s.p) / s.rho;
  s.c2 = R(gamma) * s.p / s.rho;
  return s;
}

// Euler flux in the sweep normal (Eq. 1).
template <class R>
void physical_flux(const R* U, int nvar, double gamma, R* F) {
  Prim<R> s = primitive(U, nvar, gamma);
  F[0] = U[1];
  F[1] = U[1] * s.un + s.p;
  if (nvar == 4) {
    F[2] = U[2] * s.un;
    F[3] = (U[3] + s.p) * s.un;
  } else {
    F[2] = (U[2] + s.p) * s.un;
  }
}

// Roe average of two states (sqrt(rho) weighting).
template <class R>
void roe_average(const R* UL, const R* UR, int nvar, double gamma, R& u, R& v, R& H, R& c) {
  Prim<R> a = primitive(UL, nvar, gamma), b = primitive(UR, nvar, gamma);
  R sa = sqrt(a.rho), sb = sqrt(b.rho);
  R den = sa + sb;
  u = (sa * a.un + sb * b.un) / den;
  v = (sa * a.ut + sb * b.ut) / den;
  H = (sa * a.H + sb * b.H) / den;
  R q2 = u * u + v * v;
  c = sqrt(R(gamma - 1.0) * (H - R(0.5) * q2));
}

// Right (columns) and left (rows) eigenvectors of the flux Jacobian at (u, v, H, c).
template <class R>
void eigenvectors(int nvar, double gamma, const R& u, const R& v, const R& H, const R& c,
                  R Rm[4][4], R Lm[4][4]) {
  R q2 = u * u + v * v;
  R b = R(gamma - 1.0) / (c * c);
  R bq = b * q2 / R(2.0);
  if (nvar == 3) {
    Rm[0][0] = R(1.0);      Rm[0][1] = R(1.0);            Rm[0][2] = R(1.0);
    Rm[1][0] = u - c;       Rm[1][1] = u;                 Rm[1][2] = u + c;
    Rm[2][0] = H - u * c;   Rm[2][1] = q2 / R(2.0);       Rm[2][2] = H + u * c;
    Lm[0][0] = (bq + u / c) / R(2.0); Lm[0][1] = (-b * u - R(1.0) / c) / R(2.0); Lm[0][2] = b / R(2.0);
    Lm[1][0] = R(1.0) - bq;           Lm[1][1] = b * u;                         Lm[1][2] = -b;
    Lm[2][0] = (bq - u / c) / R(2.0); Lm[2][1] = (-b * u + R(1.0) / c) / R(2.0); Lm[2][2] = b / R(2.0);
  } else {
    Rm[0][0] = R(1.0);    Rm[0][1] = R(1.0);        Rm[0][2] = R(0.0); Rm[0][3] = R(1.0);
    Rm[1][0] = u - c;     Rm[1][1] = u;             Rm[1][2] = R(0.0); Rm[1][3] = u + c;
    Rm[2][0] = v;         Rm[2][1] = v;             Rm[2][2] = R(1.0); Rm[2][3] = v;
    Rm[3][0] = H - u * c; Rm[3][1] = q2 / R(2.0);   Rm[3][2] = v;      Rm[3][3] = H + u * c;
    Lm[0][0] = (bq + u / c) / R(2.0); Lm[0][1] = (-b * u - R(1.0) / c) / R(2.0);
    Lm[0][2] = (-b * v) / R(2.0);     Lm[0][3] = b / R(2.0);
    Lm[1][0] = R(1.0) - bq; Lm[1][1] = b * u; Lm[1][2] = b * v; Lm[1][3] = -b;
    Lm[2][0] = -v; Lm[2][1] = R(0.0); Lm[2][2] = R(1.0); Lm[2][3] = R(0.0);
    Lm[3][0] = (bq - u / c) / R(2.0); Lm[3][1] = (-b * u + R(1.0) / c) / R(2.0);
    Lm[3][2] = (-b * v) / R(2.0);     Lm[3][3] = b / R(2.0);
  }
}

// Positive density and pressure: the admissibility test of an interpolated state (a
// state that fails it falls back to the cell states U_i, U_{i+1} at that interface).
template <class R>
bool physical_state(const R* U, int nvar, double gamma) {
  if (!(val(U[0]) > 0.0)) return false;
  Prim<R> s = primitive(U, nvar, gamma);
  return val(s.p) > 0.0;
}

// Approximate Riemann solvers for the midpoint flux (Eq. 6; the paper names none).
template <class R>
void riemann_flux(const R* UL, const R* UR, int nvar, const oracle_cfg& c, double alpha_frozen,
                  R* F) {
  const double g = c.gamma;
  R FL[4], FR[4];
  physical_flux(UL, nvar, g, FL);
  physical_flux(UR, nvar, g, FR);
  Prim<R> a = primitive(UL, nvar, g), b = primitive(UR, nvar, g);
  if (c.flux == 0 || c.flux == 3) {
    // Local Lax-Friedrichs (Rusanov)
    R alpha;
    if (c.flux == 3) {
      alpha = R(alpha_frozen);
    } else {
      R sl = fabs(a.un) + sqrt(a.c2);
      R sr = fabs(b.un) + sqrt(b.c2);
      alpha = rmax(sl, sr);
    }
    for (int k = 0; k < nvar; ++k)
      F[k] = R(0.5) * (FL[k] + FR[k]) - R(0.5) * alpha * (UR[k] - UL[k]);
    return;
  }
  if (c.flux == 1) {
    // Roe flux with Harten's entropy fix: F = (FL+FR)/2 - 1/2 sum_k |lambda_k| a_k r_k
    R u, v, H, cc;
    roe_average(UL, UR, nvar, g, u, v, H, cc);
    R Rm[4][4], Lm[4][4];
    eigenvectors(nvar, g, u, v, H, cc, Rm, Lm);
    R lam[4];
    if (nvar == 3) {
      lam[0] = u - cc; lam[1] = u; lam[2] = u + cc;
    } else {
      lam[0] = u - cc; lam[1] = u; lam[2] = u; lam[3] = u + cc;
    }
    R delta = R(c.harten) * (fabs(u) + cc);
    R dU[4], amp[4];
    for (int k = 0; k < nvar; ++k) dU[k] = UR[k] - UL[k];
    for (int m = 0; m < nvar; ++m) {
      R s = R(0.0);
      for (int k = 0; k < nvar; ++k) s = s + Lm[m][k] * dU[k];
      R al = fabs(lam[m]);
      // Harten's fix on the acoustic (genuinely nonlinear) fields u -/+ c only
      bool acoustic = (m == 0 || m == nvar - 1);
      if (acoustic && val(al) < val(delta)) al = (lam[m] * lam[m] + delta * delta) / (R(2.0) * delta);
      amp[m] = al * s;
    }
    for (int k = 0; k < nvar; ++k) {
      R d = R(0.0);
      for (int m = 0; m < nvar; ++m) d = d + Rm[k][m] * amp[m];
      F[k] = R(0.5) * (FL[k] + FR[k]) - R(0.5) * d;
    }
    return;
  }
  // HLLC (Toro) with Einfeldt wave-speed estimates from the Roe average
  R u, v, H, cc;
  roe_average(UL, UR, nvar, g, u, v, H, cc);
  R cl = sqrt(a.c2), cr = sqrt(b.c2);
  R SL = rmin(a.un - cl, u - cc);
  R SR = rmax(b.un + cr, u + cc);
  if (val(SL) >= 0.0) {
    for (int k = 0; k < nvar; ++k) F[k] = FL[k];
    return;
  }
  if (val(SR) <= 0.0) {
    for (int k = 0; k < nvar; ++k) F[k] = FR[k];
    return;
  }
  R ml = a.rho * (SL - a.un), mr = b.rho * (SR - b.un);
  R Sst = (b.p - a.p + a.un * ml - b.un * mr) / (ml - mr);
  const R* UK = (val(Sst) >= 0.0) ? UL : UR;
  const R* FK = (val(Sst) >= 0.0) ? FL : FR;
  const Prim<R>& s = (val(Sst) >= 0.0) ? a : b;
  R SK = (val(Sst) >= 0.0) ? SL : SR;
  R fac = s.rho * (SK - s.un) / (SK - Sst);
  R Ust[4];
  R EK = (nvar == 4) ? UK[3] : UK[2];
  R Est = fac * (EK / s.rho + (Sst - s.un) * (Sst + s.p / (s.rho * (SK - s.un))));
  Ust[0] = fac;
  Ust[1] = fac * Sst;
  if (nvar == 4) {
    Ust[2] = fac * s.ut;
    Ust[3] = Est;
  } else {
    Ust[2] = Est;
  }
  for (int k = 0; k < nvar; ++k) F[k] = FK[k] + SK * (Ust[k] - UK[k]);
}

// ---------------------------------------------------------------------------
// Grid access with ghost cells from index arithmetic
// ---------------------------------------------------------------------------
inline int64_t ghost_index(int64_t i, int64_t n, int bc) {
  if (bc == 0) {
    int64_t r = i % n;
    return r < 0 ? r + n : r;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// Cell m of a sweep line, component v in the sweep's normal ordering (component 1 is the
// normal momentum).  Inside [0, n) it is the stored cell; outside, the face rule of
// that side gives the ghost value: periodic wrap, transmissive copy of the edge cell,
// an inviscid wall (mirror cell with the normal momentum reversed), or a prescribed
// state at the ghost cell's centre (Sec. 4.3: inflow, post-shock strip, moving shock).
template <class R, class Interior>
R line_cell(const oracle_cfg& c, int dir, int64_t line, int64_t m, int64_t n, int bc, int v,
            const Interior& interior) {
  if (m >= 0 && m < n) return interior(m, v);
  const int side = m < 0 ? 0 : 1;
  int type = c.face[2 * dir + side];
  if (type == 0) type = (bc == 0) ? -1 : 1;
  const double hx = c.hx, hy = c.hy;
  const double x = dir == 0 ? c.lo_x + (m + 0.5) * hx : c.lo_x + (line + 0.5) * hx;
  const double y = dir == 0 ? c.lo_y + (line + 0.5) * hy : c.lo_y + (m + 0.5) * hy;
  if (type == 4) type = (x < c.wall_x) ? 3 : 2;
  if (type == -1) return interior(ghost_index(m, n, 0), v);
  if (type == 1) return interior(ghost_index(m, n, 1), v);
  if (type == 2) {
    const int64_t mm = m < 0 ? -1 - m : 2 * n - 1 - m;
    const R val = interior(mm, v);
    return v == 1 ? -val : val;
  }
  const double* st = c.state_a;
  if (type == 5) st = (x < c.shock_x0 + (y + c.shock_speed * c.time) * c.shock_dxdy) ? c.state_a : c.state_b;
  // conservative state in the sweep's ordering
  const double rho = st[0], un = dir == 0 ? st[1] : st[2], ut = dir == 0 ? st[2] : st[1], p = st[3];
  if (c.nvar == 3) {
    const double U[3] = {rho, rho * st[1], p / (c.gamma - 1.0) + 0.5 * rho * st[1] * st[1]};
    return R(U[v]);
  }
  const double U[4] = {rho, rho * un, rho * ut, p / (c.gamma - 1.0) + 0.5 * rho * (un * un + ut * ut)};
  return R(U[v]);
}

struct Stats {
  long long nonphysical;
  // weight statistics (optional)
  long long* hist;  // [2 (Z, final)][3][nbins] or null
  int nbins;
  long long samples;
};

// Midpoint flux at interface k+1/2 of a line of n cells.  `cell(m, var)` reads cell m
// (already ghost-mapped) of the line in the sweep's normal ordering.
// App. A bins [0, 1] into nbins equal subdomains.  The ideal weights and the control
// values are multiples of 1e-4 and so lie on bin edges; a weight within 1e-10 below an
// edge (round-off in the renormalisation) is counted in the edge's bin.
inline int weight_bin(double w, int nbins) {
  double x = w * nbins + 1e-6;
  int b = x < 0.0 ? 0 : (int)x;
  return std::min(nbins - 1, b);
}

template <class R>
void record_weights(Stats* st, const WeightTrace& tr) {
  for (int w = 0; w < 3; ++w) {
    int b0 = weight_bin(tr.wz[w], st->nbins);
    int b1 = weight_bin(tr.wfinal[w], st->nbins);
    st->hist[(0 * 3 + w) * st->nbins + b0]++;
    st->hist[(1 * 3 + w) * st->nbins + b1]++;
  }
  st->samples++;
}

// App. B (FE-WENO family): finite-difference WENO on Lax-Friedrichs split fluxes.
// f+-_m = (F(U_m) +- alpha U_m) / 2 for the six stencil cells m = i-2..i+3, with one
// dissipation speed per interface, alpha = max over those cells of |u_n| + c.  With the
// characteristic option both split fluxes are projected with the left eigenvectors at the
// Roe state of (U_i, U_{i+1}); f+ is reconstructed from the left-biased stencil
// (cells i-2..i+2), f- from the mirrored one (cells i+3..i-1), and the flux at i+1/2 is
// R (f+^ + f-^).
template <class R, class Side>
void weno_split_flux(const R U[6][4], const oracle_cfg& c, const Side& side, R* F) {
  const int nv = c.nvar;
  R Fm[6][4];
  R alpha = R(0.0);
  for (int m = 0; m < 6; ++m) {
    physical_flux(U[m], nv, c.gamma, Fm[m]);
    Prim<R> s = primitive(U[m], nv, c.gamma);
    alpha = rmax(alpha, fabs(s.un) + sqrt(s.c2));
  }
  R gp[6][4], gm[6][4];
  for (int m = 0; m < 6; ++m)
    for (int v = 0; v < nv; ++v) {
      gp[m][v] = R(0.5) * (Fm[m][v] + alpha * U[m][v]);
      gm[m][v] = R(0.5) * (Fm[m][v] - alpha * U[m][v]);
    }
  R Rm[4][4], Lm[4][4];
  if (c.characteristic) {
    R u, v, H, cc;
    roe_average(U[2], U[3], nv, c.gamma, u, v, H, cc);
    eigenvectors(nv, c.gamma, u, v, H, cc, Rm, Lm);
    R tp[6][4], tm[6][4];
    for (int m = 0; m < 6; ++m)
      for (int k = 0; k < nv; ++k) {
        R ap = R(0.0), am = R(0.0);
        for (int q = 0; q < nv; ++q) {
          ap = ap + Lm[k][q] * gp[m][q];
          am = am + Lm[k][q] * gm[m][q];
        }
        tp[m][k] = ap;
        tm[m][k] = am;
      }
    for (int m = 0; m < 6; ++m)
      for (int k = 0; k < nv; ++k) {
        gp[m][k] = tp[m][k];
        gm[m][k] = tm[m][k];
      }
  }
  R Fh[4];
  for (int k = 0; k < nv; ++k) {
    R v5[5];
    for (int s = 0; s < 5; ++s) v5[s] = gp[s][k];
    R fp = side(v5);
    for (int s = 0; s < 5; ++s) v5[s] = gm[5 - s][k];
    Fh[k] = fp + side(v5);
  }
  for (int q = 0; q < nv; ++q) {
    if (c.characteristic) {
      R acc = R(0.0);
      for (int k = 0; k < nv; ++k) acc = acc + Rm[q][k] * Fh[k];
      F[q] = acc;
    } else {
      F[q] = Fh[q];
    }
  }
}

// Midpoint flux at interface k+1/2 of a line of n cells.  `cell(m, var)` reads cell m
// (already ghost-mapped) of the line in the sweep's normal ordering.
template <class R, class Cell>
void interface_flux(int64_t k, int64_t n, int bc, const oracle_cfg& c, double alpha_frozen,
                    const Cell& cell, R* F, Stats* st) {
  const int nv = c.nvar;
  const bool rec = st && st->hist;
  // one-sided interpolation, recording the weights when statistics are requested
  auto side = [&](const R* v5) -> R {
    WeightTrace tr;
    R r = weno_midpoint(v5, c, rec ? &tr : nullptr);
    if (rec) record_weights<R>(st, tr);
    return r;
  };
  R U[6][4];
  for (int s = 0; s < 6; ++s)
    for (int v = 0; v < nv; ++v) U[s][v] = cell(k - 2 + s, v);
  if (c.system == 0 && c.family == 1) {
    // App. B on u_t + a u_x = 0: f+ = max(a, 0) u from the left-biased stencil,
    // f- = min(a, 0) u from the mirrored stencil
    R a = R(alpha_frozen);
    R ap = R(0.5) * (a + fabs(a)), am = R(0.5) * (a - fabs(a));
    R v5[5];
    for (int s = 0; s < 5; ++s) v5[s] = ap * U[s][0];
    R fp = side(v5);
    for (int s = 0; s < 5; ++s) v5[s] = am * U[5 - s][0];
    F[0] = fp + side(v5);
    return;
  }
  if (c.system == 0) {
    // scalar advection: upwind state, F = a u
    R v5[5];
    for (int s = 0; s < 5; ++s) v5[s] = U[s][0];
    R uL = side(v5);
    for (int s = 0; s < 5; ++s) v5[s] = U[5 - s][0];
    R uR = side(v5);
    R a = R(alpha_frozen);  // the advection speed of this direction
    F[0] = (val(a) >= 0.0) ? a * uL : a * uR;
    return;
  }
  if (c.family == 1) {
    weno_split_flux(U, c, side, F);
    return;
  }
  R UL[4] = {}, UR[4] = {};
  if (c.characteristic) {
    R u, v, H, cc;
    roe_average(U[2], U[3], nv, c.gamma, u, v, H, cc);
    R Rm[4][4], Lm[4][4];
    eigenvectors(nv, c.gamma, u, v, H, cc, Rm, Lm);
    R W[6][4];
    for (int s = 0; s < 6; ++s)
      for (int m = 0; m < nv; ++m) {
        R acc = R(0.0);
        for (int q = 0; q < nv; ++q) acc = acc + Lm[m][q] * U[s][q];
        W[s][m] = acc;
      }
    R WL[4], WR[4];
    for (int m = 0; m < nv; ++m) {
      R v5[5];
      for (int s = 0; s < 5; ++s) v5[s] = W[s][m];
      WL[m] = side(v5);
      for (int s = 0; s < 5; ++s) v5[s] = W[5 - s][m];
      WR[m] = side(v5);
    }
    for (int q = 0; q < nv; ++q) {
      R al = R(0.0), ar = R(0.0);
      for (int m = 0; m < nv; ++m) {
        al = al + Rm[q][m] * WL[m];
        ar = ar + Rm[q][m] * WR[m];
      }
      UL[q] = al;
      UR[q] = ar;
    }
  } else {
    for (int q = 0; q < nv; ++q) {
      R v5[5];
      for (int s = 0; s < 5; ++s) v5[s] = U[s][q];
      UL[q] = side(v5);
      for (int s = 0; s < 5; ++s) v5[s] = U[5 - s][q];
      UR[q] = side(v5);
    }
  }
  if (!physical_state(UL, nv, c.gamma) || !physical_state(UR, nv, c.gamma)) {
    for (int q = 0; q < nv; ++q) {
      UL[q] = U[2][q];
      UR[q] = U[3][q];
    }
    if (st) {
#pragma omp atomic
      st->nonphysical++;
    }
  }
  riemann_flux(UL, UR, nv, c, alpha_frozen, F);
}

// Eq. 3 coefficients
const double kD[3] = {75.0 / 64.0, -25.0 / 384.0, 3.0 / 640.0};

// Adds -(dF/dx) along one line to `out` (Eq. 2-3).  `perm` maps the sweep's
// normal ordering to storage components.
template <class R, class Cell, class Out>
void line_rhs(int64_t n, int bc, double h, const oracle_cfg& c, double alpha, const int* perm,
              const Cell& cell, const Out& out, Stats* st) {
  const int nv = c.nvar;
  // interfaces k+1/2 for k = -3..n+1
  std::vector<R> F((size_t)(n + 5) * nv);
  if (c.family == 1) {
    // App. B: conservative finite difference -(F_{i+1/2} - F_{i-1/2}) / h
    for (int64_t k = -1; k <= n - 1; ++k)
      interface_flux<R>(k, n, bc, c, alpha, cell, &F[(size_t)(k + 3) * nv], st);
    for (int64_t i = 0; i < n; ++i)
      for (int v = 0; v < nv; ++v)
        out(i, perm[v], -((F[(size_t)(i + 3) * nv + v] - F[(size_t)(i + 2) * nv + v]) / R(h)));
    return;
  }
  for (int64_t k = -3; k <= n + 1; ++k)
    interface_flux<R>(k, n, bc, c, alpha, cell, &F[(size_t)(k + 3) * nv], st);
  for (int64_t i = 0; i < n; ++i) {
    for (int v = 0; v < nv; ++v) {
      R acc = R(0.0);
      for (int m = 1; m <= 3; ++m) {
        R fp = F[(size_t)(i + m - 1 + 3) * nv + v];  // F_{i+m-1/2}
        R fm = F[(size_t)(i - m + 3) * nv + v];      // F_{i-m+1/2}
        acc = acc + R(kD[m - 1]) * (fp - fm);
      }
      out(i, perm[v], -(acc / R(h)));
    }
  }
}

// L(u) of Eq. 2 on the whole grid: the Eq. 3 difference of every x line, plus that of
// every y line on 2D grids (dimension by dimension).
template <class R>
void rhs(const oracle_cfg& c, const R* u, R* dudt, Stats* st) {
  const int64_t nx = c.nx, ny = (c.ndim == 2) ? c.ny : 1;
  const int nv = c.nvar;
  const int64_t plane = nx * ny;
  for (int64_t q = 0; q < plane * nv; ++q) dudt[q] = R(0.0);
  int permx[4] = {0, 1, 2, 3};
  double ax = (c.system == 0) ? c.ax : c.alpha_x;
#pragma omp parallel for schedule(dynamic, 1) if (ny > 1)
  for (int64_t j = 0; j < ny; ++j) {
    auto stored = [&](int64_t m, int v) -> R { return u[(size_t)v * plane + j * nx + m]; };
    auto cell = [&](int64_t m, int v) -> R { return line_cell<R>(c, 0, j, m, nx, c.bcx, v, stored); };
    auto out = [&](int64_t i, int v, const R& x) { dudt[(size_t)v * plane + j * nx + i] = dudt[(size_t)v * plane + j * nx + i] + x; };
    line_rhs<R>(nx, c.bcx, c.hx, c, ax, permx, cell, out, st);
  }
  if (c.ndim == 2) {
    // y-sweep: normal momentum is rho*v, so the sweep ordering is (rho, rho v, rho u, E)
    int permy[4] = {0, 2, 1, 3};
    double ay = (c.system == 0) ? c.ay : c.alpha_y;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < nx; ++i) {
      auto stored = [&](int64_t m, int v) -> R { return u[(size_t)permy[v] * plane + m * nx + i]; };
      auto cell = [&](int64_t m, int v) -> R { return line_cell<R>(c, 1, i, m, ny, c.bcy, v, stored); };
      auto out = [&](int64_t jj, int v, const R& x) { dudt[(size_t)v * plane + jj * nx + i] = dudt[(size_t)v * plane + jj * nx + i] + x; };
      line_rhs<R>(ny, c.bcy, c.hy, c, ay, permy, cell, out, st);
    }
  }
}

// Largest signal speed per direction: max over cells of |u_d| + c (Euler), |a_d| (scalar)
void max_wave(const oracle_cfg& c, const double* u, double* wx, double* wy) {
  const int64_t nx = c.nx, ny = (c.ndim == 2) ? c.ny : 1;
  const int64_t plane = nx * ny;
  if (c.system == 0) {
    *wx = std::fabs(c.ax);
    *wy = std::fabs(c.ay);
    return;
  }
  double mx = 0.0, my = 0.0;
  for (int64_t q = 0; q < plane; ++q) {
    double U[4];
    for (int v = 0; v < c.nvar; ++v) U[v] = u[(size_t)v * plane + q];
    Prim<double> s = primitive(U, c.nvar, c.gamma);
    double cs = std::sqrt(s.c2);
    mx = std::max(mx, std::fabs(s.un) + cs);
    if (c.nvar == 4) my = std::max(my, std::fabs(s.ut) + cs);
  }
  *wx = mx;
  *wy = my;
}

// Step at CFL number cfl (Sec. 4 marches at a fixed CFL number): dt = cfl / sum_d max_d / h_d.
double cfl_dt(const oracle_cfg& c, const double* u, double cfl) {
  double wx, wy;
  max_wave(c, u, &wx, &wy);
  double s = wx / c.hx;
  if (c.ndim == 2) s += wy / c.hy;
  return cfl / s;
}

// Third-order TVD Runge-Kutta step (Shu-Osher form):
//   u1 = u + dt L(u);  u2 = 3/4 u + 1/4 (u1 + dt L(u1));  u' = 1/3 u + 2/3 (u2 + dt L(u2))
template <class R>
void rk3_step(const oracle_cfg& c0, R* u, double dt, Stats* st) {
  // stage times t, t + dt, t + dt/2 (c0.time = t) for time-dependent boundary faces
  oracle_cfg c = c0;
  const int64_t ncell = c.nx * ((c.ndim == 2) ? c.ny : 1) * c.nvar;
  std::vector<R> L((size_t)ncell), u1((size_t)ncell), u2((size_t)ncell);
  rhs<R>(c, u, L.data(), st);
  for (int64_t q = 0; q < ncell; ++q) u1[q] = u[q] + R(dt) * L[q];
  c.time = c0.time + dt;
  rhs<R>(c, u1.data(), L.data(), st);
  for (int64_t q = 0; q < ncell; ++q)
    u2[q] = R(0.75) * u[q] + R(0.25) * (u1[q] + R(dt) * L[q]);
  c.time = c0.time + 0.5 * dt;
  rhs<R>(c, u2.data(), L.data(), st);
  for (int64_t q = 0; q < ncell; ++q)
    u[q] = R(1.0 / 3.0) * u[q] + R(2.0 / 3.0) * (u2[q] + R(dt) * L[q]);
}

// Classical fourth-order Runge-Kutta (Eq. 16, printed in the form used by the paper).
void rk4_step(const oracle_cfg& c0, double* u, double dt, Stats* st) {
  oracle_cfg c = c0;  // stage times t, t + dt/2, t + dt/2, t + dt
  const int64_t ncell = c.nx * ((c.ndim == 2) ? c.ny : 1) * c.nvar;
  std::vector<double> L((size_t)ncell), u1((size_t)ncell), u2((size_t)ncell), u3((size_t)ncell);
  rhs<double>(c, u, L.data(), st);
  for (int64_t q = 0; q < ncell; ++q) u1[q] = u[q] + 0.5 * dt * L[q];
  c.time = c0.time + 0.5 * dt;
  rhs<double>(c, u1.data(), L.data(), st);
  for (int64_t q = 0; q < ncell; ++q) u2[q] = u[q] + 0.5 * dt * L[q];
  rhs<double>(c, u2.data(), L.data(), st);
  for (int64_t q = 0; q < ncell; ++q) u3[q] = u[q] + dt * L[q];
  c.time = c0.time + dt;
  rhs<double>(c, u3.data(), L.data(), st);
  for (int64_t q = 0; q < ncell; ++q)
    u[q] = -u[q] / 3.0 + u1[q] / 3.0 + 2.0 * u2[q] / 3.0 + u3[q] / 3.0 + dt / 6.0 * L[q];
}

}  // namespace

// ---------------------------------------------------------------------------
// C entry points (ctypes)
// ---------------------------------------------------------------------------
extern "C" {

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Eq. 20 evaluated for weight index i at w (pins for Table 1 / Table 2).
double oracle_fe_map(int i, double w, double xi, double kappa) { return fe_map<double>(i, w, xi, kappa); }

// Eq. 20 with the App. B (Table B.2) control rows when family == 1.
double oracle_fe_map_family(int family, int i, double w, double xi, double kappa) {
  return fe_map<double>(i, w, xi, kappa, family);
}

// Eq. 13 evaluated at w for ideal weight d.
double oracle_m_map(double w, double d) { return m_map<double>(w, d); }

// Derivative of Eq. 20 (forward mode).
double oracle_fe_map_deriv(int i, double w, double xi, double kappa) {
  return fe_map<Dual>(i, Dual(w, 1.0), xi, kappa).d;
}

// One-sided midpoint interpolation of five values; also returns the Z (or JS)
// weights and the final weights.
double oracle_interp(const oracle_cfg* c, const double* v5, double* wz, double* wfinal, int* mapped) {
  WeightTrace tr;
  double r = weno_midpoint<double>(v5, *c, &tr);
  if (wz) for (int k = 0; k < 3; ++k) wz[k] = tr.wz[k];
  if (wfinal) for (int k = 0; k < 3; ++k) wfinal[k] = tr.wfinal[k];
  if (mapped) *mapped = tr.mapped;
  return r;
}

// Eigenvector matrices (row-major 4x4, top-left nvar x nvar used).
void oracle_eigenvectors(int nvar, double gamma, double u, double v, double H, double c, double* Rm,
                         double* Lm) {
  double R4[4][4], L4[4][4];
  eigenvectors<double>(nvar, gamma, u, v, H, c, R4, L4);
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      Rm[a * 4 + b] = (a < nvar && b < nvar) ? R4[a][b] : 0.0;
      Lm[a * 4 + b] = (a < nvar && b < nvar) ? L4[a][b] : 0.0;
    }
}

// Midpoint flux at the interface between cells 2 and 3 of six stencil states
// S[m][v] (m = 0..5 = cells i-2..i+3, x-normal ordering); returns 1 on fallback.
int oracle_interface_flux(const oracle_cfg* c, const double* S, double* F) {
  const int nv = c->nvar;
  auto cell = [&](int64_t m, int v) -> double { return S[m * nv + v]; };
  Stats st{0, nullptr, 0, 0};
  interface_flux<double>(2, 6, 1, *c, (c->system == 0) ? c->ax : c->alpha_x, cell, F, &st);
  return (int)st.nonphysical;
}

// Midpoint Riemann flux of two states in the x normal.
void oracle_riemann(const oracle_cfg* c, const double* UL, const double* UR, double* F) {
  riemann_flux<double>(UL, UR, c->nvar, *c, c->alpha_x, F);
}

// L(u) on the whole grid.  u, dudt: [nvar][ny][nx] contiguous.  Returns the number of
// interfaces that fell back to first order.
long long oracle_rhs(const oracle_cfg* c, const double* u, double* dudt) {
  Stats st{0, nullptr, 0, 0};
  rhs<double>(*c, u, dudt, &st);
  return st.nonphysical;
}

// Histogram of the weights of every one-sided interpolation in one RHS evaluation
// (App. A statistics).  hist: [2][3][nbins] = (Z weights, final weights) x (w0, w1, w2).
long long oracle_weight_hist(const oracle_cfg* c, const double* u, long long* hist, int nbins) {
  std::vector<double> tmp((size_t)c->nx * ((c->ndim == 2) ? c->ny : 1) * c->nvar);
  Stats st{0, hist, nbins, 0};
  int old = oracle_max_threads();
  oracle_set_threads(1);
  rhs<double>(*c, u, tmp.data(), &st);
  oracle_set_threads(old);
  return st.samples;
}

// L(u) at selected cells.  cells: flattened indices j*nx + i.  out: [ncells][nvar].
void oracle_rhs_cells(const oracle_cfg* c, const double* u, int64_t ncells, const int64_t* cells,
                      double* out) {
  const oracle_cfg cfg = *c;
  const int64_t nx = cfg.nx, ny = (cfg.ndim == 2) ? cfg.ny : 1, plane = nx * ny;
  const int nv = cfg.nvar;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t s = 0; s < ncells; ++s) {
    const int64_t j = cells[s] / nx, i = cells[s] % nx;
    double acc[4] = {0, 0, 0, 0};
    for (int dir = 0; dir < cfg.ndim; ++dir) {
      int perm[4] = {0, 1, 2, 3};
      if (dir == 1 && nv == 4) { perm[1] = 2; perm[2] = 1; }
      const int64_t n = dir == 0 ? nx : ny;
      const int bc = dir == 0 ? cfg.bcx : cfg.bcy;
      const double h = dir == 0 ? cfg.hx : cfg.hy;
      const double al = (cfg.system == 0) ? (dir == 0 ? cfg.ax : cfg.ay) : (dir == 0 ? cfg.alpha_x : cfg.alpha_y);
      auto stored = [&](int64_t m, int v) -> double {
        return dir == 0 ? u[(size_t)perm[v] * plane + j * nx + m] : u[(size_t)perm[v] * plane + m * nx + i];
      };
      auto cell = [&](int64_t m, int v) -> double {
        return line_cell<double>(cfg, dir, dir == 0 ? j : i, m, n, bc, v, stored);
      };
      const int64_t pos = dir == 0 ? i : j;
      double F[6][4];
      for (int k = 0; k < 6; ++k) interface_flux<double>(pos - 3 + k, n, bc, cfg, al, cell, F[k], nullptr);
      for (int v = 0; v < nv; ++v) {
        double a = 0.0;
        if (cfg.family == 1) {
          a = F[3][v] - F[2][v];  // App. B: F_{i+1/2} - F_{i-1/2}
        } else {
          for (int m = 1; m <= 3; ++m) a = a + kD[m - 1] * (F[m + 2][v] - F[3 - m][v]);
        }
        acc[perm[v]] += -(a / h);
      }
    }
    for (int v = 0; v < nv; ++v) out[s * nv + v] = acc[v];
  }
}

void oracle_max_wave(const oracle_cfg* c, const double* u, double* wx, double* wy) { max_wave(*c, u, wx, wy); }

// nsteps TVD-RK3 steps.  dt > 0: fixed step; dt <= 0: CFL step cfl / sum(maxwave/h).
// t_end > 0 clips the step so that t never passes t_end (no further steps once reached).
// Returns the number of steps taken; *t is advanced; *nonphys counts fallbacks.
int oracle_step(const oracle_cfg* c, double* u, double dt, int nsteps, double cfl, double t_end,
                double* t, long long* nonphys) {
  Stats st{0, nullptr, 0, 0};
  int taken = 0;
  double tt = t ? *t : 0.0;
  for (int s = 0; s < nsteps; ++s) {
    double d = dt > 0 ? dt : cfl_dt(*c, u, cfl);
    if (t_end > 0) {
      d = std::min(d, t_end - tt);
      if (!(d > 0)) break;
    }
    oracle_cfg cs = *c;
    cs.time = tt;
    rk3_step<double>(cs, u, d, &st);
    tt = (t_end > 0 && d == t_end - tt) ? t_end : tt + d;
    ++taken;
  }
  if (t) *t = tt;
  if (nonphys) *nonphys = st.nonphysical;
  return taken;
}

// Classical RK4 steps (Eq. 16) with the same dt rules.
int oracle_step_rk4(const oracle_cfg* c, double* u, double dt, int nsteps, double cfl, double t_end,
                    double* t) {
  Stats st{0, nullptr, 0, 0};
  int taken = 0;
  double tt = t ? *t : 0.0;
  for (int s = 0; s < nsteps; ++s) {
    double d = dt > 0 ? dt : cfl_dt(*c, u, cfl);
    if (t_end > 0) {
      d = std::min(d, t_end - tt);
      if (!(d > 0)) break;
    }
    oracle_cfg cs = *c;
    cs.time = tt;
    rk4_step(cs, u, d, &st);
    tt = (t_end > 0 && d == t_end - tt) ? t_end : tt + d;
    ++taken;
  }
  if (t) *t = tt;
  return taken;
}

// Jacobian-vector product of L at u in direction du (forward mode).
void oracle_rhs_jvp(const oracle_cfg* c, const double* u, const double* du, double* L, double* dL) {
  const int64_t n = c->nx * ((c->ndim == 2) ? c->ny : 1) * c->nvar;
  std::vector<Dual> x((size_t)n), y((size_t)n);
  for (int64_t q = 0; q < n; ++q) x[q] = Dual(u[q], du[q]);
  rhs<Dual>(*c, x.data(), y.data(), nullptr);
  for (int64_t q = 0; q < n; ++q) {
    if (L) L[q] = y[q].v;
    dL[q] = y[q].d;
  }
}

// nsteps TVD-RK3 steps with a fixed dt, carrying the tangent du along (forward mode).
void oracle_step_jvp(const oracle_cfg* c, double* u, double* du, double dt, int nsteps) {
  const int64_t n = c->nx * ((c->ndim == 2) ? c->ny : 1) * c->nvar;
  std::vector<Dual> x((size_t)n);
  for (int64_t q = 0; q < n; ++q) x[q] = Dual(u[q], du[q]);
  for (int s = 0; s < nsteps; ++s) rk3_step<Dual>(*c, x.data(), dt, nullptr);
  for (int64_t q = 0; q < n; ++q) {
    u[q] = x[q].v;
    du[q] = x[q].d;
  }
}

// Floating-point operations of one RHS evaluation (single-threaded count).
double oracle_count_rhs_flops(const oracle_cfg* c, const double* u) {
  const int64_t n = c->nx * ((c->ndim == 2) ? c->ny : 1) * c->nvar;
  std::vector<Count> x((size_t)n), y((size_t)n);
  for (int64_t q = 0; q < n; ++q) x[q] = Count(u[q]);
  int old = oracle_max_threads();
  oracle_set_threads(1);
  g_flops = 0.0;
  rhs<Count>(*c, x.data(), y.data(), nullptr);
  oracle_set_threads(old);
  return g_flops;
}

}  // extern "C"
