// Test tool: the library's double-precision interface numerics (wcns_device.cuh) and their
// reverse sweep (wcns_adjoint.cuh) compiled
// for the host, behind a C interface the CPU tests load with ctypes.  On the host the
// divisions are IEEE divisions and the comparisons plain ones (the device build uses
// Newton reciprocals and bit-pattern compares), so results agree with the device up to
// rounding; the tests compare them with the oracle interface by interface.
#include "../paper_2306_09760_gb300/csrc/wcns_device.cuh"
#include "../paper_2306_09760_gb300/csrc/wcns_adjoint.cuh"

using namespace wcns;

static SchemeT<double> make_scheme(int system, int weights, int flux, int characteristic, int zp, int family,
                                   double xi, double eps, double alpha) {
  Scheme s{};
  s.system = system; s.weights = weights; s.flux = flux; s.characteristic = characteristic; s.zp = zp;
  s.renorm = 1; s.gamma = 1.4; s.eps = eps; s.xi = xi; s.cv = 1e-3; s.harten = 0.1;
  s.speed[0] = alpha; s.speed[1] = alpha;
  fill_family_tables(s, family, 0.5);
  return scheme_as<double>(s);
}

template <int NV, int FIX>
static int flux_nv(const SchemeT<double>& st, const double* S, double* F) {
  double SS[6][NV], FF[NV];
  for (int m = 0; m < 6; ++m)
    for (int k = 0; k < NV; ++k) SS[m][k] = S[m * NV + k];
  const bool fb = interface_flux<double, NV, FIX>(SS, st, 0, FF);
  for (int k = 0; k < NV; ++k) F[k] = FF[k];
  return fb ? 1 : 0;
}

template <int NV>
static void vjp_nv(const SchemeT<double>& st, const double* S, const double* Fb, double* Sb) {
  double SS[6][NV], FB[NV], SB[6][NV];
  for (int m = 0; m < 6; ++m)
    for (int k = 0; k < NV; ++k) { SS[m][k] = S[m * NV + k]; SB[m][k] = 0.0; }  // the sweep adds into SB
  for (int k = 0; k < NV; ++k) FB[k] = Fb[k];
  interface_flux_vjp<double, NV>(SS, st, 0, FB, SB);
  for (int m = 0; m < 6; ++m)
    for (int k = 0; k < NV; ++k) Sb[m * NV + k] = SB[m][k];
}

extern "C" {

// Midpoint flux of the interface between cells 2 and 3 of S[6][nvar] (x normal): Euler
// for nvar = 3 or 4 (alpha: the frozen Lax-Friedrichs speed), scalar advection with speed
// alpha for nvar = 1; run-time options (fixed = 0) or the compiled default configuration
// (fixed = 1, Euler only).  Returns 1 if the interface fell back to (U_i, U_{i+1}), -1 on
// an unsupported nvar.
int host_interface_flux(int nvar, int weights, int flux, int characteristic, int zp, int family, double xi,
                        double eps, double alpha, int fixed, const double* S, double* F) {
  const SchemeT<double> st =
      make_scheme(nvar == 1 ? 0 : 1, weights, flux, characteristic, zp, family, xi, eps, alpha);
  if (nvar == 1) return flux_nv<1, 0>(st, S, F);
  if (nvar == 3) return fixed ? flux_nv<3, 1>(st, S, F) : flux_nv<3, 0>(st, S, F);
  if (nvar == 4) return fixed ? flux_nv<4, 1>(st, S, F) : flux_nv<4, 0>(st, S, F);
  return -1;
}

// One-sided midpoint interpolation of v[0..4] (WCNS family): the value, and the base and
// final weights in wz[3], wf[3].
double host_weno_side(int weights, int zp, double xi, double eps, const double* v, double* wz, double* wf) {
  const SchemeT<double> st = make_scheme(0, weights, 0, 0, zp, 0, xi, eps, 0.0);
  return weno_side<double, 0>(v[0], v[1], v[2], v[3], v[4], st, wz, wf);
}

// Reverse sweep of the interface flux: Sb[6][nvar] = (dF/dS)^T Fb for the flux of
// host_interface_flux with the same options.  Returns -1 on an unsupported nvar.
int host_interface_flux_vjp(int nvar, int weights, int flux, int characteristic, int zp, double xi, double eps,
                            double alpha, const double* S, const double* Fb, double* Sb) {
  const SchemeT<double> st = make_scheme(1, weights, flux, characteristic, zp, 0, xi, eps, alpha);
  if (nvar == 3) { vjp_nv<3>(st, S, Fb, Sb); return 0; }
  if (nvar == 4) { vjp_nv<4>(st, S, Fb, Sb); return 0; }
  return -1;
}

// Ghost or interior value of component v at cell m of line `line` in direction dir, with
// the boundary faces types[4] (x-lo, x-hi, y-lo, y-hi; active if any is not the grid's bc)
// and their states ua, ub (conservative, storage ordering), at the state's time.
double host_face_cell(const double* u, int64_t pitch, int64_t fstride, int dir, int64_t line, int64_t m, int64_t n,
                      int bc, int v, const int* types, const double* ua, const double* ub, double wall_x, double x0,
                      double dxdy, double speed, double lo_x, double lo_y, double hx, double hy, double time) {
  Faces<double> f{};
  for (int k = 0; k < 4; ++k) {
    f.type[k] = types[k];
    f.ua[k] = ua[k];
    f.ub[k] = ub[k];
    if (types[k] != kFaceGrid) f.active = 1;
  }
  f.wall_x = wall_x; f.x0 = x0; f.dxdy = dxdy; f.speed = speed;
  f.lo_x = lo_x; f.lo_y = lo_y; f.hx = hx; f.hy = hy;
  return face_cell<double>(u, pitch, fstride, dir, line, m, n, bc, v, f, time);
}

// Eq. 3 (WCNS family) or the two-point difference (WENO family) of six midpoint fluxes
// f[0..5] = F_{i-5/2} .. F_{i+5/2}, divided by h = 1 / inv_h.
double host_flux_difference(int family, const double* f, double inv_h) {
  return flux_difference_family<double>(family, f[0], f[1], f[2], f[3], f[4], f[5], inv_h);
}

}  // extern "C"
