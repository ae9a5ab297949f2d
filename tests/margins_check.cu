// Host-side dump of the FE ideal-plateau margins (SchemeT::ideal_margin, ideal_ratio) that
// the library derives from a scheme's control rows, for the test that checks them against
// the oracle's evaluation of Eq. 20.  One line per (precision, family, xi, kappa, weights):
//   bytes family xi kappa weights m0 m1 m2 ratio sat_dist
#include <cstdio>

#include "../paper_2306_09760_gb300/csrc/wcns_device.cuh"

using namespace wcns;

template <typename T>
static void row(int family, double xi, double kappa, int weights) {
  Scheme s{};
  s.system = 1; s.weights = weights; s.flux = 2; s.characteristic = 1; s.zp = 1; s.renorm = 1;
  s.gamma = 1.4; s.eps = 1e-40; s.xi = xi; s.cv = 1e-3; s.harten = 0.1;
  fill_family_tables(s, family, kappa);
  const SchemeT<T> r = scheme_as<T>(s);
  std::printf("%d %d %.17g %.17g %d %.17g %.17g %.17g %.17g %.17g\n", (int)sizeof(T), family, xi, kappa, weights,
              (double)r.ideal_margin[0], (double)r.ideal_margin[1], (double)r.ideal_margin[2], (double)r.ideal_ratio,
              (double)r.sat_dist);
}

int main() {
  const double xis[] = {100.0, 1e3, 1e4, 1e5, 1e6, 1e8};
  for (int family = 0; family < 2; ++family)
    for (double xi : xis)
      for (double kappa : {0.5, 0.3})
        for (int weights : {2, 3}) {
          row<float>(family, xi, kappa, weights);
          row<double>(family, xi, kappa, weights);
        }
  return 0;
}
