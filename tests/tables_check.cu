// Host-side dump of the FE-map tables the library hands its kernels (fill_family_tables):
// for each family at kappa = 1/2, one line per table:
//   family name v0 v1 ...
// with name one of ideal, null0, null1, null2, ctrl0, ctrl1, ctrl2.
#include <cstdio>

#include "../paper_2306_09760_gb300/csrc/wcns_device.cuh"

using namespace wcns;

static void line(int family, const char* name, const double* v, int n) {
  std::printf("%d %s", family, name);
  for (int j = 0; j < n; ++j) std::printf(" %.17g", v[j]);
  std::printf("\n");
}

int main() {
  for (int family = 0; family < 2; ++family) {
    Scheme s{};
    fill_family_tables(s, family, 0.5);
    line(family, "ideal", s.ideal, 3);
    line(family, "null0", s.null0, 3);
    line(family, "null1", s.null1, 4);
    line(family, "null2", s.null2, 3);
    line(family, "ctrl0", s.ctrl0, 2);
    line(family, "ctrl1", s.ctrl1, 3);
    line(family, "ctrl2", s.ctrl2, 2);
  }
  return 0;
}
