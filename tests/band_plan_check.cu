// Host-side check of the banded 2D stage's work list (make_band_plan, band_decode):
// every x tile and every y tile of the grid is listed exactly once, in the band that
// holds its rows; ring rows stay inside a slot; and every wait of the kernel targets
// items listed before the waiting one (the kernel's progress argument).  Prints "ok"
// or the first failure.
#include <cstdio>
#include <vector>

#include "../paper_2306_09760_gb300/csrc/wcns_internal.h"
#include "../paper_2306_09760_gb300/csrc/wcns_band.cuh"

using namespace wcns;

static int fail(const char* what, long long nx, long long ny, long long a, long long b) {
  std::printf("FAIL %s (grid %lld x %lld): %lld %lld\n", what, nx, ny, a, b);
  return 1;
}

static int check(int64_t nx, int64_t ny, int xtile) {
  GridInfo g{};
  g.ndim = 2; g.nvar = 4; g.nx = nx; g.ny = ny; g.pitch = (nx + 31) / 32 * 32;
  const BandPlan L = make_band_plan(g, xtile);
  const int64_t rows = band_rows(ny);
  if (L.nband < 1 || L.nband > kBandMax) return fail("band count", nx, ny, L.nband, 0);
  if (L.nseg != 2 * L.nband) return fail("segment count", nx, ny, L.nseg, L.nband);
  if (L.row0[0] != 0 || L.row0[L.nband] != ny) return fail("band rows", nx, ny, L.row0[0], L.row0[L.nband]);
  for (int j = 0; j < L.nseg; ++j)
    if (L.seg_start[j + 1] <= L.seg_start[j]) return fail("segment order", nx, ny, j, L.seg_start[j]);
  const int64_t xt = (nx + xtile - 1) / xtile, nty = (ny + kYTile - 1) / kYTile, ycols = (nx + kYCols - 1) / kYCols;
  const int64_t total = L.seg_start[L.nseg];
  if (total != ny * xt + nty * ycols) return fail("item count", nx, ny, total, ny * xt + nty * ycols);
  std::vector<int> xseen(ny * xt, 0), yseen(nty * ycols, 0);
  std::vector<long long> xfirst(L.nband, -1), xlast(L.nband, -1), yfirst(L.nband, -1), ylast(L.nband, -1);
  for (int item = 0; item < total; ++item) {
    int kind, b;
    int64_t p0, p1;
    band_decode(L, item, kind, b, p0, p1);
    if (b < 0 || b >= L.nband) return fail("band of item", nx, ny, item, b);
    if (kind == 0) {
      if (p0 < L.row0[b] || p0 >= L.row0[b + 1] || p1 < 0 || p1 >= xt) return fail("x tile", nx, ny, p0, p1);
      if (p0 - L.row0[b] >= rows) return fail("x ring row", nx, ny, p0, b);
      if (xseen[p0 * xt + p1]++) return fail("x tile twice", nx, ny, p0, p1);
      if (xfirst[b] < 0) xfirst[b] = item;
      xlast[b] = item;
    } else {
      if (p0 < 0 || p0 >= ycols || p1 < 0 || p1 >= nty) return fail("y tile", nx, ny, p0, p1);
      const int64_t r0 = p1 * kYTile, r1 = std::min<int64_t>(r0 + kYTile, ny);
      if (r0 < L.row0[b] || r1 > L.row0[b + 1]) return fail("y tile rows", nx, ny, r0, b);
      if (r1 - L.row0[b] > rows) return fail("y ring row", nx, ny, r1, b);
      if (yseen[p1 * ycols + p0]++) return fail("y tile twice", nx, ny, p0, p1);
      if (yfirst[b] < 0) yfirst[b] = item;
      ylast[b] = item;
    }
  }
  for (int64_t k = 0; k < ny * xt; ++k)
    if (xseen[k] != 1) return fail("x tile missing", nx, ny, k / xt, k % xt);
  for (int64_t k = 0; k < nty * ycols; ++k)
    if (yseen[k] != 1) return fail("y tile missing", nx, ny, k % ycols, k / ycols);
  for (int b = 0; b < L.nband; ++b) {
    if ((int64_t)L.x_items[b] != xlast[b] - xfirst[b] + 1) return fail("x items of band", nx, ny, b, L.x_items[b]);
    if ((int64_t)L.y_items[b] != ylast[b] - yfirst[b] + 1) return fail("y items of band", nx, ny, b, L.y_items[b]);
    // y tiles of band b wait on the x tiles of band b
    if (yfirst[b] <= xlast[b]) return fail("y before its x tiles", nx, ny, b, yfirst[b]);
    // x tiles of band b wait on the y tiles of band b - kBandRing (ring slot reuse)
    if (b >= kBandRing && ylast[b - kBandRing] >= xfirst[b]) return fail("x before slot is free", nx, ny, b, xfirst[b]);
    if (L.slot_vstride != rows * g.pitch || L.slot_elems != 4 * L.slot_vstride)
      return fail("slot size", nx, ny, L.slot_vstride, L.slot_elems);
  }
  return 0;
}

int main() {
  const int64_t sizes[][3] = {{2048, 2048, 1019}, {2048, 700, 1019}, {1300, 1000, 1019}, {700, 900, 251},
                              {2048, 640, 1019}, {3057, 751, 1019}, {64, 601, 251},  {5000, 30000, 1019},
                              {16, 4800, 251},   {9000, 4801, 251}, {2048, 4096, 1019}};
  for (const auto& s : sizes)
    if (check(s[0], s[1], (int)s[2])) return 1;
  std::printf("ok\n");
  return 0;
}
