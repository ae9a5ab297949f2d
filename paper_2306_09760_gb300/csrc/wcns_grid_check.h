// Layout checks of a wcns_grid descriptor shared by every entry point that reads one:
// element type, dimensions, row pitch and total size.  wcns_init adds the checks that
// only a solver needs (variable count per system, domain, boundaries).
#pragma once

#include <cstdint>

#include "../../include/wcns.h"

namespace wcns {

// Largest cell count per direction.
constexpr int64_t kMaxCellsPerDir = (int64_t)1 << 26;

// WCNS_OK if (ndim, dtype, reserved, nx, ny, pitch) describe a grid buffer the kernels
// can address: 1 <= nx, ny <= 2^26; at most 65535 * 43 rows (65535 independent lines
// when ndim = 1); pitch >= nx and a multiple of 32 elements; nvar * ny * pitch <= 4e9
// elements.  nvar itself is checked by the caller.
inline wcns_status check_grid_layout(const wcns_grid& g) {
  if (g.ndim != 1 && g.ndim != 2) return WCNS_ERR_ARG;
  if (g.dtype != WCNS_F64 && g.dtype != WCNS_F32) return WCNS_ERR_ARG;
  if (g.reserved != 0) return WCNS_ERR_ARG;
  if (g.nx < 1 || g.ny < 1 || g.nx > kMaxCellsPerDir || g.ny > kMaxCellsPerDir) return WCNS_ERR_ARG;
  // ndim 1 with ny > 1: ny independent lines of nx cells (rows are not coupled)
  if (g.ny > 65535 * (int64_t)43 || (g.ndim == 1 && g.ny > 65535)) return WCNS_ERR_ARG;
  if (g.pitch < g.nx || g.pitch % 32 != 0) return WCNS_ERR_ARG;
  if (g.nvar < 1 || (double)g.nvar * (double)g.ny * (double)g.pitch > 4.0e9) return WCNS_ERR_ARG;
  return WCNS_OK;
}

}  // namespace wcns
