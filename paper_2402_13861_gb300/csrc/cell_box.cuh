// Box of one cell of a CellSource (codes of an octree level or a k-d depth, or explicit boxes) as
// a float32 centre and half-width per axis, shared by the float32 bound kernels.
#pragma once

#include "internal.cuh"

namespace isx {

// Box of cell `i` of the source: centre and half-width per axis.
__device__ __forceinline__ void cell_box(const CellSource& s, int64_t i, int inflate, float xc[3],
                                         float h[3]) {
  if (s.codes) {
    uint32_t code = s.codes[i];
    int ijk[3] = {int(code & 1023u), int((code >> 10) & 1023u), int((code >> 20) & 1023u)};
    for (int d = 0; d < 3; ++d) {
      const float size = ldexpf(2.0f, -axis_level(s, d));   // exact dyadic
      float lo = -1.0f + size * float(ijk[d]);      // exact
      h[d] = 0.5f * size;
      xc[d] = lo + h[d];
    }
  } else {
    for (int d = 0; d < 3; ++d) {
      float lo = s.lo[3 * i + d], hi = s.hi[3 * i + d];
      xc[d] = 0.5f * (lo + hi);
      if (inflate) {
        // cover [lo, hi] despite the rounding of xc
        float hu = __fmul_ru(__fsub_ru(hi, lo), 0.5f);
        h[d] = __fadd_ru(hu, fabsf(xc[d]) * 1.2e-7f);
      } else {
        h[d] = 0.5f * (hi - lo);
      }
    }
  }
}

}  // namespace isx
