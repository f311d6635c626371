// Tile groupings the tensor-core rasterizer is instantiated for (k_raster_tc dispatch); the FP32
// rasterizer takes any grouping of 1..TGS_MAX_GROUP tiles per side. Objects that rasterize later
// (frame sequences, the rendering service) check their grouping against this when they are created.
#pragma once

#include "tgs.h"

namespace tgs {

inline bool tc_grouping_supported(int gw, int gh) {
  return (gw == 1 && gh == 1) || (gw == 2 && gh == 2) || (gw == 4 && gh == 2) ||
         (gw == 2 && gh == 4) || (gw == 4 && gh == 4);
}

inline bool grouping_supported(int32_t precision, int gw, int gh) {
  if (gw < 1 || gw > TGS_MAX_GROUP || gh < 1 || gh > TGS_MAX_GROUP) return false;
  return precision == TGS_PRECISION_FP32 || tc_grouping_supported(gw, gh);
}

}  // namespace tgs
