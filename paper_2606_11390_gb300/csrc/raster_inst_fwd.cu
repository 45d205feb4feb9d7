// Forward rasteriser variants: every tile shape and pixels per thread, with
// 64, 128, 256 and 512 splats per shared-memory batch.
#include "raster_kernels.cuh"

#define GS_FWD_SET(TW, TH, PPT)            \
  GS_RASTER_FWD(TW, TH, PPT, 64, false)   \
  GS_RASTER_FWD(TW, TH, PPT, 128, false)  \
  GS_RASTER_FWD(TW, TH, PPT, 256, false)  \
  GS_RASTER_FWD(TW, TH, PPT, 512, false)

GS_FWD_SET(8, 8, 2)
GS_FWD_SET(16, 16, 2)
GS_FWD_SET(16, 16, 4)
GS_FWD_SET(32, 16, 2)
GS_FWD_SET(32, 16, 4)
GS_FWD_SET(32, 32, 2)
GS_FWD_SET(32, 32, 4)
