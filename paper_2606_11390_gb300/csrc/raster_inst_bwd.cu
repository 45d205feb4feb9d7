// Backward rasteriser variants without the background term (the default
// zero background): every tile shape and pixels per thread, with 64, 128 and
// 256 splats per shared-memory batch, and 512 where its shared memory fits
// (tiles of at most 4 warps: 8x8, 16x16, 32x16 at 4 pixels per thread).
#include "raster_kernels.cuh"

#define GS_BWD_SET(TW, TH, PPT)                  \
  GS_RASTER_BWD(TW, TH, PPT, 64, false, false)   \
  GS_RASTER_BWD(TW, TH, PPT, 128, false, false)  \
  GS_RASTER_BWD(TW, TH, PPT, 256, false, false)

GS_BWD_SET(8, 8, 2)
GS_BWD_SET(16, 16, 2)
GS_BWD_SET(16, 16, 4)
GS_BWD_SET(32, 16, 2)
GS_BWD_SET(32, 16, 4)
GS_BWD_SET(32, 32, 2)
GS_BWD_SET(32, 32, 4)
GS_RASTER_BWD(8, 8, 2, 512, false, false)
GS_RASTER_BWD(16, 16, 2, 512, false, false)
GS_RASTER_BWD(16, 16, 4, 512, false, false)
GS_RASTER_BWD(32, 16, 4, 512, false, false)
