// Backward rasteriser variants without the background term (the default
// zero background): every tile shape and pixels per thread, with 64, 128,
// 256 and 512 splats per shared-memory batch (above 48 KB of shared memory,
// as for 512 splats on tiles of more than 4 warps, the launch opts in).
#include "raster_kernels.cuh"

#define GS_BWD_SET(TW, TH, PPT)                  \
  GS_RASTER_BWD(TW, TH, PPT, 64, false, false)   \
  GS_RASTER_BWD(TW, TH, PPT, 128, false, false)  \
  GS_RASTER_BWD(TW, TH, PPT, 256, false, false)  \
  GS_RASTER_BWD(TW, TH, PPT, 512, false, false)

GS_BWD_SET(8, 8, 2)
GS_BWD_SET(16, 16, 2)
GS_BWD_SET(16, 16, 4)
GS_BWD_SET(32, 16, 2)
GS_BWD_SET(32, 16, 4)
GS_BWD_SET(32, 32, 2)
GS_BWD_SET(32, 32, 4)
