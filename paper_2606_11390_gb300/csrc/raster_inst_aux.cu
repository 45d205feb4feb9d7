// Rasteriser variants at the default batch sizes: the backward with a
// background term, and the pair-counting variants of the forward and the
// backward (the counting backward carries the background term, which is zero
// work when the background is zero).
#include "raster_kernels.cuh"

#define GS_AUX_SET(TW, TH, PPT)                                                              \
  GS_RASTER_BWD(TW, TH, PPT, gs::rast::default_batch_bwd<TW * TH / PPT>(), true, false)  \
  GS_RASTER_BWD(TW, TH, PPT, gs::rast::default_batch_bwd<TW * TH / PPT>(), true, true)   \
  GS_RASTER_FWD(TW, TH, PPT, gs::rast::default_batch_fwd<TW * TH / PPT>(), true)

GS_AUX_SET(8, 8, 2)
GS_AUX_SET(16, 16, 2)
GS_AUX_SET(16, 16, 4)
GS_AUX_SET(32, 16, 2)
GS_AUX_SET(32, 16, 4)
GS_AUX_SET(32, 32, 2)
GS_AUX_SET(32, 32, 4)
