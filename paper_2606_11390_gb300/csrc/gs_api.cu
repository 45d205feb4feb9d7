// Host-side pieces of the C ABI shared by all entry points: version, status
// text and the view-layout builder.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gs_common.cuh"
#include "gs_internal.h"

namespace gs {

int build_layout(const int32_t* sizes, int32_t V, const gs_config* cfg, Layout* L, int64_t* n_pixels) {
  if (!sizes || !cfg || !L) return GS_ERR_ARG;
  if (V < 1 || V > kMaxViews) return GS_ERR_ARG;
  const int tw = cfg->tile_w, th = cfg->tile_h;
  if (!((tw == 8 && th == 8) || (tw == 16 && th == 16) || (tw == 32 && th == 16) || (tw == 32 && th == 32)))
    return GS_ERR_UNSUPPORTED;
  L->V = V;
  L->tile_w = tw;
  L->tile_h = th;
  uint64_t tiles = 0, pix = 0;
  for (int v = 0; v < V; ++v) {
    const int W = sizes[2 * v], H = sizes[2 * v + 1];
    if (W <= 0 || H <= 0 || W > 32767 * 8 || H > 32767 * 8) return GS_ERR_ARG;
    L->width[v] = W;
    L->height[v] = H;
    L->ntx[v] = (W + tw - 1) / tw;
    L->nty[v] = (H + th - 1) / th;
    if (L->ntx[v] > 32767 || L->nty[v] > 32767) return GS_ERR_ARG;
    L->tile_base[v] = static_cast<uint32_t>(tiles);
    L->pix_base[v] = static_cast<uint32_t>(pix);
    tiles += static_cast<uint64_t>(L->ntx[v]) * L->nty[v];
    pix += static_cast<uint64_t>(W) * H;
    if (tiles >= (1ull << 31) || pix >= (1ull << 32)) return GS_ERR_ARG;
  }
  for (int v = V; v <= kMaxViews; ++v) {
    if (v < kMaxViews) {
      L->width[v] = L->height[v] = L->ntx[v] = L->nty[v] = 0;
    }
    L->tile_base[v] = static_cast<uint32_t>(tiles);
    L->pix_base[v] = static_cast<uint32_t>(pix);
  }
  L->n_tiles = static_cast<int32_t>(tiles);
  if (n_pixels) *n_pixels = static_cast<int64_t>(pix);
  return GS_OK;
}

}  // namespace gs

extern "C" int gs_version(void) { return 400; }  // 0.4.0: cull masks handed from the raster forward to its backward

extern "C" const char* gs_status_string(int code) {
  switch (code) {
    case GS_OK: return "ok";
    case GS_ERR_ARG: return "invalid argument";
    case GS_ERR_CUDA: return "CUDA error while enqueuing";
    case GS_ERR_UNSUPPORTED: return "unsupported configuration";
    case GS_ERR_TOO_LARGE: return "problem too large for the static scratch of gs_bin_sort_static";
    default: break;
  }
  return "device status bits set (capacity / timeout / bounds)";
}

extern "C" int gs_layout_totals(const int32_t* sizes, int32_t V, const gs_config* cfg, int64_t* n_tiles,
                                int64_t* n_pixels) {
  gs::Layout L;
  int64_t pix = 0;
  const int rc = gs::build_layout(sizes, V, cfg, &L, &pix);
  if (rc != GS_OK) return rc;
  if (n_tiles) *n_tiles = L.n_tiles;
  if (n_pixels) *n_pixels = pix;
  return GS_OK;
}
