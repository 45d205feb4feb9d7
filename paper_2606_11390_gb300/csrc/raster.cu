// Tile rasterisation entry points of the C ABI: argument checks and the
// dispatch over tile shape, pixels per thread and splats per shared-memory
// batch to the kernel variants of raster_kernels.cuh (instantiated by the
// raster_inst_*.cu units).
//
// Paper: arXiv 2606.11390 §4 - rasterisation is partitioned per camera (or per
// image tile), and its backward keeps the forward partitioning and sums the
// per-Gaussian gradients with atomics (device scope suffices on one GPU).
#include <cuda_runtime.h>
#include <stdint.h>

#include "gs_common.cuh"
#include "gs_internal.h"
#include "raster_launch.h"

namespace gs {
namespace {

using rast::BwdArgs;
using rast::FwdArgs;

// Pixels per thread: 4 for 16x16, 32x16 and 32x32 tiles unless the
// configuration asks for 2 (GS_FLAG_RASTER_2PX); 8x8 tiles always use 2.
inline int pixels_per_thread(const Layout& L, const Consts& K) {
  if (L.tile_w == 8) return 2;
  return (K.flags & GS_FLAG_RASTER_2PX) ? 2 : 4;
}

// 0 (the default) or a batch size the kernels are instantiated for.
inline bool valid_batch(int32_t b) { return b == 0 || b == 64 || b == 128 || b == 256 || b == 512; }

// The backward's batch must fit a CTA's shared memory (opted in above
// 48 KB); every batch size does on every layout.
inline bool bwd_batch_fits(const Layout& L, int ppt, int32_t b) {
  return b == 0 || rast::bwd_smem_bytes(b, L.tile_w * L.tile_h / ppt / 32) <= rast::kMaxSmem;
}

template <int TW, int TH, int PPT>
int fwd_variant(int32_t batch, bool count, const FwdArgs& a, cudaStream_t s) {
  constexpr int BD = rast::default_batch_fwd<TW * TH / PPT>();
  if (count) return rast::launch_fwd<TW, TH, PPT, BD, true>(a, s);
  const int b = batch ? batch : BD;
  if (b == BD) return rast::launch_fwd<TW, TH, PPT, BD, false>(a, s);
  if (b == 64) return rast::launch_fwd<TW, TH, PPT, 64, false>(a, s);
  if (b == 128) return rast::launch_fwd<TW, TH, PPT, 128, false>(a, s);
  if (b == 256) return rast::launch_fwd<TW, TH, PPT, 256, false>(a, s);
  if (b == 512) return rast::launch_fwd<TW, TH, PPT, 512, false>(a, s);
  return GS_ERR_UNSUPPORTED;
}

// With a non-zero background the backward runs its default batch (the tuned
// sizes are compiled without the background term); results are the same.
template <int TW, int TH, int PPT>
int bwd_variant(int32_t batch, bool bg, bool count, const BwdArgs& a, cudaStream_t s) {
  constexpr int BD = rast::default_batch_bwd<TW * TH / PPT>();
  if (count) return rast::launch_bwd<TW, TH, PPT, BD, true, true>(a, s);
  if (bg) return rast::launch_bwd<TW, TH, PPT, BD, true, false>(a, s);
  const int b = batch ? batch : BD;
  if (b == 64) return rast::launch_bwd<TW, TH, PPT, 64, false, false>(a, s);
  if (b == 128) return rast::launch_bwd<TW, TH, PPT, 128, false, false>(a, s);
  if (b == 256) return rast::launch_bwd<TW, TH, PPT, 256, false, false>(a, s);
  if (b == 512) return rast::launch_bwd<TW, TH, PPT, 512, false, false>(a, s);
  return GS_ERR_UNSUPPORTED;
}

int dispatch_fwd(int ppt, int32_t batch, bool count, const FwdArgs& a, cudaStream_t s) {
  const int tw = a.L.tile_w, th = a.L.tile_h;
  if (tw == 8 && th == 8) return fwd_variant<8, 8, 2>(batch, count, a, s);
  if (tw == 16 && th == 16)
    return ppt == 4 ? fwd_variant<16, 16, 4>(batch, count, a, s) : fwd_variant<16, 16, 2>(batch, count, a, s);
  if (tw == 32 && th == 16)
    return ppt == 4 ? fwd_variant<32, 16, 4>(batch, count, a, s) : fwd_variant<32, 16, 2>(batch, count, a, s);
  if (tw == 32 && th == 32)
    return ppt == 4 ? fwd_variant<32, 32, 4>(batch, count, a, s) : fwd_variant<32, 32, 2>(batch, count, a, s);
  return GS_ERR_UNSUPPORTED;
}

int dispatch_bwd(int ppt, int32_t batch, bool bg, bool count, const BwdArgs& a, cudaStream_t s) {
  const int tw = a.L.tile_w, th = a.L.tile_h;
  if (tw == 8 && th == 8) return bwd_variant<8, 8, 2>(batch, bg, count, a, s);
  if (tw == 16 && th == 16)
    return ppt == 4 ? bwd_variant<16, 16, 4>(batch, bg, count, a, s) : bwd_variant<16, 16, 2>(batch, bg, count, a, s);
  if (tw == 32 && th == 16)
    return ppt == 4 ? bwd_variant<32, 16, 4>(batch, bg, count, a, s) : bwd_variant<32, 16, 2>(batch, bg, count, a, s);
  if (tw == 32 && th == 32)
    return ppt == 4 ? bwd_variant<32, 32, 4>(batch, bg, count, a, s) : bwd_variant<32, 32, 2>(batch, bg, count, a, s);
  return GS_ERR_UNSUPPORTED;
}

int rasterize_fwd_impl(const float* projected, const uint32_t* vals, const uint32_t* tile_ranges, const int32_t* sizes,
                       int32_t V, const gs_config* cfg, float* image, float* final_T, uint32_t* last,
                       const rast::ImageLoss& IL, unsigned long long* counts, uint16_t* cull, cudaStream_t stream) {
  FwdArgs a;
  int rc = build_layout(sizes, V, cfg, &a.L, nullptr);
  if (rc != GS_OK) return rc;
  if (!projected || !tile_ranges || !image || !final_T || !last) return GS_ERR_ARG;
  if (!aligned16(projected) || (reinterpret_cast<uintptr_t>(tile_ranges) & 7u)) return GS_ERR_ARG;
  if (counts && (reinterpret_cast<uintptr_t>(counts) & 7u)) return GS_ERR_ARG;
  if (cull && (reinterpret_cast<uintptr_t>(cull) & 1u)) return GS_ERR_ARG;
  if (!valid_batch(cfg->raster_batch_fwd)) return GS_ERR_UNSUPPORTED;
  a.K = make_consts(*cfg);
  a.projected = reinterpret_cast<const float4*>(projected);
  a.vals = vals;
  a.ranges = reinterpret_cast<const uint2*>(tile_ranges);
  a.order = (a.K.flags & GS_FLAG_TILE_ORDER) ? tile_ranges + 2 * static_cast<size_t>(a.L.n_tiles) : nullptr;
  a.image = image;
  a.final_T = final_T;
  a.last = last;
  a.IL = IL;
  a.counts = counts;
  a.cull = cull;
  return dispatch_fwd(pixels_per_thread(a.L, a.K), cfg->raster_batch_fwd, counts != nullptr, a, stream);
}

int rasterize_bwd_pixels_impl(const float* projected, const uint32_t* vals, const uint32_t* tile_ranges,
                              const int32_t* sizes, int32_t V, const gs_config* cfg, int64_t N, const float* final_T,
                              const uint32_t* last, const float* dL_dimage, float* d_projected,
                              unsigned long long* counts, const uint16_t* cull, cudaStream_t stream) {
  BwdArgs a;
  int rc = build_layout(sizes, V, cfg, &a.L, nullptr);
  if (rc != GS_OK) return rc;
  if (N < 0) return GS_ERR_ARG;
  if (N == 0) return GS_OK;
  if (N * static_cast<int64_t>(V) >= (int64_t(1) << 32)) return GS_ERR_ARG;
  if (!projected || !tile_ranges || !final_T || !last || !dL_dimage || !d_projected) return GS_ERR_ARG;
  if (!aligned16(projected) || (reinterpret_cast<uintptr_t>(tile_ranges) & 7u)) return GS_ERR_ARG;
  if (counts && (reinterpret_cast<uintptr_t>(counts) & 7u)) return GS_ERR_ARG;
  if (cull && (reinterpret_cast<uintptr_t>(cull) & 1u)) return GS_ERR_ARG;
  a.K = make_consts(*cfg);
  if (!valid_batch(cfg->raster_batch_bwd) || !bwd_batch_fits(a.L, pixels_per_thread(a.L, a.K), cfg->raster_batch_bwd))
    return GS_ERR_UNSUPPORTED;
  if (cudaMemsetAsync(d_projected, 0, sizeof(float) * kDRecordFloats * static_cast<size_t>(N) * V, stream) !=
      cudaSuccess)
    return GS_ERR_CUDA;
  a.projected = reinterpret_cast<const float4*>(projected);
  a.vals = vals;
  a.ranges = reinterpret_cast<const uint2*>(tile_ranges);
  a.order = (a.K.flags & GS_FLAG_TILE_ORDER) ? tile_ranges + 2 * static_cast<size_t>(a.L.n_tiles) : nullptr;
  a.final_T = final_T;
  a.last = last;
  a.dL_dimage = dL_dimage;
  a.d_proj = d_projected;
  a.counts = counts;
  a.cull = cull;
  const bool bg = a.K.bg[0] != 0.0f || a.K.bg[1] != 0.0f || a.K.bg[2] != 0.0f;
  return dispatch_bwd(pixels_per_thread(a.L, a.K), cfg->raster_batch_bwd, bg, counts != nullptr, a, stream);
}

}  // namespace
}  // namespace gs

extern "C" int gs_rasterize_fwd(const float* projected, const uint32_t* vals, const uint32_t* tile_ranges,
                                const int32_t* sizes, int32_t V, const gs_config* cfg, float* image, float* final_T,
                                uint32_t* last, uint16_t* cull_masks, gs_stream_t stream) {
  gs::rast::ImageLoss none{};
  return gs::rasterize_fwd_impl(projected, vals, tile_ranges, sizes, V, cfg, image, final_T, last, none, nullptr,
                                cull_masks, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int gs_rasterize_fwd_counted(const float* projected, const uint32_t* vals, const uint32_t* tile_ranges,
                                        const int32_t* sizes, int32_t V, const gs_config* cfg, float* image,
                                        float* final_T, uint32_t* last, uint64_t* pair_counts_dev,
                                        uint16_t* cull_masks, gs_stream_t stream) {
  if (!pair_counts_dev) return GS_ERR_ARG;
  gs::rast::ImageLoss none{};
  return gs::rasterize_fwd_impl(projected, vals, tile_ranges, sizes, V, cfg, image, final_T, last, none,
                                reinterpret_cast<unsigned long long*>(pair_counts_dev), cull_masks,
                                reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int gs_rasterize_fwd_l1l2(const float* projected, const uint32_t* vals, const uint32_t* tile_ranges,
                                     const int32_t* sizes, int32_t V, const gs_config* cfg, float* image,
                                     float* final_T, uint32_t* last, const float* target, int64_t n_values, float w_l1,
                                     float w_l2, int32_t accumulate, float* dL_dimage, double* loss_dev,
                                     uint16_t* cull_masks, gs_stream_t stream_) {
  using namespace gs;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (!target || !dL_dimage || !loss_dev || n_values <= 0) return GS_ERR_ARG;
  int64_t n_pixels = 0;
  int64_t n_tiles = 0;
  const int rc = gs_layout_totals(sizes, V, cfg, &n_tiles, &n_pixels);
  if (rc != GS_OK) return rc;
  if (n_values < 3 * n_pixels) return GS_ERR_ARG;
  if (!valid_batch(cfg->raster_batch_fwd)) return GS_ERR_UNSUPPORTED;
  if (!accumulate && cudaMemsetAsync(loss_dev, 0, sizeof(double), stream) != cudaSuccess) return GS_ERR_CUDA;
  rast::ImageLoss IL;
  IL.target = target;
  IL.grad = dL_dimage;
  IL.loss = loss_dev;
  IL.w1 = w_l1;
  IL.w2 = w_l2;
  IL.inv_n = 1.0f / static_cast<float>(n_values);
  IL.inv_n_d = 1.0 / static_cast<double>(n_values);
  return rasterize_fwd_impl(projected, vals, tile_ranges, sizes, V, cfg, image, final_T, last, IL, nullptr,
                            cull_masks, stream);
}

extern "C" int gs_rasterize_bwd_pixels(const float* projected, const uint32_t* vals, const uint32_t* tile_ranges,
                                       const int32_t* sizes, int32_t V, const gs_config* cfg, int64_t N,
                                       const float* final_T, const uint32_t* last, const float* dL_dimage,
                                       float* d_projected, const uint16_t* cull_masks, gs_stream_t stream) {
  return gs::rasterize_bwd_pixels_impl(projected, vals, tile_ranges, sizes, V, cfg, N, final_T, last, dL_dimage,
                                       d_projected, nullptr, cull_masks, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int gs_rasterize_bwd_pixels_counted(const float* projected, const uint32_t* vals,
                                               const uint32_t* tile_ranges, const int32_t* sizes, int32_t V,
                                               const gs_config* cfg, int64_t N, const float* final_T,
                                               const uint32_t* last, const float* dL_dimage, float* d_projected,
                                               uint64_t* pair_counts_dev, const uint16_t* cull_masks,
                                               gs_stream_t stream) {
  if (!pair_counts_dev) return GS_ERR_ARG;
  return gs::rasterize_bwd_pixels_impl(projected, vals, tile_ranges, sizes, V, cfg, N, final_T, last, dL_dimage,
                                       d_projected, reinterpret_cast<unsigned long long*>(pair_counts_dev),
                                       cull_masks, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int gs_rasterize_bwd(const float* means, const float* log_scales, const float* quats,
                                const float* opacity_logits, const float* sh, int64_t N, const gs_camera* cams_dev,
                                const int32_t* sizes, int32_t V, const gs_config* cfg, const float* projected,
                                const uint32_t* counts, const uint32_t* vals, const uint32_t* tile_ranges,
                                const float* final_T, const uint32_t* last, const float* dL_dimage,
                                float* d_projected, float* d_means, float* d_log_scales, float* d_quats,
                                float* d_opacity_logits, float* d_sh, const uint16_t* cull_masks, int32_t* status_dev,
                                gs_stream_t stream) {
  const int rc = gs_rasterize_bwd_pixels(projected, vals, tile_ranges, sizes, V, cfg, N, final_T, last, dL_dimage,
                                         d_projected, cull_masks, stream);
  if (rc != GS_OK) return rc;
  return gs_project_bwd(means, log_scales, quats, opacity_logits, sh, N, cams_dev, sizes, V, cfg, counts, d_projected,
                        d_means, d_log_scales, d_quats, d_opacity_logits, d_sh, status_dev, stream);
}
