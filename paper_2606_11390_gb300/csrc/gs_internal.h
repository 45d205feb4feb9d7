// Host-side declarations shared by the translation units of libgs_gb300.
#pragma once

#include <cuda_runtime.h>

#include "gs_common.cuh"

namespace gs {

// Validates sizes/cfg and fills a Layout; returns a GS_* code.
int build_layout(const int32_t* sizes, int32_t V, const gs_config* cfg, Layout* L, int64_t* n_pixels);

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Device ordinals that the host-side per-device caches (launch geometry,
// kernel attributes, the static scratch address) keep a slot for.
constexpr int kMaxDevices = 64;

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? GS_OK : GS_ERR_CUDA; }

// Launch of the per-Gaussian backward (defined in project.cu, used by
// gs_rasterize_bwd in raster.cu).
int launch_project_bwd(const float* means, const float* log_scales, const float* quats, const float* opacity_logits,
                       const float* sh, int64_t N, const gs_camera* cams, const Layout& L, const Consts& K,
                       const uint32_t* counts, const float* d_projected, float* d_means, float* d_log_scales,
                       float* d_quats, float* d_opacity_logits, float* d_sh, int32_t* status, cudaStream_t stream);

// Onesweep digit passes over (u32 key, u32 value) pairs (binsort.cu), shared
// with the Morton ordering. A pass p sorts stably by key bits [8p, 8p + 8)
// using the exclusive digit offsets hist[p][256]; pairs alternate between
// keys[0]/vals[0] and keys[1]/vals[1], so after an even number of passes the
// result is back in buffer 0. The item count is read on the device from
// *n_dev (clamped to cap). tickets[passes] and the look-back words
// ((sort_tiles_for(cap) + 1) * 256 per pass) must be zero.
int64_t sort_tiles_for(int64_t n);
void launch_hist_scan(uint32_t* hist, int passes, cudaStream_t stream);
int run_u32_sort_passes(uint32_t* const keys[2], uint32_t* const vals[2], const int64_t* n_dev, int64_t cap,
                        int passes, const uint32_t* hist, uint32_t* tickets, uint64_t* lookback, int32_t* status,
                        cudaStream_t stream);

}  // namespace gs
