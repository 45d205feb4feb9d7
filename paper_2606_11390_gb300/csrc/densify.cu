// Densification statistics gathered during training.
//
// Paper: arXiv 2606.11390 §5.2 densifies (Kerbl et al. 2023) to much larger
// Gaussian counts during training; the densification decisions rest on two
// per-Gaussian statistics that the backward pass can emit for free: the
// accumulated norm of the loss gradient with respect to the Gaussian's
// screen-space position, and its largest screen-space radius.
//
// Per Gaussian g and every view v where g is visible (tile count > 0):
//   grad_accum[g] += || (dL/dmean2d.x * W_v / 2, dL/dmean2d.y * H_v / 2) ||
//   denom[g]      += 1
//   max_radii[g]   = max(max_radii[g], radius of g in v, in pixels)
// The factors W/2, H/2 turn the pixel-space gradient into the gradient with
// respect to normalised device coordinates, so the statistic does not depend
// on the image resolution. One thread per Gaussian loops over the views, so
// there are no atomics and the result is deterministic.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "gs_common.cuh"
#include "gs_internal.h"

namespace gs {
namespace {

constexpr int kDensifyThreads = 256;
constexpr int kMaxDensifyViews = 64;

struct HalfSizes {
  float hw[kMaxDensifyViews], hh[kMaxDensifyViews];
};

__global__ void __launch_bounds__(kDensifyThreads) densify_stats_kernel(
    const float* __restrict__ projected, const uint32_t* __restrict__ counts, const float* __restrict__ d_projected,
    int64_t N, int V, const HalfSizes hs, float* __restrict__ grad_accum, float* __restrict__ denom,
    float* __restrict__ max_radii) {
  const int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (g >= N) return;
  float acc = 0.0f, seen = 0.0f, rmax = 0.0f;
  for (int v = 0; v < V; ++v) {
    const int64_t r = static_cast<int64_t>(v) * N + g;
    if (counts[r] == 0) continue;
    const float gx = d_projected[9 * r + 0] * hs.hw[v];
    const float gy = d_projected[9 * r + 1] * hs.hh[v];
    acc += sqrtf(gx * gx + gy * gy);
    seen += 1.0f;
    rmax = fmaxf(rmax, projected[12 * r + 7]);
  }
  if (seen > 0.0f) {
    grad_accum[g] += acc;
    denom[g] += seen;
    max_radii[g] = fmaxf(max_radii[g], rmax);
  }
}

}  // namespace
}  // namespace gs

extern "C" int gs_densify_stats(const float* projected, const uint32_t* counts, const float* d_projected, int64_t N,
                                const int32_t* sizes, int32_t V, float* grad_accum, float* denom, float* max_radii,
                                gs_stream_t stream_) {
  using namespace gs;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (N < 0 || V < 1 || V > kMaxDensifyViews || !sizes) return GS_ERR_ARG;
  if (N == 0) return GS_OK;
  if (!projected || !counts || !d_projected || !grad_accum || !denom || !max_radii) return GS_ERR_ARG;
  HalfSizes hs;
  for (int v = 0; v < V; ++v) {
    if (sizes[2 * v] < 1 || sizes[2 * v + 1] < 1) return GS_ERR_ARG;
    hs.hw[v] = 0.5f * static_cast<float>(sizes[2 * v]);
    hs.hh[v] = 0.5f * static_cast<float>(sizes[2 * v + 1]);
  }
  const int64_t grid = (N + kDensifyThreads - 1) / kDensifyThreads;
  if (grid > 0x7fffffff) return GS_ERR_ARG;
  densify_stats_kernel<<<static_cast<unsigned>(grid), kDensifyThreads, 0, stream>>>(
      projected, counts, d_projected, N, V, hs, grad_accum, denom, max_radii);
  return cuda_status(cudaGetLastError());
}
