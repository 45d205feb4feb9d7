// Morton (Z-order) ordering of Gaussians in 3D and row gathers.
//
// Paper: arXiv 2606.11390 §5.2 sorts the Gaussians along a three-dimensional
// Morton curve (Morton 1966, as in LiteGS) during densification, so that
// Gaussians near each other in space sit near each other in memory; the
// rasteriser's gathers of projected records and its gradient atomics then
// touch fewer distinct cache lines. The paper reports 5-10 %.
//
// The order: lo/hi = per-axis minimum/maximum of the means; each coordinate
// is quantised to 10 bits, q = clamp(floor((x - lo) * (1024 / (hi - lo))),
// 0, 1023), evaluated as single rounded float operations in that order (q = 0
// on an axis with hi == lo); the 30-bit code interleaves the bits of
// (qx, qy, qz) with x in the lowest position; the permutation is the stable
// sort of the codes (ties in index order), done with the onesweep digit passes
// of the tile sort. A caller applies it with gs_gather_rows to every
// per-Gaussian array.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gs_common.cuh"
#include "gs_internal.h"

namespace gs {
namespace {

constexpr int kMortonThreads = 256;
constexpr int kMortonPasses = 4;  // 30 code bits in 8-bit digits
constexpr int kMortonRadix = 256;

// Monotone map of floats to unsigned integers (order-preserving), so the
// bounding box can be reduced with integer atomics on a zeroed buffer: max
// via atomicMax of the key, min via atomicMax of its complement.
__device__ __forceinline__ uint32_t order_key(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float from_order_key(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// bbox[0..2] = complement keys of the minima, bbox[3..5] = keys of the maxima.
__global__ void __launch_bounds__(kMortonThreads) bbox_kernel(const float* __restrict__ means, int64_t N,
                                                              uint32_t* __restrict__ bbox) {
  uint32_t mn[3] = {0u, 0u, 0u}, mx[3] = {0u, 0u, 0u};
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const uint32_t k = order_key(means[3 * i + a]);
      mn[a] = max(mn[a], ~k);
      mx[a] = max(mx[a], k);
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mn[a] = max(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
      mx[a] = max(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
    }
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      atomicMax(&bbox[a], mn[a]);
      atomicMax(&bbox[3 + a], mx[a]);
    }
  }
}

// Spreads the low 10 bits of v to every third bit (bit b -> bit 3b).
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__device__ __forceinline__ uint32_t quantise(float x, float lo, float scale) {
  if (!(scale > 0.0f)) return 0u;
  const float t = __fmul_rn(__fsub_rn(x, lo), scale);
  const float f = floorf(t);
  if (!(f > 0.0f)) return 0u;  // also a NaN coordinate
  return f >= 1023.0f ? 1023u : static_cast<uint32_t>(f);
}

// Codes and identity values, plus the digit histograms of all passes.
__global__ void __launch_bounds__(kMortonThreads) morton_codes_kernel(const float* __restrict__ means, int64_t N,
                                                                      const uint32_t* __restrict__ bbox,
                                                                      uint32_t* __restrict__ codes,
                                                                      uint32_t* __restrict__ idx,
                                                                      uint32_t* __restrict__ hist,
                                                                      int64_t* __restrict__ n_dev) {
  __shared__ uint32_t s_hist[kMortonPasses][kMortonRadix];
  __shared__ float s_lo[3], s_scale[3];
  for (int i = threadIdx.x; i < kMortonPasses * kMortonRadix; i += blockDim.x) (&s_hist[0][0])[i] = 0u;
  if (threadIdx.x < 3) {
    const int a = threadIdx.x;
    const float lo = from_order_key(~bbox[a]), hi = from_order_key(bbox[3 + a]);
    const float ext = __fsub_rn(hi, lo);
    s_lo[a] = lo;
    s_scale[a] = ext > 0.0f ? __fdiv_rn(1024.0f, ext) : 0.0f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_dev = N;
  __syncthreads();
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint32_t qx = quantise(means[3 * i + 0], s_lo[0], s_scale[0]);
    const uint32_t qy = quantise(means[3 * i + 1], s_lo[1], s_scale[1]);
    const uint32_t qz = quantise(means[3 * i + 2], s_lo[2], s_scale[2]);
    const uint32_t code = spread3(qx) | (spread3(qy) << 1) | (spread3(qz) << 2);
    codes[i] = code;
    idx[i] = static_cast<uint32_t>(i);
#pragma unroll
    for (int p = 0; p < kMortonPasses; ++p) atomicAdd(&s_hist[p][(code >> (8 * p)) & 0xffu], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kMortonPasses * kMortonRadix; i += blockDim.x) {
    const uint32_t c = (&s_hist[0][0])[i];
    if (c) atomicAdd(&hist[i], c);
  }
}

// dst[i] = src[perm[i]], rows of `row` floats; 16-byte rows move as float4.
__global__ void gather_rows_kernel(const float* __restrict__ src, float* __restrict__ dst, int64_t n_rows, int row,
                                   const uint32_t* __restrict__ perm, int64_t n_src, int32_t* __restrict__ status) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  if ((row & 3) == 0) {
    const int r4 = row >> 2;
    const int64_t total = n_rows * r4;
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += stride) {
      const int64_t i = e / r4;
      const int k = static_cast<int>(e - i * r4);
      const uint32_t j = perm[i];
      if (j < n_src) d4[e] = s4[static_cast<int64_t>(j) * r4 + k];
      else set_status(status, GS_STATUS_BOUNDS);
    }
  } else {
    const int64_t total = n_rows * row;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += stride) {
      const int64_t i = e / row;
      const int k = static_cast<int>(e - i * row);
      const uint32_t j = perm[i];
      if (j < n_src) dst[e] = src[static_cast<int64_t>(j) * row + k];
      else set_status(status, GS_STATUS_BOUNDS);
    }
  }
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct MortonWs {
  size_t keys0, keys1, vals1, zero_begin, bbox, hist, tickets, n, lookback, zero_end, total;
};

MortonWs morton_ws(int64_t N) {
  MortonWs w;
  const size_t n = static_cast<size_t>(N > 0 ? N : 1);
  size_t o = 0;
  w.keys0 = o; o = align256(o + 4 * n);
  w.keys1 = o; o = align256(o + 4 * n);
  w.vals1 = o; o = align256(o + 4 * n);
  w.zero_begin = o;
  w.bbox = o; o = align256(o + 4 * 6);
  w.hist = o; o = align256(o + 4 * kMortonPasses * kMortonRadix);
  w.tickets = o; o = align256(o + 4 * kMortonPasses);
  w.n = o; o = align256(o + 8);
  w.lookback = o;
  o = align256(o + 8 * static_cast<size_t>(kMortonRadix) * kMortonPasses * static_cast<size_t>(sort_tiles_for(N) + 1));
  w.zero_end = o;
  w.total = o;
  return w;
}

int grid_for(int64_t work, int threads) {
  int64_t g = (work + threads - 1) / threads;
  if (g > 4096) g = 4096;
  return static_cast<int>(g > 0 ? g : 1);
}

}  // namespace
}  // namespace gs

extern "C" size_t gs_morton_workspace_bytes(int64_t N) {
  if (N < 0) return 0;
  return gs::morton_ws(N).total;
}

extern "C" int gs_morton_order(const float* means, int64_t N, uint32_t* perm, uint32_t* codes, void* workspace,
                               size_t workspace_bytes, int32_t* status_dev, gs_stream_t stream_) {
  using namespace gs;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (N < 0 || N >= (int64_t(1) << 32) - 1) return GS_ERR_ARG;
  if (N == 0) return GS_OK;
  if (!means || !perm || !workspace || !status_dev) return GS_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(workspace) & 255u) return GS_ERR_ARG;
  const MortonWs w = morton_ws(N);
  if (workspace_bytes < w.total) return GS_ERR_ARG;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  auto u32 = [&](size_t off) { return reinterpret_cast<uint32_t*>(ws + off); };
  if (cudaMemsetAsync(ws + w.zero_begin, 0, w.zero_end - w.zero_begin, stream) != cudaSuccess) return GS_ERR_CUDA;
  // after four passes the pairs are back in buffer 0: the caller's arrays
  uint32_t* keys[2] = {codes ? codes : u32(w.keys0), u32(w.keys1)};
  uint32_t* vals[2] = {perm, u32(w.vals1)};
  uint32_t* bbox = u32(w.bbox);
  uint32_t* hist = u32(w.hist);
  int64_t* n_dev = reinterpret_cast<int64_t*>(ws + w.n);
  bbox_kernel<<<grid_for(N, kMortonThreads), kMortonThreads, 0, stream>>>(means, N, bbox);
  morton_codes_kernel<<<grid_for(N, kMortonThreads), kMortonThreads, 0, stream>>>(means, N, bbox, keys[0], vals[0],
                                                                                  hist, n_dev);
  launch_hist_scan(hist, kMortonPasses, stream);
  return run_u32_sort_passes(keys, vals, n_dev, N, kMortonPasses, hist, u32(w.tickets),
                             reinterpret_cast<uint64_t*>(ws + w.lookback), status_dev, stream);
}

extern "C" int gs_gather_rows(const float* src, float* dst, int64_t n_rows, int32_t row_floats, const uint32_t* perm,
                              int32_t* status_dev, gs_stream_t stream_) {
  using namespace gs;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (n_rows < 0 || row_floats < 1) return GS_ERR_ARG;
  if (n_rows == 0) return GS_OK;
  if (!src || !dst || !perm || !status_dev || src == dst) return GS_ERR_ARG;
  if ((row_floats & 3) == 0 && (!aligned16(src) || !aligned16(dst))) return GS_ERR_ARG;
  gather_rows_kernel<<<grid_for(n_rows * row_floats / ((row_floats & 3) == 0 ? 4 : 1), 256), 256, 0, stream>>>(
      src, dst, n_rows, row_floats, perm, n_rows, status_dev);
  return cuda_status(cudaGetLastError());
}
