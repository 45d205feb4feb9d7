// gs_bin_sort_static: the key sort with its scratch in a fixed device array.
//
// Why: gs_bin_sort needs a caller-provided device workspace. Some callers
// cannot allocate device memory where they sort: plug-ins whose host
// application owns every device allocation and hands them only their input
// and output buffers; services that forbid allocation after start-up so that
// their memory use stays fixed; and latency-critical threads that must not
// call cudaMalloc because it can synchronise the device. This entry point
// serves them with scratch that lives in this file: a __device__ array of
// GS_STATIC_SCRATCH_BYTES (64 MiB) that every GPU which loads this code keeps
// until the process exits. The paper has no counterpart.
//
// Host code must not pass g_static_scratch itself to a kernel: on the host
// that name only stands in for the device symbol. Its device address is
// looked up once per device with cudaGetSymbolAddress, with that device
// current, on the first call made on it.
#include <cuda_runtime.h>

#include <mutex>

#include "gs_common.cuh"
#include "gs_internal.h"

namespace gs {
namespace {

static __device__ __align__(256) unsigned char g_static_scratch[GS_STATIC_SCRATCH_BYTES];

std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device (looked up once).
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GS_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return GS_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return GS_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return GS_OK;
}

}  // namespace
}  // namespace gs

extern "C" int gs_bin_sort_static(const float* projected, const int16_t* rects, const uint32_t* counts, int64_t N,
                                  const int32_t* sizes, int32_t V, const gs_config* cfg, uint64_t* keys,
                                  uint32_t* vals, int64_t capacity, uint32_t* tile_ranges, int64_t* n_isect_dev,
                                  int32_t* status_dev, gs_stream_t stream) {
  int64_t n_tiles = 0;
  const int rc = gs_layout_totals(sizes, V, cfg, &n_tiles, nullptr);
  if (rc != GS_OK) return rc;
  // the argument checks of gs_bin_sort come first, so both return the same
  // code for an invalid argument (sizes that no workspace could serve)
  if (N < 0 || capacity < 0 || capacity >= (int64_t(1) << 32) - 1) return GS_ERR_ARG;
  if (N * static_cast<int64_t>(V) >= (int64_t(1) << 32) - 1) return GS_ERR_ARG;
  const size_t need = gs_bin_sort_workspace_bytes(N, V, capacity, n_tiles);
  if (need == 0 || need > static_cast<size_t>(GS_STATIC_SCRATCH_BYTES)) return GS_ERR_TOO_LARGE;
  void* scratch = nullptr;
  const int arc = gs::scratch_address(&scratch);
  if (arc != GS_OK) return arc;
  // gs_bin_sort clears the part of its workspace that must start at zero on
  // every call, so whatever an earlier call left in the array is harmless.
  return gs_bin_sort(projected, rects, counts, nullptr, N, sizes, V, cfg, keys, vals, capacity, tile_ranges, n_isect_dev,
                     scratch, static_cast<size_t>(GS_STATIC_SCRATCH_BYTES), status_dev, stream);
}
